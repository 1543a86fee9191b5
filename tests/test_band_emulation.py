"""The per-term constant of the score kernel's error bound, checked by
emulating the kernel's FP32 arithmetic on the CPU.

The band derivation (tests/_band.py) bounds the FP32 value of one support
point's sum of RQ summands (Eq. 3 inside the FK kernel of Eq. 4), computed
from FP32 control points p and s, by (max(15u + rho, 10u + 2 rho) + (Mv - NP) u)
relative to its exact value from the same inputs, u = 2^-24, rho = 2^-23 the
reciprocal's error.  Here the kernel's operation sequence is replayed with
every FP32 rounding emulated (products and sums rounded to the nearest FP32,
fused multiply-adds rounded once) and the reciprocal replaced by its worst
admissible value (the FP32 neighbour of 1/x on the far side, an error just
below one ulp), on random control points spread like the 7-DOF and 12-point
workloads and on near-coincident ones.  The largest relative error must stay
within the derived constant.
"""
import numpy as np
import pytest

U = 2.0 ** -24
RHO = 2.0 ** -23

F32 = np.float32
LD = np.longdouble  # 64-bit or wider significand: FP32 products are exact in it


def rn(x):
    """Round to the nearest FP32 value."""
    return np.asarray(x, dtype=LD).astype(np.float32)


def fma(a, b, c):
    """FP32 fused multiply-add: the exact a b + c rounded once (the sum is formed
    in long double, whose extra bits make the double rounding negligible here)."""
    return rn(LD(1) * np.asarray(a, dtype=LD) * np.asarray(b, dtype=LD) + np.asarray(c, dtype=LD))


def rcp_worst(x):
    """A reciprocal with an error just below one ulp: the FP32 neighbour of
    1/x on the far side of the exact value."""
    exact = LD(1) / np.asarray(x, dtype=LD)
    r = rn(exact)
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(0))
    return np.where(np.abs(up.astype(LD) - exact) > np.abs(dn.astype(LD) - exact), up, dn).astype(np.float32)


def kernel_acc(P, S, n_const, mv):
    """One support point's sum as score_core.cuh forms it: P, S (n, mv, 3) FP32."""
    npp = (mv + 5) // 14
    t = []
    for m in range(mv):
        d = [rn(P[:, m, r].astype(LD) - S[:, m, r].astype(LD)) for r in range(3)]
        t.append(fma(d[0], d[0], fma(d[1], d[1], fma(d[2], d[2], F32(1)))))
    acc = np.full(P.shape[0], F32(n_const), dtype=np.float32)
    for pp in range(npp):
        t1, t2 = t[2 * pp], t[2 * pp + 1]
        pr = rn(t1.astype(LD) * t2)
        num = fma(t1, t1, rn(t2.astype(LD) * t2))
        acc = fma(num, rcp_worst(rn(pr.astype(LD) * pr)), acc)
    for m in range(2 * npp, mv):
        rr = rcp_worst(t[m])
        acc = fma(rr, rr, acc)
    return acc


def exact_acc(P, S, n_const):
    d = P.astype(LD) - S.astype(LD)
    t = 1 + np.sum(d * d, axis=2)
    return n_const + np.sum(1 / (t * t), axis=1)


def derived(mv):
    npp = (mv + 5) // 14
    pair = 15 * U + RHO if npp > 0 else 0.0
    single = 10 * U + 2 * RHO if mv > 2 * npp else 0.0
    return max(pair, single) + (mv - npp) * U


@pytest.mark.parametrize("mv,scale", [(7, 16.0), (11, 16.0), (3, 6.0), (2, 16.0)])
def test_summand_error_within_derived_constant(mv, scale):
    rng = np.random.default_rng(mv * 101 + int(scale))
    n = 200_000
    P = (rng.uniform(-1, 1, size=(n, mv, 3)) * scale).astype(np.float32)
    # half the pairs far apart, half close (|d| around 1, where t^-2 is most sensitive)
    S = P + (rng.normal(size=(n, mv, 3)) * np.where(rng.uniform(size=(n, 1, 1)) < 0.5, scale, 0.6)).astype(np.float32)
    S = S.astype(np.float32)
    got = kernel_acc(P, S, 1, mv).astype(LD)
    want = exact_acc(P, S, 1)
    rel = np.abs(got - want) / want
    assert float(np.max(rel)) <= derived(mv), (float(np.max(rel)) / U, derived(mv) / U)
    # the emulation is not vacuous: the worst reciprocal shows up in the error
    assert float(np.max(rel)) > 0.5 * RHO


def test_rounded_coordinates_move_t_by_at_most_their_error():
    # premise (1): with d the exact difference and e the coordinates' error,
    # |t(d + e) / t(d) - 1| <= |e| + |e|^2 for t = 1 + |d|^2
    rng = np.random.default_rng(3)
    d = rng.normal(size=(100_000, 3)) * rng.uniform(0, 20, size=(100_000, 1))
    e = rng.normal(size=(100_000, 3)) * 1e-6
    t0 = 1 + np.sum(d * d, axis=1)
    t1 = 1 + np.sum((d + e) ** 2, axis=1)
    ne = np.linalg.norm(e, axis=1)
    assert np.all(np.abs(t1 / t0 - 1) <= (ne + ne * ne) * (1 + 1e-9))
