"""The circle form of the first control point in the FP32 score, on the CPU.

When the first configuration-dependent control point sits on frame 1 of a
revolute joint 1, Eq. 1 for link 1 and Eq. 2 put it at p0 + R0 Rz(theta) u
with a constant u, so it moves on a circle of radius rho = |(u_x, u_y)| about
the joint's axis and |p - s| = 2 rho |sin((theta - theta_s) / 2)| for two
configurations (theta = theta0 + q_1).  The FP32 kernel computes that point's
t = 1 + g^2 |p - s|^2 from sin and cos of theta / 2 and the support's
2 rho g (cos, sin)(theta_s / 2).  Pinned here:

  * the geometry, against the oracle's FP64 kinematics (tests/_band.py's
    rho, arms with offsets, twists and base transforms);
  * the summand's error bound 12 u (1 + u) rho g + 6u + 2 rho_rcp (+ u for
    its accumulation), by emulating the kernel's FP32 roundings with a
    worst-case reciprocal, at the worst place (two nearly equal angles);
  * which chains qualify.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_06451_gb300 import synth
from tests import _band

U = 2.0 ** -24
RHO = 2.0 ** -23
F32 = np.float32
LD = np.longdouble


def rn(x):
    return np.asarray(x, dtype=LD).astype(np.float32)


def fma(a, b, c):
    return rn(np.asarray(a, dtype=LD) * np.asarray(b, dtype=LD) + np.asarray(c, dtype=LD))


def rcp_worst(x):
    exact = LD(1) / np.asarray(x, dtype=LD)
    r = rn(exact)
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(0))
    return np.where(np.abs(up.astype(LD) - exact) > np.abs(dn.astype(LD) - exact), up, dn).astype(np.float32)


def _rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def _offset_arm(seed):
    """A revolute arm with a random base transform, random twists and a
    control point off the frame-1 origin."""
    rng = np.random.default_rng(seed)
    arm = synth.arm_7dof(seed)
    dh = arm.dh.copy()
    dh[:, 1] = rng.uniform(-math.pi, math.pi, size=len(dh))
    dh[:, 3] = rng.uniform(-1, 1, size=len(dh))
    base = np.eye(4)
    base[:3, :3] = _rot(rng)
    base[:3, 3] = rng.uniform(-0.5, 0.5, size=3)
    off = arm.cp_off.copy()
    off[1] = rng.uniform(-0.3, 0.3, size=3)
    return synth.Arm(dh=dh, base=base, cp_joint=arm.cp_joint, cp_off=off, qlim=arm.qlim)


@pytest.mark.parametrize("which", ["arm3", "arm7", "arm7m12", "offset1", "offset2"])
def test_circle_geometry_matches_oracle_kinematics(which):
    arm = {"arm3": lambda: synth.arm_3dof(11), "arm7": lambda: synth.arm_7dof(7),
           "arm7m12": lambda: synth.arm_7dof_m12(7), "offset1": lambda: _offset_arm(1),
           "offset2": lambda: _offset_arm(2)}[which]()
    rho = _band.circle_radius(arm)
    assert rho is not None and rho > 0
    rng = np.random.default_rng(5)
    n = 2000
    qa = rng.uniform(-arm.qlim, arm.qlim, size=(n, arm.D))
    qb = rng.uniform(-arm.qlim, arm.qlim, size=(n, arm.D))
    qb[: n // 4, 0] = qa[: n // 4, 0] + rng.normal(size=n // 4) * 1e-4  # nearly equal joint-1 angles
    v0 = int(np.flatnonzero(np.asarray(arm.cp_joint) != 0)[0])
    pa, pb = O.fk_points(arm, qa)[:, v0, :], O.fk_points(arm, qb)[:, v0, :]
    got = np.linalg.norm(pa - pb, axis=1)
    th0 = arm.dh[0, 3]
    want = 2.0 * rho * np.abs(np.sin(0.5 * ((th0 + qa[:, 0]) - (th0 + qb[:, 0]))))
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-13)
    # the radius is the distance from joint 1's axis: |u| with its axial
    # component (a plausible mistake) fails wherever that component is not zero
    a, al, d = arm.dh[0, 0], arm.dh[0, 1], arm.dh[0, 2]
    t = np.asarray(arm.cp_off, dtype=np.float64)[v0]
    u = np.array([a + t[0], math.cos(al) * t[1] - math.sin(al) * t[2], d + math.sin(al) * t[1] + math.cos(al) * t[2]])
    if abs(np.linalg.norm(u) - rho) > 1e-6:
        wrong = 2.0 * np.linalg.norm(u) * np.abs(np.sin(0.5 * (qa[:, 0] - qb[:, 0])))
        assert not np.allclose(got, wrong, rtol=1e-9, atol=1e-13)


def test_circle_summand_within_bound():
    rng = np.random.default_rng(9)
    n = 400_000
    th = rng.uniform(-2 * math.pi, 2 * math.pi, size=n)
    far = rng.uniform(-2 * math.pi, 2 * math.pi, size=n)
    near = th + rng.normal(size=n) * 10.0 ** rng.uniform(-7, -1, size=n)
    ths = np.where(rng.uniform(size=n) < 0.5, far, near)
    rg = 10.0 ** rng.uniform(-1.5, math.log10(4.0), size=n)
    thl, thsl = th.astype(LD), ths.astype(LD)
    # query: sin and cos of theta / 2 from pair arithmetic (error below 2^-44), rounded once
    e_sc = 2.0 ** -44
    sg = rn(np.sin(thl / 2) + LD(e_sc) * rng.uniform(-1, 1, size=n))
    cg = rn(np.cos(thl / 2) + LD(e_sc) * rng.uniform(-1, 1, size=n))
    C = rn(2 * rg.astype(LD) * np.cos(thsl / 2))
    S = rn(2 * rg.astype(LD) * np.sin(thsl / 2))
    a = rn(-(cg.astype(LD) * S.astype(LD)))  # fl(-cg S): the kernel's product
    D = fma(sg, C, a)
    t = fma(D, D, F32(1))
    r = rcp_worst(t)
    k = rn(r.astype(LD) * r)  # one more rounding: the accumulating FMA
    d_exact = 2 * rg.astype(LD) * np.sin((thl - thsl) / 2)
    k_exact = 1 / (1 + d_exact * d_exact) ** 2
    rel = np.abs(k.astype(LD) - k_exact) / k_exact
    bound = 12 * U * (1 + U) * rg + 6 * U + 2 * RHO + U
    assert np.all(rel <= bound * (1 + 2.0 ** -10)), float(np.max(rel / bound))
    # not vacuous: close to the bound where the angles nearly agree and rho g is large
    assert float(np.max(rel / bound)) > 0.3
    # and within the band's share for it: eps1 cnorm + 10u + 2 rho_rcp + u
    eps1 = 2 * U * (1 + U)
    assert np.all(rel <= eps1 * 6 * rg + 10 * U + 2 * RHO + U)


def test_circle_form_qualifying_chains():
    arm = synth.arm_7dof(7)
    assert _band.circle_radius(arm) == pytest.approx(abs(arm.dh[0, 0]), rel=1e-15)
    # prismatic joint 1: no circle
    dh = arm.dh.copy()
    dh[0, 4] = 1
    assert _band.circle_radius(synth.Arm(dh=dh, base=arm.base, cp_joint=arm.cp_joint, cp_off=arm.cp_off,
                                         qlim=arm.qlim)) is None
    # first configuration-dependent point on frame 2: no circle
    cj = np.array(arm.cp_joint)
    cj[1] = 2
    assert _band.circle_radius(synth.Arm(dh=arm.dh, base=arm.base, cp_joint=cj, cp_off=arm.cp_off,
                                         qlim=arm.qlim)) is None
    # rho g above 4: direct form
    rho = _band.circle_radius(arm)
    assert _band.circle_norm(arm, 2.0 * (4.0 / rho) ** 2 * 1.01, 800) == 0.0
    assert _band.circle_norm(arm, 40.0, 800) > 6.0 * rho * math.sqrt(20.0)
    assert _band.circle_norm(arm, 40.0, 800, on=False) == 0.0
    # small support sets: the per-query sine and cosine would cost more than the form saves
    assert _band.circle_norm(arm, 40.0, 127) == 0.0 and _band.circle_norm(arm, 40.0, 128) > 0.0
