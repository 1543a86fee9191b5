"""The premises of the score kernel's error bound, checked on the GPU.

The band of fk_score (tests/_band.py) rests on three facts about the
kernel's arithmetic:

  1. the MUFU reciprocal rcp.approx.ftz.f32 has |rcp(x) x - 1| <= 2^-23,
     checked on every FP32 mantissa of the binades the kernel reaches
     (t >= 1 up to (t1 t2)^2 for the largest scaled reach);
  2. the pair-arithmetic sine and cosine are within 2^-40 of FP64, on every
     FP32 angle of [-8, 8] and with a pair-valued joint offset;
  3. the kinematics of the score kernel give every configuration-dependent
     control point within u |p| + 2^-32 (1 + g reach) of the FP64 oracle's
     (Eqs. 1-2), scaled by g = sqrt(gamma/2) and rounded once to FP32.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth
from tests import _band

pytestmark = pytest.mark.gpu


def test_mufu_reciprocal_within_one_ulp(fk):
    # every mantissa of [2^-4, 2^64): the kernel's t lies in [1, 1 + 4 (g reach)^2]
    # and its shared reciprocal takes (t1 t2)^2 <= 2^48 on every workload here
    worst = fk.fk_check_rcp(-4, 63)
    assert 0.0 < worst <= 2.0 ** -23, worst


def test_pair_sincos_exhaustive(fk):
    assert fk.fk_check_sincos(8.0, 0.0) <= 2.0 ** -40
    # a joint offset with a non-zero low word
    assert fk.fk_check_sincos(4.0, 0.3183098861837907) <= 2.0 ** -40
    assert fk.fk_check_sincos(1.0, -2.5) <= 2.0 ** -40


@pytest.mark.parametrize("name", ["arm3-n1000", "arm7-n5000", "arm7m12-n65536"])
def test_pair_kinematics_rounded_once(fk, name):
    dev = torch.device("cuda:0")
    w = synth.workload(name)
    arm = w.scene.arm
    n = 200_000
    Q = w.query_configs(n)
    # joint limits and zero: the configurations at the corners of the range
    Q[:3] = np.float32([w.scene.arm.qlim, -w.scene.arm.qlim, 0.0])[:, None]
    ch = fk.chain_from_arm(arm)
    try:
        mv = int(np.sum(arm.cp_joint != 0))
        cp = torch.empty((mv, 3, n), dtype=torch.float32, device=dev)
        g = np.sqrt(0.5 * w.gamma)
        fk.fk_forward_dd(ch, torch.from_numpy(Q).to(dev), g, cp)
        torch.cuda.synchronize()
    finally:
        fk.fk_chain_destroy(ch)
    got = cp.permute(2, 0, 1).cpu().numpy().astype(np.float64)  # (n, mv, 3)
    exact = g * _band.dependent(arm, O.fk_points(arm, Q.astype(np.float64)))
    efk = 2.0 ** -32 * (1.0 + g * _band.reach(arm))
    err = np.abs(got - exact)
    assert np.all(err <= _band.U * np.abs(exact) * (1 + 1e-9) + efk)
    # rounded once: equal to the FP64 value rounded to FP32 except where that
    # value lies within the pair error of a rounding boundary
    same = got == exact.astype(np.float32).astype(np.float64)
    assert np.mean(same) >= 0.9999, np.mean(same)


def test_band_constants_match_the_derivation(fk):
    # every workload's model: the library's (eps0, eps1) are the derivation's
    for name in ("arm3-n1000", "arm7-n5000", "arm7m12-n65536"):
        w = synth.workload(name)
        ch = fk.chain_from_arm(w.scene.arm)
        m = fk.fastron_model_create(ch)
        try:
            for ns in (1, 800, 11677):
                S = w.train_configs()[:ns].astype(np.float64)
                ns = len(S)
                fk.fastron_model_set(m, S, np.ones(ns), w.gamma)
                assert fk.fk_score_band(m) == _band.constants(w.scene.arm, w.gamma, ns)
                assert fk.fk_score_band(m, fk.FK_F16) == _band.constants(w.scene.arm, w.gamma, ns, half=True)
                cn = _band.circle_norm(w.scene.arm, w.gamma, ns)
                assert (cn > 0) == (ns >= 128) and fk.fk_score_circle(m) == pytest.approx(cn, rel=1e-6, abs=0.0)
        finally:
            fk.fastron_model_destroy(m)
            fk.fk_chain_destroy(ch)
