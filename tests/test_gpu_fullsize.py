"""Parity at the full sizes the benchmark runs, in its launch configuration,
on sampled outputs the oracle computes one by one.

  7-DOF workload: labels of all 5000 training configurations equal the
  checker's; the training trace equals the oracle's; 4,194,304 queries are
  scored with the band re-score and every label in a 20,000-query sample
  equals the sign of the oracle's FP64 score.
  12-point arm: a model trained on all 65,536 configurations scores
  16,777,216 queries; a 4000-query sample of its labels equals the sign of the
  oracle's FP64 score of the same support set and weights, and the FP32
  values of the sample lie within eps/2 B(q) of it.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu
EPS_BAND = 6e-6


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def test_seven_dof_step_at_full_size(fk, dev):
    w = synth.workload("arm7-n5000")
    arm = w.scene.arm
    ch = fk.chain_from_arm(arm)
    m = fk.fastron_model_create(ch)
    try:
        X = w.train_configs()
        Xd = X.astype(np.float64)
        y = torch.empty(len(X), dtype=torch.int8, device=dev)
        fk.fk_label(ch, w.scene.boxes, w.scene.radius, torch.from_numpy(X).to(dev), y)
        want_y = O.check(w.scene, Xd)
        assert np.array_equal(y.cpu().numpy(), want_y)
        st = fk.fastron_train(m, torch.from_numpy(Xd).to(dev), y, w.gamma, w.beta, w.iter_max, w.s_max, trace=True)
        r = O.fastron_train(O.fk_points(arm, Xd), want_y, w.gamma, w.beta, w.iter_max, w.s_max, trace=True)
        kind, idx, _ = fk.fastron_model_trace(m, r.iters + 1)
        assert st["iterations"] == r.iters and np.array_equal(kind, r.trace[0]) and np.array_equal(idx, r.trace[1])
        nq = 1 << 22
        Q = w.query_configs(nq)
        tq = torch.from_numpy(Q).to(dev)
        lab = torch.empty(nq, dtype=torch.int8, device=dev)
        nres = fk.fk_score(m, tq, lab, rescore=True, count=True)
        assert 0 < nres < nq // 100
        rng = np.random.default_rng(11)
        sample = rng.choice(nq, 20000, replace=False)
        sup, alpha = fk.fastron_model_get(m)
        want = O.score(arm, Xd[sup], alpha, Q[sample].astype(np.float64), w.gamma, nthreads=16)
        assert np.array_equal(lab.cpu().numpy()[sample], O.labels_from_f(want))
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


def test_twelve_point_scoring_at_full_size(fk, dev):
    w = synth.workload("arm7m12-n65536")
    arm = w.scene.arm
    ch = fk.chain_from_arm(arm)
    m = fk.fastron_model_create(ch)
    try:
        X = w.train_configs()
        Xd = torch.from_numpy(X.astype(np.float64)).to(dev)
        y = torch.empty(len(X), dtype=torch.int8, device=dev)
        fk.fk_label(ch, w.scene.boxes, w.scene.radius, torch.from_numpy(X).to(dev), y)
        st = fk.fastron_train(m, Xd, y, w.gamma, w.beta, w.iter_max, w.s_max, gram=fk.FK_DF32)
        assert st["converged"] and st["n_support"] > 5000
        nq = 1 << 24
        Q = w.query_configs(nq)
        tq = torch.from_numpy(Q).to(dev)
        lab = torch.empty(nq, dtype=torch.int8, device=dev)
        f_raw = torch.empty(nq, dtype=torch.float32, device=dev)
        fk.fk_score(m, tq, lab, rescore=True)
        lab_raw = torch.empty(nq, dtype=torch.int8, device=dev)
        fk.fk_score(m, tq, lab_raw, f_raw, rescore=False)
        torch.cuda.synchronize()
        rng = np.random.default_rng(12)
        sample = rng.choice(nq, 4000, replace=False)
        sup, alpha = fk.fastron_model_get(m)
        S = X[sup].astype(np.float64)
        cps, cpq = O.fk_points(arm, S), O.fk_points(arm, Q[sample].astype(np.float64))
        want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=16)
        B = O.score_points(cps, np.abs(alpha), cpq, w.gamma, nthreads=16)
        assert np.array_equal(lab.cpu().numpy()[sample], O.labels_from_f(want))
        err = np.abs(f_raw.cpu().numpy()[sample].astype(np.float64) - want)
        assert np.all(err <= 0.5 * EPS_BAND * B)
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)
