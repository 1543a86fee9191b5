"""Parity at the full sizes the benchmark runs, in its launch configuration.

The label of a query is the sign of the model value f (Sec. III-B); the FP32
kernel decides it alone only where |f32| > eps(q) B(q), the derived bound of
its whole error (tests/_band.py), and re-scores the rest.  These tests hold
that to the FP64 oracle at full size:

  7-DOF workload (N = 5000, 4,194,304 queries): labels of the training set
  equal the checker's; the training trace equals the oracle's; EVERY query
  label equals the sign of the oracle's FP64 f, and EVERY query's FP32 value
  lies within eps(q) B(q) of it.
  12-point arm (N = 65,536, 16,777,216 queries): the oracle trains its own
  model (Algorithm 1, threaded kernel-matrix columns); the GPU scores all
  queries with that support set and those weights; every query of the GPU's
  band (a superset recomputed from the FP32 values) and every query of a
  1,048,576-query sample get the oracle's label, and on the sample's queries
  with |f| < 10 eps(q) B(q) and on the band the FP32 value lies within
  eps(q) B(q) of the oracle's.
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth
from tests import _band

pytestmark = pytest.mark.gpu
NT = max(1, min(64, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def _raw_and_labels(fk, m, tq, n, dev):
    """Labels with the re-score, the FP32 values without it, and the band size."""
    lab = torch.empty(n, dtype=torch.int8, device=dev)
    nres = fk.fk_score(m, tq, lab, rescore=True, count=True)
    f_raw = torch.empty(n, dtype=torch.float32, device=dev)
    lab_raw = torch.empty(n, dtype=torch.int8, device=dev)
    fk.fk_score(m, tq, lab_raw, f_raw, rescore=False)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), f_raw.cpu().numpy().astype(np.float64), nres


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
        lab, f_raw, nres = _raw_and_labels(fk, m, torch.from_numpy(Q).to(dev), nq, dev)
        eps0, eps1 = fk.fk_score_band(m)
        assert (eps0, eps1) == _band.constants(arm, w.gamma, r.n_support)
        cnorm = fk.fk_score_circle(m)
        assert cnorm == pytest.approx(_band.circle_norm(arm, w.gamma, r.n_support), rel=1e-6, abs=0.0)
        assert 0 < nres < nq // 100
        # the oracle's own model on every query
        S, alpha = Xd[r.support], r.alpha[r.support]
        cps, cpq = O.fk_points(arm, S), O.fk_points(arm, Q.astype(np.float64))
        want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=NT)
        B = O.score_points(cps, np.abs(alpha), cpq, w.gamma, nthreads=NT)
        eps = _band.per_query(arm, w.gamma, eps0, eps1, cps, cpq, cnorm)
        assert np.array_equal(lab, O.labels_from_f(want))
        err = np.abs(f_raw - want)
        assert np.all(err <= eps * B), np.max(err / (eps * B))
        # the band holds every query the bound leaves open
        assert nres >= np.sum(np.abs(f_raw) < 0.999 * eps * B)
        # exact-sign ties (|f| at FP64 rounding level) would be reported, not compared: there are none
        assert np.sum(np.abs(want) < 1e-12 * B) == 0
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


def test_twelve_point_scoring_at_full_size(fk, dev):
    w = synth.workload("arm7m12-n65536")
    arm = w.scene.arm
    X = w.train_configs().astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max, nthreads=NT)
    assert r.converged and r.n_support > 5000
    S, alpha = X[r.support], r.alpha[r.support]
    ch = fk.chain_from_arm(arm)
    m = fk.fastron_model_create(ch)
    mb = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        fk.fastron_model_set(mb, S, np.abs(alpha), w.gamma)
        nq = 1 << 24
        Q = w.query_configs(nq)
        tq = torch.from_numpy(Q).to(dev)
        lab, f_raw, nres = _raw_and_labels(fk, m, tq, nq, dev)
        # B(q) in FP32 from the model with weights |alpha| (all terms in one sum)
        _, b_raw, _ = _raw_and_labels(fk, mb, tq, nq, dev)
        eps0, eps1 = fk.fk_score_band(m)
        assert (eps0, eps1) == _band.constants(arm, w.gamma, len(S))
        cnorm = fk.fk_score_circle(m)
        assert cnorm == pytest.approx(_band.circle_norm(arm, w.gamma, len(S)), rel=1e-6, abs=0.0)
    finally:
        fk.fastron_model_destroy(m)
        fk.fastron_model_destroy(mb)
        fk.fk_chain_destroy(ch)
    cps = O.fk_points(arm, S)
    g = np.sqrt(0.5 * w.gamma)
    smax = g * np.max(np.linalg.norm(_band.dependent(arm, cps), axis=2))
    # eps(q) upper bound for every query without the oracle: |p(q)| <= reach
    eps_hi = eps0 + eps1 * max(g * _band.reach(arm) + smax, cnorm)
    band = np.flatnonzero(np.abs(f_raw) <= 1.01 * eps_hi * b_raw)
    assert nres <= len(band)
    rng = np.random.default_rng(12)
    sample = np.sort(rng.choice(nq, 1 << 20, replace=False))
    pick = np.union1d(band, sample)
    cpq = O.fk_points(arm, Q[pick].astype(np.float64))
    want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=NT)
    assert np.array_equal(lab[pick], O.labels_from_f(want))
    # the bound, where it decides: the band and the sample's near-zero queries
    eps = _band.per_query(arm, w.gamma, eps0, eps1, cps, cpq, cnorm)
    near = np.isin(pick, band) | (np.abs(want) < 10.0 * eps * b_raw[pick] * 1.01)
    Bn = O.score_points(cps, np.abs(alpha), cpq[near], w.gamma, nthreads=NT)
    err = np.abs(f_raw[pick][near] - want[near])
    assert np.all(err <= eps[near] * Bn), np.max(err / (eps[near] * Bn))
    assert np.sum(np.abs(want[near]) < 1e-12 * Bn) == 0
