"""The non-paper Gaussian summand (FK_SUMMAND_GAUSS) on the GPU against the
FP64 oracle (oracle.SUMMANDS["gauss"]), through the C ABI.  Tolerances:

  kernel matrix (FP64)       |dK| <= 1e-14;  (FP32) |dK| <= 2e-6
  training (FP64 matrix)     pass sequence and support set identical, alpha within 1e-12
  score FP32 (MUFU ex2, and  |df| <= eps/2 * B(q), eps = 6e-6 the library's band,
  1 or 2 polynomial points)  B(q) = sum_s |alpha_s| K(S_s, q)
  score packed half          |df| <= eps16/2 * B(q), eps16 = 2e-3
  double-float tier          every query forced into the band: f = the FP64 value
                             rounded to FP32, 1 ulp at most on at most 1e-3 of them
  labels after re-score      identical to the oracle's
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu

EPS = 6e-6
EPS16 = 2e-3


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def _chain(fk, name):
    w = synth.workload(name)
    ch = fk.chain_from_arm(w.scene.arm)
    fk.fk_chain_set_summand(ch, fk.FK_SUMMAND_GAUSS)
    return w, ch


@pytest.fixture(scope="module")
def g3(fk):
    w, ch = _chain(fk, "arm3-n1000")
    yield w, ch
    fk.fk_chain_destroy(ch)


@pytest.fixture(scope="module")
def g7(fk):
    w, ch = _chain(fk, "arm7-n5000")
    yield w, ch
    fk.fk_chain_destroy(ch)


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_gauss_gram_matches_oracle(fk, g3, g7, dev, which):
    w, ch = g3 if which == "arm3" else g7
    arm = w.scene.arm
    Xa = w.train_configs()[:300].astype(np.float64)
    Xb = w.query_configs(77).astype(np.float64)
    cpa, cpb = O.fk_points(arm, Xa), O.fk_points(arm, Xb)
    for A, B, ta, tb in ((cpa, cpa, Xa, Xa), (cpa, cpb, Xa, Xb)):
        want = O.gram(A, B, w.gamma, "gauss")
        da = torch.from_numpy(ta).to(dev)
        db = da if tb is ta else torch.from_numpy(tb).to(dev)
        K = torch.empty((len(ta), len(tb)), dtype=torch.float64, device=dev)
        fk.fk_gram(ch, da, db, w.gamma, K)
        got = K.cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-14
        if tb is ta:
            assert np.array_equal(got, got.T) and np.all(np.diag(got) == 1.0)
        K32 = torch.empty((len(ta), len(tb)), dtype=torch.float32, device=dev)
        fk.fk_gram(ch, da.float(), da.float() if tb is ta else db.float(), w.gamma, K32)
        assert np.max(np.abs(K32.cpu().numpy() - want)) <= 2e-6
    # no double-float form of the Gaussian summand
    Kd = torch.empty((300, 300), dtype=torch.float64, device=dev)
    d = torch.from_numpy(Xa).to(dev)
    with pytest.raises(fk.FkError):
        fk.fk_gram(ch, d, d, w.gamma, Kd, double_float=True)


@pytest.mark.parametrize("which,n", [("arm3", 1000), ("arm7", 3000)])
def test_gauss_training_matches_oracle(fk, g3, g7, dev, which, n):
    w, ch = g3 if which == "arm3" else g7
    X = w.train_configs()[:n].astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max, trace=True,
                        summand="gauss")
    m = fk.fastron_model_create(ch)
    try:
        st = fk.fastron_train(m, torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), w.gamma, w.beta,
                              w.iter_max, w.s_max, trace=True)
        assert st["iterations"] == r.iters and st["n_support"] == r.n_support and st["converged"] == r.converged
        kind, idx, delta = fk.fastron_model_trace(m, r.iters + 1)
        assert np.array_equal(kind, r.trace[0]) and np.array_equal(idx, r.trace[1])
        np.testing.assert_allclose(delta, r.trace[2], rtol=1e-12, atol=1e-12)
        gidx, galpha = fk.fastron_model_get(m)
        assert np.array_equal(gidx, r.support)
        np.testing.assert_allclose(galpha, r.alpha[r.support], rtol=1e-12)
        with pytest.raises(fk.FkError):  # the Gaussian matrix is FP64 only
            fk.fastron_train(m, torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), w.gamma, w.beta,
                             w.iter_max, w.s_max, gram=fk.FK_DF64)
    finally:
        fk.fastron_model_destroy(m)


def _score(fk, w, ch, dev, S, alpha, Q, precision, poly=0):
    m = fk.fastron_model_create(ch)
    fk.fk_set_gauss_poly(poly)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        n = len(Q)
        tq = torch.from_numpy(Q).to(dev)
        f_raw = torch.empty(n, dtype=torch.float32, device=dev)
        lab_raw = torch.empty(n, dtype=torch.int8, device=dev)
        fk.fk_score(m, tq, lab_raw, f_raw, rescore=False, precision=precision)
        f = torch.empty(n, dtype=torch.float32, device=dev)
        lab = torch.empty(n, dtype=torch.int8, device=dev)
        nres = fk.fk_score(m, tq, lab, f, rescore=True, count=True, precision=precision)
        lab_na = torch.empty(n, dtype=torch.int8, device=dev)
        if precision == fk.FK_F32 and n <= 1 << 20:
            fk.fk_score_noalloc(m, tq, lab_na)
        torch.cuda.synchronize()
    finally:
        fk.fk_set_gauss_poly(0)
        fk.fastron_model_destroy(m)
    arm = w.scene.arm
    cps, cpq = O.fk_points(arm, S), O.fk_points(arm, Q.astype(np.float64))
    want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=8, summand="gauss")
    B = O.score_points(cps, np.abs(alpha), cpq, w.gamma, nthreads=8, summand="gauss")
    return (f_raw.cpu().numpy(), lab_raw.cpu().numpy(), f.cpu().numpy(), lab.cpu().numpy(), nres, want, B,
            lab_na.cpu().numpy())


def _trained(w, n=None):
    X = w.train_configs()[:n].astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max, summand="gauss")
    return X[r.support], r.alpha[r.support]


@pytest.mark.parametrize("which,poly", [("arm3", 0), ("arm7", 0), ("arm7", 1), ("arm7", 2)])
def test_gauss_score_fp32_matches_oracle(fk, g3, g7, dev, which, poly):
    w, ch = g3 if which == "arm3" else g7
    S, alpha = _trained(w, None if which == "arm3" else 3000)
    Q = w.query_configs(20000)
    f_raw, lab_raw, f, lab, nres, want, B, lab_na = _score(fk, w, ch, dev, S, alpha, Q, fk.FK_F32, poly)
    err = np.abs(f_raw.astype(np.float64) - want)
    assert np.all(err <= 0.5 * EPS * B + 1e-30), np.max(err / np.maximum(B, 1e-300))
    assert np.array_equal(lab_raw == 1, f_raw >= 0)
    assert np.array_equal(lab, O.labels_from_f(want))
    assert np.array_equal(lab_na, lab)
    assert nres >= np.sum(np.abs(f_raw.astype(np.float64)) < 0.99 * EPS * B)
    # re-scored queries carry the FP64 value rounded to FP32
    sel = np.abs(f_raw.astype(np.float64)) < 0.99 * EPS * B
    np.testing.assert_allclose(f[sel], want[sel].astype(np.float32), rtol=1e-6, atol=1e-30)


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_gauss_score_half_matches_oracle(fk, g3, g7, dev, which):
    w, ch = g3 if which == "arm3" else g7
    S, alpha = _trained(w, None if which == "arm3" else 3000)
    Q = w.query_configs(20000)
    f_raw, lab_raw, f, lab, nres, want, B, _ = _score(fk, w, ch, dev, S, alpha, Q, fk.FK_F16)
    err = np.abs(f_raw.astype(np.float64) - want)
    assert np.all(err <= 0.5 * EPS16 * B + 1e-30), np.max(err / np.maximum(B, 1e-300))
    assert np.array_equal(lab, O.labels_from_f(want))
    assert 0 < nres < len(Q)


def test_gauss_edge_sizes_and_self_score(fk, g7, dev):
    w, ch = g7
    S = w.train_configs()[:129].astype(np.float64)
    alpha = np.random.default_rng(5).normal(size=129) * 2
    for n in (1, 513, 1025):
        f_raw, lab_raw, f, lab, nres, want, B, _ = _score(fk, w, ch, dev, S, alpha, w.query_configs(n), fk.FK_F32)
        assert np.all(np.abs(f_raw - want) <= 0.5 * EPS * B + 1e-30)
        assert np.array_equal(lab, O.labels_from_f(want))
    # K(x, x) = 1: one support point scored at itself gives its weight
    f_raw, _, f, lab, _, want, _, _ = _score(fk, w, ch, dev, S[:1], np.array([-0.75]), S[:1].astype(np.float32),
                                              fk.FK_F32)
    assert abs(f_raw[0] + 0.75) <= 1e-6 and lab[0] == -1


def test_gauss_model_keeps_its_summand_and_batches_reject_it(fk, dev):
    w = synth.workload("arm7-n5000")
    ch = fk.chain_from_arm(w.scene.arm)
    try:
        S = w.train_configs()[:50].astype(np.float64)
        alpha = np.random.default_rng(6).normal(size=50)
        Q = w.query_configs(3000)
        m_rq = fk.fastron_model_create(ch)
        fk.fastron_model_set(m_rq, S, alpha, w.gamma)  # packed with the RQ summand
        fk.fk_chain_set_summand(ch, fk.FK_SUMMAND_GAUSS)
        m_g = fk.fastron_model_create(ch)
        fk.fastron_model_set(m_g, S, alpha, w.gamma)
        lab = torch.empty(3000, dtype=torch.int8, device=dev)
        fk.fk_score(m_rq, torch.from_numpy(Q).to(dev), lab)
        cps, cpq = O.fk_points(w.scene.arm, S), O.fk_points(w.scene.arm, Q.astype(np.float64))
        assert np.array_equal(lab.cpu().numpy(), O.labels_from_f(O.score_points(cps, alpha, cpq, w.gamma)))
        with pytest.raises(fk.FkError):
            fk.fk_batch_create([m_g])
        with pytest.raises(fk.FkError):
            fk.fk_chain_set_summand(ch, 7)
        with pytest.raises(fk.FkError):
            fk.fk_set_gauss_poly(3)
        fk.fastron_model_destroy(m_rq)
        fk.fastron_model_destroy(m_g)
    finally:
        fk.fk_chain_destroy(ch)


def _ulps32(a, b):
    ia = np.asarray(a, dtype=np.float32).view(np.int32).astype(np.int64)
    ib = np.asarray(b, dtype=np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_gauss_double_float_tier_on_every_query(fk, g3, g7, dev, which):
    # a band of eps = 1 holds every query, so the double-float tier (the pair
    # arithmetic 2^(-t)) evaluates all of them: rounded to FP32 its f is the
    # FP64 value rounded to FP32 (1 ulp where that value sits on a rounding
    # boundary within the pair error)
    w, ch = g3 if which == "arm3" else g7
    S, alpha = _trained(w, None if which == "arm3" else 1500)
    Q = w.query_configs(6000)
    cps, cpq = O.fk_points(w.scene.arm, S), O.fk_points(w.scene.arm, Q.astype(np.float64))
    want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=8, summand="gauss")
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        tq = torch.from_numpy(Q).to(dev)
        f = torch.empty(len(Q), dtype=torch.float32, device=dev)
        lab = torch.empty(len(Q), dtype=torch.int8, device=dev)
        nres = fk.fk_score(m, tq, lab, f, rescore=True, eps=1.0, count=True)
        torch.cuda.synchronize()
    finally:
        fk.fastron_model_destroy(m)
    assert nres == len(Q)
    u = _ulps32(f.cpu().numpy(), want.astype(np.float32))
    assert u.max() <= 1 and np.mean(u > 0) <= 1e-3, (u.max(), np.mean(u > 0))
    assert np.array_equal(lab.cpu().numpy(), O.labels_from_f(want))
