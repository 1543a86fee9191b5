"""The changing-environment workload through the C ABI: the 7-DOF arm with 12
control points, a kernel matrix stored in FP32 (FK_DF32), training sets up to
65,536 points, warm-started Algorithm 1 on a fixed training set relabelled as
the boxes move (reuse_gram), the paper's two-stage active learning with
carried-over weights (fk_active_samples, warm_start = 2), and scoring with 11
configuration-dependent control points.  Tolerances:

  FP32-stored kernel matrix   each entry the FP32 rounding of the FP64 entry;
                              1 ulp where the FP64 value lies within the
                              double-float error (~1e-13) of a rounding
                              boundary (at most 1e-4 of the entries)
  training                    pass sequence identical to the oracle's with
                              FP32-rounded columns; deltas and alpha within
                              1e-6 (FP32 storage: an entry one FP32 ulp off
                              moves later deltas by ~|delta| 6e-8) or 1e-9
                              (FP64 storage)
  active-learning samples     bit-identical to the oracle's (same SplitMix64
                              draws, same FP64 operations, one FP32 rounding)
  large N                     the first 40 passes identical; converged margins
                              positive and no removal applicable, on sampled
                              points recomputed by the oracle
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def arm12(fk):
    w = synth.workload("arm7m12-n65536")
    ch = fk.chain_from_arm(w.scene.arm)
    yield w, ch
    fk.fk_chain_destroy(ch)


def _ulps32(a, b):
    ia = np.asarray(a, dtype=np.float32).view(np.int32).astype(np.int64)
    ib = np.asarray(b, dtype=np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def test_gram_fp32_storage_rounds_the_fp64_entries(fk, arm12, dev):
    w, ch = arm12
    X = w.train_configs()[:700].astype(np.float64)
    cp = O.fk_points(w.scene.arm, X)
    want = O.gram(cp, cp, w.gamma).astype(np.float32)
    tX = torch.from_numpy(X).to(dev)
    K = torch.empty((700, 700), dtype=torch.float32, device=dev)
    fk.fk_gram(ch, tX, tX, w.gamma, K, double_float=True)
    got = K.cpu().numpy()
    u = _ulps32(got, want)
    assert u.max() <= 1 and np.mean(u > 0) <= 1e-4
    assert np.array_equal(got, got.T) and np.all(np.diag(got) == 1.0)
    Xb = w.query_configs(333).astype(np.float64)
    Kb = torch.empty((700, 333), dtype=torch.float32, device=dev)
    fk.fk_gram(ch, tX, torch.from_numpy(Xb).to(dev), w.gamma, Kb, double_float=True)
    u = _ulps32(Kb.cpu().numpy(), O.gram(cp, O.fk_points(w.scene.arm, Xb), w.gamma).astype(np.float32))
    assert u.max() <= 1 and np.mean(u > 0) <= 1e-4


def _labels(fk, ch, boxes, X, dev):
    y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
    fk.fk_label(ch, boxes, 0.03, torch.from_numpy(X.astype(np.float32)).to(dev), y)
    return y


def _compare_trace(fk, m, r, store32):
    # FP32 storage: an entry one FP32 ulp (6e-8) from the oracle's rounding
    # moves later deltas by about |delta| 6e-8, hence 1e-6; FP64 storage 1e-9
    tol = 1e-6 if store32 else 1e-9
    kind, idx, delta = fk.fastron_model_trace(m, r.iters + 1)
    assert len(kind) == r.iters
    assert np.array_equal(kind, r.trace[0]) and np.array_equal(idx, r.trace[1])
    np.testing.assert_allclose(delta, r.trace[2], rtol=tol, atol=tol)
    gidx, galpha = fk.fastron_model_get(m)
    assert np.array_equal(gidx, r.support)
    np.testing.assert_allclose(galpha, r.alpha[r.support], rtol=tol, atol=tol)


@pytest.mark.parametrize("gram", ["df32", "df64"])
def test_changing_environment_frames_match_oracle(fk, arm12, dev, gram):
    # a fixed training set relabelled as the boxes move: frame 0 cold, later
    # frames warm-started from the previous alpha and F (loadPreviousModel)
    # with the stored kernel matrix reused
    w, ch = arm12
    n, frames = 2500, 4
    X = w.train_configs()[:n].astype(np.float64)
    cp = O.fk_points(w.scene.arm, X)
    path = synth.moving_boxes(w.seed, w.scene.boxes, frames)
    store32 = gram == "df32"
    code = fk.FK_DF32 if store32 else fk.FK_DF64
    tX = torch.from_numpy(X).to(dev)
    m = fk.fastron_model_create(ch)
    alpha = F = None
    try:
        for k in range(frames):
            sc = synth.Scene(w.scene.arm, path[k], 0.03)
            y = O.check(sc, X)
            ty = _labels(fk, ch, path[k], X, dev)
            assert np.array_equal(ty.cpu().numpy(), y)
            r = O.fastron_train(cp, y, w.gamma, w.beta, 20000, w.s_max, alpha0=alpha, F0=F, trace=True,
                                store32=store32)
            alpha, F = r.alpha, r.F
            st = fk.fastron_train(m, tX, ty, w.gamma, w.beta, 20000, w.s_max, warm_start=k > 0, trace=True,
                                  gram=code, reuse_gram=k > 0)
            assert (st["iterations"], st["adds"], st["removes"], st["converged"], st["n_support"]) == \
                (r.iters, r.adds, r.removes, r.converged, r.n_support)
            _compare_trace(fk, m, r, store32)
            if k > 0:
                assert 0 < r.iters
    finally:
        fk.fastron_model_destroy(m)


def test_reuse_gram_needs_a_matching_previous_call(fk, arm12, dev):
    w, ch = arm12
    X = torch.from_numpy(w.train_configs()[:300].astype(np.float64)).to(dev)
    y = _labels(fk, ch, w.scene.boxes, X.cpu().numpy(), dev)
    m = fk.fastron_model_create(ch)
    try:
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, X, y, w.gamma, reuse_gram=True)
        fk.fastron_train(m, X, y, w.gamma, gram=fk.FK_DF32)
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, X, y, w.gamma, gram=fk.FK_DF64, reuse_gram=True)
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, X[:200], y[:200], w.gamma, gram=fk.FK_DF32, reuse_gram=True)
        with pytest.raises(fk.FkError) as e:  # same size, another buffer: the matrix is not X2's
            fk.fastron_train(m, X.clone(), y, w.gamma, gram=fk.FK_DF32, reuse_gram=True)
        assert e.value.code == fk.FK_ERR_STATE
        st = fk.fastron_train(m, X, y, w.gamma, gram=fk.FK_DF32, reuse_gram=True)
        assert st["converged"]
    finally:
        fk.fastron_model_destroy(m)


def test_large_training_set_sixteen_points_per_thread(fk, arm12, dev):
    # N = 40,000 needs the 16-CTA cluster with 10 points per thread (the
    # 16-point variant); the oracle gives the first passes, the oracle's
    # margins of sampled points check the converged model
    w, ch = arm12
    n, prefix = 40_000, 40
    X = w.train_configs()[:n].astype(np.float64)
    y = O.check(w.scene, X)
    cp = O.fk_points(w.scene.arm, X)
    tX, ty = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
    m = fk.fastron_model_create(ch)
    try:
        st = fk.fastron_train(m, tX, ty, w.gamma, w.beta, w.iter_max, w.s_max, trace=True, gram=fk.FK_DF32)
        kind, idx, delta = fk.fastron_model_trace(m, prefix)
        r = O.fastron_train(cp, y, w.gamma, w.beta, prefix, w.s_max, trace=True, store32=True)
        assert np.array_equal(kind, r.trace[0]) and np.array_equal(idx, r.trace[1])
        np.testing.assert_allclose(delta, r.trace[2], rtol=1e-6, atol=1e-6)
        assert st["converged"] and 0 < st["n_support"] <= w.s_max
        sup, alpha = fk.fastron_model_get(m)
        assert np.all(np.diff(sup) > 0) and np.all(alpha != 0)
        rng = np.random.default_rng(5)
        js = np.unique(np.concatenate([rng.choice(n, 200, replace=False), sup[rng.choice(len(sup), 100)]]))
        K = O.gram(cp[sup], cp[js], w.gamma).astype(np.float32).astype(np.float64)
        Fj = alpha @ K
        assert np.all(y[js] * Fj > 0)  # every sampled margin positive
        pos = {s: i for i, s in enumerate(sup)}
        for t, j in enumerate(js):
            if j in pos:  # no removal applies: y_j (F_j - alpha_j) <= 0
                assert y[j] * (Fj[t] - alpha[pos[j]]) <= 1e-9
    finally:
        fk.fastron_model_destroy(m)


def test_score_twelve_control_points(fk, arm12, dev):
    w, ch = arm12
    X = w.train_configs()[:3000].astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, 20000, w.s_max)
    S, alpha = X[r.support], r.alpha[r.support]
    Q = w.query_configs(20000)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        tq = torch.from_numpy(Q).to(dev)
        f_raw = torch.empty(len(Q), dtype=torch.float32, device=dev)
        lab_raw = torch.empty(len(Q), dtype=torch.int8, device=dev)
        fk.fk_score(m, tq, lab_raw, f_raw, rescore=False)
        lab = torch.empty(len(Q), dtype=torch.int8, device=dev)
        fk.fk_score(m, tq, lab, rescore=True)
        torch.cuda.synchronize()
    finally:
        fk.fastron_model_destroy(m)
    cps, cpq = O.fk_points(w.scene.arm, S), O.fk_points(w.scene.arm, Q.astype(np.float64))
    want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=8)
    B = O.score_points(cps, np.abs(alpha), cpq, w.gamma, nthreads=8)
    err = np.abs(f_raw.cpu().numpy().astype(np.float64) - want)
    assert np.all(err <= 3e-6 * B + 1e-30)
    assert np.array_equal(lab.cpu().numpy(), O.labels_from_f(want))


def test_active_samples_match_oracle(fk, arm12, dev):
    w, ch = arm12
    X = w.train_configs()[:1500].astype(np.float64)
    y = O.check(w.scene, X)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_train(m, torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), w.gamma, w.beta, 20000,
                         w.s_max)
        sup, _ = fk.fastron_model_get(m)
        ns = len(sup)
        rows = ns * 3 + 700
        Xd = torch.empty((rows + 5, 7), dtype=torch.float64, device=dev)
        X32 = torch.empty((rows + 5, 7), dtype=torch.float32, device=dev)
        n = fk.fk_active_samples(m, 2, 0.1, 700, w.scene.arm.qlim, 0xC0FFEE, Xd, X32)
        assert n == rows
        want = O.active_samples(X[sup], 2, 0.1, 700, w.scene.arm.qlim, 0xC0FFEE)
        got = Xd[:rows].cpu().numpy()
        assert np.array_equal(got, want)
        assert np.array_equal(X32[:rows].cpu().numpy().astype(np.float64), want)
        small = torch.empty((rows - 1, 7), dtype=torch.float64, device=dev)
        with pytest.raises(fk.FkError):
            fk.fk_active_samples(m, 2, 0.1, 700, w.scene.arm.qlim, 1, small)
    finally:
        fk.fastron_model_destroy(m)


@pytest.mark.parametrize("gram", ["df32", "df64"])
def test_active_learning_frames_match_oracle(fk, arm12, dev, gram):
    # the paper's update loop: the next training set is the support set, one
    # perturbed copy of it and uniform samples up to n_max; labels from the
    # moved boxes; Algorithm 1 from the carried weights (F = K alpha)
    w, ch = arm12
    n_max, frames, sigma = 3000, 3, 0.1
    qlim = w.scene.arm.qlim
    store32 = gram == "df32"
    code = fk.FK_DF32 if store32 else fk.FK_DF64
    path = synth.moving_boxes(w.seed, w.scene.boxes, frames)
    X = w.train_configs()[:2000].astype(np.float64)
    y = O.check(synth.Scene(w.scene.arm, path[0], 0.03), X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, 20000, w.s_max, store32=store32)
    m = fk.fastron_model_create(ch)
    Xd = torch.empty((n_max, 7), dtype=torch.float64, device=dev)
    X32 = torch.empty((n_max, 7), dtype=torch.float32, device=dev)
    try:
        st = fk.fastron_train(m, torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), w.gamma, w.beta, 20000,
                              w.s_max, gram=code)
        assert st["n_support"] == r.n_support
        S, aS = X[r.support], r.alpha[r.support]
        for k in range(1, frames):
            ns = len(S)
            nu = max(0, n_max - 2 * ns)
            seed = 1000 + k
            n = fk.fk_active_samples(m, 1, sigma, nu, qlim, seed, Xd, X32)
            Xk = O.active_samples(S, 1, sigma, nu, qlim, seed)
            assert n == len(Xk) and np.array_equal(Xd[:n].cpu().numpy(), Xk)
            yk = O.check(synth.Scene(w.scene.arm, path[k], 0.03), Xk)
            ty = torch.empty(n, dtype=torch.int8, device=dev)
            fk.fk_label(ch, path[k], 0.03, X32[:n], ty)
            assert np.array_equal(ty.cpu().numpy(), yk)
            cp = O.fk_points(w.scene.arm, Xk)
            F0 = O.margins(cp, ns, aS, w.gamma, store32=store32)
            a0 = np.zeros(n)
            a0[:ns] = aS
            r = O.fastron_train(cp, yk, w.gamma, w.beta, 20000, w.s_max, alpha0=a0, F0=F0, trace=True,
                                store32=store32)
            st = fk.fastron_train(m, Xd[:n], ty, w.gamma, w.beta, 20000, w.s_max, warm_start=2, trace=True,
                                  gram=code)
            assert (st["iterations"], st["n_support"], st["converged"]) == (r.iters, r.n_support, r.converged)
            _compare_trace(fk, m, r, store32)
            S, aS = Xk[r.support], r.alpha[r.support]
    finally:
        fk.fastron_model_destroy(m)


def test_new_entry_points_reject_bad_arguments(fk, arm12, dev):
    w, ch = arm12
    X = torch.from_numpy(w.train_configs()[:200].astype(np.float64)).to(dev)
    y = _labels(fk, ch, w.scene.boxes, X.cpu().numpy(), dev)
    out = torch.empty((1000, 7), dtype=torch.float64, device=dev)
    m = fk.fastron_model_create(ch)
    try:
        with pytest.raises(fk.FkError) as e:  # untrained model: nothing to carry or sample from
            fk.fk_active_samples(m, 1, 0.1, 10, w.scene.arm.qlim, 1, out)
        assert e.value.code == fk.FK_ERR_STATE
        with pytest.raises(fk.FkError) as e:
            fk.fastron_train(m, X, y, w.gamma, warm_start=2)
        assert e.value.code == fk.FK_ERR_STATE
        fk.fastron_train(m, X, y, w.gamma, gram=fk.FK_DF32)
        ns = fk.fastron_model_get(m)[0].shape[0]
        for bad in ((-1, 0.1, 10, w.scene.arm.qlim), (1, -0.1, 10, w.scene.arm.qlim), (1, 0.1, -5, w.scene.arm.qlim),
                    (1, 0.1, 10, 0.0), (1, float("nan"), 10, w.scene.arm.qlim)):
            with pytest.raises(fk.FkError) as e:
                fk.fk_active_samples(m, *bad, 1, out)
            assert e.value.code == fk.FK_ERR_ARG
        with pytest.raises(fk.FkError) as e:  # a changed training set cannot reuse the matrix
            fk.fastron_train(m, X, y, w.gamma, warm_start=2, reuse_gram=True, gram=fk.FK_DF32)
        assert e.value.code == fk.FK_ERR_ARG
        with pytest.raises(fk.FkError) as e:  # fewer rows than the carried support set
            fk.fastron_train(m, X[:ns - 1], y[:ns - 1], w.gamma, warm_start=2)
        assert e.value.code == fk.FK_ERR_STATE
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, X, y, w.gamma, warm_start=3)
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, X, y, w.gamma, gram=99)
        # a carried model on its own support set plus nothing new is a fixed point
        n = fk.fk_active_samples(m, 0, 0.0, 0, w.scene.arm.qlim, 1, out)
        assert n == ns
        sup, alpha = fk.fastron_model_get(m)
        yy = y[torch.from_numpy(sup).to(dev)]
        st = fk.fastron_train(m, out[:n], yy.contiguous(), w.gamma, warm_start=2, gram=fk.FK_DF32)
        assert st["converged"] and st["iterations"] <= ns
    finally:
        fk.fastron_model_destroy(m)
