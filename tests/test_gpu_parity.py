"""Parity of the CUDA library against the FP64 oracle, element by element,
through the C ABI.  Tolerances:

  control points (FP32)   |dp| <= 1e-5 * max(|p|, reach)
  control points (FP64)   |dp| <= 1e-13
  kernel matrix (FP64)    |dK| <= 1e-14;  (FP32) |dK| <= 2e-6
  score (FP32, tier 1)    |df| <= 1e-4 * sum|alpha|   and   |df| <= eps(q) B(q),
                          B(q) = sum_s |alpha_s| K_FK(S_s, q), eps(q) the derived
                          re-score band (tests/_band.py), on every query
  labels after re-score   identical
  training                support set, pass sequence identical; alpha within 1e-12 relative
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth
from tests import _band

pytestmark = pytest.mark.gpu


def _reach(arm):
    return float(np.sum(np.hypot(arm.dh[:, 0], arm.dh[:, 2])))


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def arm3(fk):
    w = synth.workload("arm3-n1000")
    ch = fk.chain_from_arm(w.scene.arm)
    yield w, ch
    fk.fk_chain_destroy(ch)


@pytest.fixture(scope="module")
def arm7(fk):
    w = synth.workload("arm7-n5000")
    ch = fk.chain_from_arm(w.scene.arm)
    yield w, ch
    fk.fk_chain_destroy(ch)


def _cp_soa_to_aos(cp):
    return cp.permute(2, 0, 1).cpu().numpy()  # (M, 3, n) -> (n, M, 3)


@pytest.mark.parametrize("n", [1, 31, 257, 10001])
@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_fk_forward(fk, arm3, arm7, dev, n, which):
    w, ch = arm3 if which == "arm3" else arm7
    arm = w.scene.arm
    q = w.query_configs(n)
    want = O.fk_points(arm, q.astype(np.float64))
    cp32 = torch.empty((arm.M, 3, n), dtype=torch.float32, device=dev)
    fk.fk_forward(ch, torch.from_numpy(q).to(dev), cp32)
    cp64 = torch.empty((arm.M, 3, n), dtype=torch.float64, device=dev)
    fk.fk_forward_f64(ch, torch.from_numpy(q.astype(np.float64)).to(dev), cp64)
    got32, got64 = _cp_soa_to_aos(cp32), _cp_soa_to_aos(cp64)
    scale = np.maximum(np.linalg.norm(want, axis=2, keepdims=True), _reach(arm))
    assert np.all(np.abs(got32 - want) <= 1e-5 * scale)
    assert np.max(np.abs(got64 - want)) <= 1e-13


@pytest.mark.parametrize("na,nb", [(77, 77), (1000, 1000), (50, 33), (1, 5)])
def test_gram(fk, arm3, dev, na, nb):
    w, ch = arm3
    arm = w.scene.arm
    Xa = w.train_configs()[:na].astype(np.float64)
    Xb = Xa if na == nb else w.query_configs(nb).astype(np.float64)
    want = O.gram(O.fk_points(arm, Xa), O.fk_points(arm, Xb), w.gamma)
    ta = torch.from_numpy(Xa).to(dev)
    tb = ta if na == nb else torch.from_numpy(Xb).to(dev)
    K = torch.empty((na, nb), dtype=torch.float64, device=dev)
    fk.fk_gram(ch, ta, tb, w.gamma, K)
    got = K.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-14
    if na == nb:
        assert np.array_equal(got, got.T)
        assert np.all(np.diag(got) == 1.0)
    Kd = torch.empty((na, nb), dtype=torch.float64, device=dev)
    fk.fk_gram(ch, ta, tb, w.gamma, Kd, double_float=True)
    gotd = Kd.cpu().numpy()
    assert np.max(np.abs(gotd - want)) <= 2e-13
    if na == nb:
        assert np.array_equal(gotd, gotd.T)
        assert np.all(np.diag(gotd) == 1.0)
    K32 = torch.empty((na, nb), dtype=torch.float32, device=dev)
    t32a = ta.float()
    fk.fk_gram(ch, t32a, t32a if na == nb else tb.float(), w.gamma, K32)
    assert np.max(np.abs(K32.cpu().numpy() - want)) <= 2e-6


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_labels(fk, arm3, arm7, dev, which):
    w, ch = arm3 if which == "arm3" else arm7
    q = w.query_configs(20000)
    want = O.check(w.scene, q.astype(np.float64))
    y = torch.empty(20000, dtype=torch.int8, device=dev)
    fk.fk_label(ch, w.scene.boxes, w.scene.radius, torch.from_numpy(q).to(dev), y)
    got = y.cpu().numpy()
    assert np.array_equal(got, want)
    assert 0 < np.sum(want == 1) < len(want)


@pytest.mark.parametrize("gap", [0.0, 1e-7, -1e-7, 3e-6, 2e-5])
def test_labels_at_the_radius(fk, arm3, dev, gap):
    # the first link of the 3-DOF arm lies in the plane z = 0; a box whose
    # lower face is at z = radius + gap puts every configuration within |gap|
    # of the decision, so the FP32 filter must hand them to FP64
    w, ch = arm3
    q = w.query_configs(4000)
    boxes = np.array([[-0.6, -0.6, 0.03 + gap, 0.6, 0.6, 0.6]])
    sc = synth.Scene(w.scene.arm, boxes, 0.03)
    want = O.check(sc, q.astype(np.float64))
    y = torch.empty(len(q), dtype=torch.int8, device=dev)
    fk.fk_label(ch, boxes, 0.03, torch.from_numpy(q).to(dev), y)
    assert np.array_equal(y.cpu().numpy(), want)


def _train_both(fk, w, ch, dev, n=None, beta=None, gram=None):
    X = w.train_configs()[:n].astype(np.float64)
    y = O.check(w.scene, X)
    beta = w.beta if beta is None else beta
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, beta, w.iter_max, w.s_max, trace=True)
    m = fk.fastron_model_create(ch)
    st = fk.fastron_train(m, torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), w.gamma, beta,
                          w.iter_max, w.s_max, trace=True, gram=fk.FK_DF64 if gram is None else gram)
    return X, y, r, m, st


@pytest.mark.parametrize("gram", ["df64", "f64"])
@pytest.mark.parametrize("which,n,beta", [("arm3", 1000, 1.0), ("arm3", 1000, 1.5), ("arm3", 333, 1.0),
                                          ("arm7", 5000, 1.0)])
def test_fastron_train_matches_oracle(fk, arm3, arm7, dev, which, n, beta, gram):
    w, ch = arm3 if which == "arm3" else arm7
    X, y, r, m, st = _train_both(fk, w, ch, dev, n, beta, fk.FK_DF64 if gram == "df64" else fk.FK_F64)
    try:
        assert st["iterations"] == r.iters and st["adds"] == r.adds and st["removes"] == r.removes
        assert st["converged"] == r.converged and st["n_support"] == r.n_support
        kind, idx, delta = fk.fastron_model_trace(m, r.iters + 1)
        assert np.array_equal(kind, r.trace[0]) and np.array_equal(idx, r.trace[1])
        np.testing.assert_allclose(delta, r.trace[2], rtol=1e-12, atol=1e-12)
        gidx, galpha = fk.fastron_model_get(m)
        assert np.array_equal(gidx, r.support)
        np.testing.assert_allclose(galpha, r.alpha[r.support], rtol=1e-12)
    finally:
        fk.fastron_model_destroy(m)


def test_fastron_train_limits_and_warm_start(fk, arm3, dev):
    w, ch = arm3
    X = w.train_configs()[:400].astype(np.float64)
    y = O.check(w.scene, X)
    cp = O.fk_points(w.scene.arm, X)
    tX, ty = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
    m = fk.fastron_model_create(ch)
    try:
        for it, smax in ((7, 400), (5000, 6)):
            r = O.fastron_train(cp, y, w.gamma, 1.0, it, smax)
            st = fk.fastron_train(m, tX, ty, w.gamma, 1.0, it, smax)
            assert (st["iterations"], st["n_support"], st["converged"]) == (r.iters, r.n_support, r.converged)
            assert np.array_equal(fk.fastron_model_get(m)[0], r.support)
        # warm start continues from the last alpha and F (loadPreviousModel)
        r1 = O.fastron_train(cp, y, w.gamma, 1.0, 9)
        r2 = O.fastron_train(cp, y, w.gamma, 1.0, 5000, alpha0=r1.alpha, F0=r1.F)
        fk.fastron_train(m, tX, ty, w.gamma, 1.0, 9)
        st = fk.fastron_train(m, tX, ty, w.gamma, 1.0, 5000, warm_start=True)
        assert st["iterations"] == r2.iters and np.array_equal(fk.fastron_model_get(m)[0], r2.support)
        st = fk.fastron_train(m, tX, ty, w.gamma, 1.0, 5000, warm_start=True)
        assert st["iterations"] == 0 and st["converged"]
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, tX[:10], ty[:10], w.gamma, 1.0, 10, warm_start=True)
    finally:
        fk.fastron_model_destroy(m)


def _score_case(fk, w, ch, dev, S, alpha, Q, circle=True):
    arm = w.scene.arm
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        n = Q.shape[0]
        tq = torch.from_numpy(Q).to(dev)
        f_raw = torch.empty(n, dtype=torch.float32, device=dev)
        lab_raw = torch.empty(n, dtype=torch.int8, device=dev)
        fk.fk_score(m, tq, lab_raw, f_raw, rescore=False)
        f = torch.empty(n, dtype=torch.float32, device=dev)
        lab = torch.empty(n, dtype=torch.int8, device=dev)
        nres = fk.fk_score(m, tq, lab, f, rescore=True, count=True)
        torch.cuda.synchronize()
        eps0, eps1 = fk.fk_score_band(m)
        cnorm = fk.fk_score_circle(m)
    finally:
        fk.fastron_model_destroy(m)
    # the library's band constants are the derivation's
    assert (eps0, eps1) == _band.constants(arm, w.gamma, len(S))
    assert cnorm == pytest.approx(_band.circle_norm(arm, w.gamma, len(S), on=circle), rel=1e-6, abs=0.0)
    Qd = Q.astype(np.float64)
    cps, cpq = O.fk_points(arm, S), O.fk_points(arm, Qd)
    want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=8)
    B = O.score_points(cps, np.abs(alpha), cpq, w.gamma, nthreads=8)
    eps = _band.per_query(arm, w.gamma, eps0, eps1, cps, cpq, cnorm)
    return f_raw.cpu().numpy(), lab_raw.cpu().numpy(), f.cpu().numpy(), lab.cpu().numpy(), nres, want, B, eps


def _check_score(f_raw, lab_raw, f, lab, nres, want, B, eps, alpha):
    sa = np.sum(np.abs(alpha))
    err = np.abs(f_raw.astype(np.float64) - want)
    assert np.all(err <= 1e-4 * sa + 1e-30)
    # the derived bound holds on every query (with the FP64 B(q) and norms)
    assert np.all(err <= eps * B + 1e-30), np.max(err / np.maximum(eps * B, 1e-300))
    assert np.array_equal(lab_raw == 1, f_raw >= 0)
    assert np.array_equal(lab, O.labels_from_f(want))
    # the band holds every query the bound cannot decide, and not many more
    assert nres >= np.sum(np.abs(f_raw.astype(np.float64)) < 0.999 * eps * B)
    assert nres <= np.sum(np.abs(f_raw.astype(np.float64)) <= 1.001 * eps * B) + 8
    # re-scored queries carry the FP64 value (rounded to FP32)
    sel = np.abs(f_raw.astype(np.float64)) < 0.999 * eps * B
    np.testing.assert_allclose(f[sel], want[sel].astype(np.float32), rtol=1e-6, atol=1e-30)


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_score_trained_model(fk, arm3, arm7, dev, which):
    w, ch = arm3 if which == "arm3" else arm7
    X = w.train_configs().astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max)
    S, alpha = X[r.support], r.alpha[r.support]
    Q = w.query_configs(10000 if which == "arm3" else 20000)
    out = _score_case(fk, w, ch, dev, S, alpha, Q)
    _check_score(*out, alpha)


def test_score_circle_form_on_and_off(fk, arm7, dev):
    # the first control point of the 7-DOF arm sits on frame 1 of a revolute
    # joint: the FP32 kernel takes its summand in the circle form unless it is
    # switched off; both forms give the oracle's labels, and their FP32 values
    # differ by no more than the two bounds
    w, ch = arm7
    rng = np.random.default_rng(41)
    S = w.train_configs()[:801].astype(np.float64)
    alpha = rng.normal(size=len(S)) * 2
    Q = w.query_configs(30001)
    # queries whose joint-1 angle nearly equals a support point's (the circle
    # form's worst case: t close to 1 by cancellation)
    Q[:5000, 0] = (S[rng.integers(0, len(S), 5000), 0] + rng.normal(size=5000) * 1e-5).astype(np.float32)
    fk.fk_set_circle_form(False)
    try:
        off = _score_case(fk, w, ch, dev, S, alpha, Q, circle=False)
    finally:
        fk.fk_set_circle_form(True)
    on = _score_case(fk, w, ch, dev, S, alpha, Q)
    assert _band.circle_norm(w.scene.arm, w.gamma, len(S)) > 0
    _check_score(*off, alpha)
    _check_score(*on, alpha)
    B = on[6]
    assert np.all(np.abs(on[0].astype(np.float64) - off[0]) <= (on[7] + off[7]) * B)
    assert not np.array_equal(on[0], off[0])  # the two forms do differ in rounding
    assert np.array_equal(on[3], off[3])


def test_score_circle_norm_zero_without_a_circle(fk, arm7, dev):
    # joint 1 prismatic: no circle; the direct form throughout
    w, _ = arm7
    arm = w.scene.arm
    dh = arm.dh.copy()
    dh[0, 4] = synth.PRISMATIC
    arm_p = synth.Arm(dh=dh, base=arm.base, cp_joint=arm.cp_joint, cp_off=arm.cp_off, qlim=arm.qlim)
    assert _band.circle_norm(arm_p, w.gamma, 800) == 0.0
    ch = fk.chain_from_arm(arm_p)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, w.train_configs()[:800].astype(np.float64), np.ones(800), w.gamma)
        assert fk.fk_score_circle(m) == 0.0
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


@pytest.mark.parametrize("ns,n", [(0, 100), (1, 1), (1, 513), (127, 700), (128, 512), (129, 1025), (300, 3)])
def test_score_edge_sizes(fk, arm7, dev, ns, n):
    w, ch = arm7
    rng = np.random.default_rng(ns * 7 + n)
    S = w.train_configs()[:ns].astype(np.float64)
    alpha = rng.normal(size=ns) * 3
    Q = w.query_configs(n)
    out = _score_case(fk, w, ch, dev, S, alpha, Q)
    if ns == 0:
        assert np.all(out[2] == 0) and np.all(out[3] == 1)
    else:
        _check_score(*out, alpha)


def test_score_query_equal_to_support_point(fk, arm7, dev):
    # K(x, x) = 1: a single support point scored at itself gives alpha
    w, ch = arm7
    S = w.train_configs()[:1].astype(np.float64)
    f_raw, lab_raw, f, lab, nres, want, B, eps = _score_case(fk, w, ch, dev, S, np.array([-0.75]), S.astype(np.float32))
    assert want[0] == -0.75
    assert abs(f_raw[0] + 0.75) <= 1e-6 and lab[0] == -1


def _ulps32(a, b):
    ia = np.asarray(a, dtype=np.float32).view(np.int32).astype(np.int64)
    ib = np.asarray(b, dtype=np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_score_double_float_tier_on_every_query(fk, arm3, arm7, dev, which):
    # a band of eps = 1 holds every query (|f| <= B(q) always), so the
    # double-float tier evaluates all of them: its f, rounded to FP32, is the
    # FP64 value rounded to FP32 (1 ulp where the FP64 value sits on a
    # rounding boundary within the pair error)
    w, ch = arm3 if which == "arm3" else arm7
    X = w.train_configs()[:1500].astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max)
    S, alpha = X[r.support], r.alpha[r.support]
    Q = w.query_configs(6000)
    want = O.score(w.scene.arm, S, alpha, Q.astype(np.float64), w.gamma, nthreads=8)
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
    assert u.max() <= 1 and np.mean(u > 0) <= 1e-3
    assert np.array_equal(lab.cpu().numpy(), O.labels_from_f(want))


def test_score_cancelling_support_points_reach_fp64(fk, arm7, dev):
    # the same configuration twice with weights +1 and -1: f = 0 exactly for
    # every query, which no reduced precision can decide; the FP64 re-score
    # returns 0 and the label of f = 0, +1
    w, ch = arm7
    x = w.train_configs()[:1].astype(np.float64)
    S = np.concatenate([x, x])
    Q = w.query_configs(1000)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, np.array([1.0, -1.0]), w.gamma)
        tq = torch.from_numpy(Q).to(dev)
        f = torch.full((len(Q),), 7.0, dtype=torch.float32, device=dev)
        lab = torch.zeros(len(Q), dtype=torch.int8, device=dev)
        nres = fk.fk_score(m, tq, lab, f, rescore=True, count=True)
        torch.cuda.synchronize()
    finally:
        fk.fastron_model_destroy(m)
    assert nres == len(Q)
    assert np.all(f.cpu().numpy() == 0.0) and np.all(lab.cpu().numpy() == 1)


def test_score_timeout_path_reports_and_recovers(fk, arm7, dev):
    # a tile wait that gives up at once returns FK_ERR_TIMEOUT; the context
    # stays usable and the next call with the normal limit succeeds
    w, ch = arm7
    S = w.train_configs()[:300].astype(np.float64)
    alpha = np.random.default_rng(0).normal(size=300)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        q = torch.from_numpy(w.query_configs(4096)).to(dev)
        lab = torch.empty(4096, dtype=torch.int8, device=dev)
        fk.fk_set_wait_limit(0)
        try:
            with pytest.raises(fk.FkError) as e:
                fk.fk_score(m, q, lab, rescore=True, count=True)
            assert e.value.code == fk.FK_ERR_TIMEOUT
        finally:
            fk.fk_set_wait_limit(1 << 22)
        fk.fk_score(m, q, lab, rescore=True, count=True)
    finally:
        fk.fastron_model_destroy(m)


@pytest.mark.parametrize("n", [333, 1000, 5000])
def test_training_timeout_path_reports_and_recovers(fk, arm3, arm7, dev, n):
    # the cluster exchange of Algorithm 1 giving up at once returns
    # FK_ERR_TIMEOUT (a cluster of 1 CTA at 333 points, 2 at 1000, 16 at
    # 5000); the context stays usable, warm start and matrix reuse are
    # refused, and the next cold call with the normal limit reproduces the
    # oracle's model
    w, ch = arm3 if n < 5000 else arm7
    X = w.train_configs()[:n].astype(np.float64)
    y = O.check(w.scene, X)
    Xt, yt = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
    m = fk.fastron_model_create(ch)
    try:
        fk.fk_set_wait_limit(0)
        try:
            with pytest.raises(fk.FkError) as e:
                fk.fastron_train(m, Xt, yt, w.gamma, w.beta, w.iter_max, w.s_max)
            assert e.value.code == fk.FK_ERR_TIMEOUT
        finally:
            fk.fk_set_wait_limit(1 << 22)
        for kw in ({"warm_start": True}, {"reuse_gram": True}):
            with pytest.raises(fk.FkError) as e:
                fk.fastron_train(m, Xt, yt, w.gamma, w.beta, w.iter_max, w.s_max, **kw)
            assert e.value.code == fk.FK_ERR_STATE
        st = fk.fastron_train(m, Xt, yt, w.gamma, w.beta, w.iter_max, w.s_max)
        r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max)
        assert st["n_support"] == len(r.support) and st["iterations"] == r.iters
        idx, alpha = fk.fastron_model_get(m)
        np.testing.assert_array_equal(idx, r.support)
        np.testing.assert_allclose(alpha, r.alpha[r.support], rtol=1e-12, atol=0)
    finally:
        fk.fastron_model_destroy(m)


def test_empty_batches_are_no_ops(fk, arm7, dev):
    """Zero configurations, zero queries and an empty side of the kernel
    matrix return FK_OK without a launch, and the next full call still
    matches the oracle."""
    w, ch = arm7
    arm = w.scene.arm
    e32 = torch.empty((0, arm.D), dtype=torch.float32, device=dev)
    e64 = torch.empty((0, arm.D), dtype=torch.float64, device=dev)
    fk.fk_forward(ch, e32, torch.empty((arm.M, 3, 0), dtype=torch.float32, device=dev))
    fk.fk_forward_f64(ch, e64, torch.empty((arm.M, 3, 0), dtype=torch.float64, device=dev))
    fk.fk_label(ch, w.scene.boxes, w.scene.radius, e32, torch.empty(0, dtype=torch.int8, device=dev))
    X = torch.from_numpy(w.train_configs()[:40].astype(np.float64)).to(dev)
    fk.fk_gram(ch, e64, X, w.gamma, torch.empty((0, 40), dtype=torch.float64, device=dev))
    fk.fk_gram(ch, X, e64, w.gamma, torch.empty((40, 0), dtype=torch.float64, device=dev))
    Xn = X.cpu().numpy()
    y = O.check(w.scene, Xn)
    r = O.fastron_train(O.fk_points(arm, Xn), y, w.gamma, w.beta, w.iter_max, w.s_max)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, Xn[r.support], r.alpha[r.support], w.gamma)
        assert fk.fk_score(m, e32, torch.empty(0, dtype=torch.int8, device=dev), count=True) == 0
        Q = w.query_configs(300)
        lab = torch.empty(300, dtype=torch.int8, device=dev)
        fk.fk_score(m, torch.from_numpy(Q).to(dev), lab)
        want = O.labels_from_f(O.score(arm, Xn[r.support], r.alpha[r.support], Q.astype(np.float64), w.gamma))
        np.testing.assert_array_equal(lab.cpu().numpy(), want)
    finally:
        fk.fastron_model_destroy(m)


def test_argument_errors(fk, arm3, dev):
    w, ch = arm3
    m = fk.fastron_model_create(ch)
    try:
        q = torch.zeros((4, 3), dtype=torch.float32, device=dev)
        lab = torch.empty(4, dtype=torch.int8, device=dev)
        with pytest.raises(fk.FkError) as e:
            fk.fk_score(m, q, lab)
        assert e.value.code == fk.FK_ERR_STATE
        X = torch.zeros((65537, 3), dtype=torch.float64, device=dev)
        y = torch.ones(65537, dtype=torch.int8, device=dev)
        with pytest.raises(fk.FkError) as e:
            fk.fastron_train(m, X, y, 10.0)
        assert e.value.code == fk.FK_ERR_CAPACITY
        with pytest.raises(fk.FkError):
            fk.fastron_train(m, X[:10], y[:10], -1.0)
        with pytest.raises(ValueError):
            fk.fk_score(m, q.double(), lab)
    finally:
        fk.fastron_model_destroy(m)


@pytest.mark.parametrize("which", ["arm3", "arm7"])
def test_score_half_precision_path(fk, arm3, arm7, dev, which):
    """Packed-half distances: the half pass stays within its band bound and,
    after its band goes through the FP32 path and the FP64 re-score, every
    label equals the oracle's."""
    w, ch = arm3 if which == "arm3" else arm7
    X = w.train_configs().astype(np.float64)
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max)
    S, alpha = X[r.support], r.alpha[r.support]
    Q = w.query_configs(20000)
    m = fk.fastron_model_create(ch)
    try:
        fk.fastron_model_set(m, S, alpha, w.gamma)
        tq = torch.from_numpy(Q).to(dev)
        f16 = torch.empty(len(Q), dtype=torch.float32, device=dev)
        l16 = torch.empty(len(Q), dtype=torch.int8, device=dev)
        fk.fk_score(m, tq, l16, f16, rescore=False, precision=fk.FK_F16)
        lab = torch.empty(len(Q), dtype=torch.int8, device=dev)
        nb = fk.fk_score(m, tq, lab, rescore=True, count=True, precision=fk.FK_F16)
        torch.cuda.synchronize()
        eps0, eps1 = fk.fk_score_band(m, fk.FK_F16)
    finally:
        fk.fastron_model_destroy(m)
    assert (eps0, eps1) == _band.constants(w.scene.arm, w.gamma, len(S), half=True)
    cps, cpq = O.fk_points(w.scene.arm, S), O.fk_points(w.scene.arm, Q.astype(np.float64))
    want = O.score_points(cps, alpha, cpq, w.gamma, nthreads=8)
    B = O.score_points(cps, np.abs(alpha), cpq, w.gamma, nthreads=8)
    eps = _band.per_query(w.scene.arm, w.gamma, eps0, eps1, cps, cpq)
    err = np.abs(f16.cpu().numpy().astype(np.float64) - want)
    print(f"half pass: max |df|/(eps B) = {np.max(err / (eps * B)):.3e}, band = {nb} of {len(Q)}")
    assert np.all(err <= eps * B)
    assert np.array_equal(lab.cpu().numpy(), O.labels_from_f(want))


@pytest.mark.parametrize("pattern", ["all_pos", "all_neg", "odd_odd", "even_odd", "one_pos"])
def test_score_sign_ordered_records(fk, arm7, dev, pattern):
    # the pair records hold the positive weights first, each sign group
    # padded to an even count: every mix of group sizes scores as the oracle
    w, ch = arm7
    rng = np.random.default_rng(len(pattern))
    n_pos, n_neg = {"all_pos": (129, 0), "all_neg": (0, 130), "odd_odd": (63, 65), "even_odd": (64, 33),
                    "one_pos": (1, 200)}[pattern]
    S = w.train_configs()[:n_pos + n_neg].astype(np.float64)
    mag = rng.uniform(0.5, 3.0, n_pos + n_neg)
    sign = np.concatenate([np.ones(n_pos), -np.ones(n_neg)])
    alpha = mag * sign[rng.permutation(n_pos + n_neg)]  # signs interleaved in support order
    Q = w.query_configs(3001)
    out = _score_case(fk, w, ch, dev, S, alpha, Q)
    _check_score(*out, alpha)
