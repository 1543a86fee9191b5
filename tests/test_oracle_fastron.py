"""Pins of the oracle's Fastron update, Algorithm 1 (Sec. III-B): closed-form
tiny cases, the update rule's invariants (Eqs. 6-8), the loss decrease and step
bound of Claim 2, and the S_max cap."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_06451_gb300 import synth


def _small_problem(n=150, seed=0, name="arm3-n1000"):
    w = synth.workload(name, trial=seed)
    X = w.train_configs()[:n].astype(np.float64)
    y = O.check(w.scene, X)
    cp = O.fk_points(w.scene.arm, X)
    return w, X, y, cp


def test_single_point():
    cp = np.zeros((1, 2, 3))
    for y, beta, want in ((1, 1.5, 1.5), (-1, 1.5, -1.0), (1, 1.0, 1.0)):
        r = O.fastron_train(cp, np.array([y]), 10.0, beta=beta, iter_max=100, trace=True)
        assert r.converged and r.adds == 1 and r.removes == 0 and r.iters == 1
        assert r.alpha[0] == want and r.F[0] == want
        assert list(r.support) == [0]


def _two_points(sep):
    cp = np.zeros((2, 1, 3))
    cp[1, 0, 0] = sep
    return cp


def test_two_points_opposite_labels_closed_form():
    g = 10.0
    cp = _two_points(0.3)
    k = O.k_fk(cp[0], cp[1], g)
    assert k < 0.6
    r = O.fastron_train(cp, np.array([1, -1]), g, iter_max=100, trace=True)
    # pass 1: all margins 0, tie -> index 0, delta = 1; pass 2: index 1 with
    # margin -k, delta = -1 - k; then every margin is positive, nothing to remove
    kind, idx, delta = r.trace
    assert list(kind) == [1, 1] and list(idx) == [0, 1]
    assert delta[0] == 1.0 and delta[1] == pytest.approx(-1 - k, rel=1e-15)
    np.testing.assert_allclose(r.alpha, [1.0, -1.0 - k], rtol=1e-15)
    np.testing.assert_allclose(r.F, [1 - k - k * k, -1.0], rtol=1e-14)
    assert r.converged and list(r.support) == [0, 1]


def test_adjusting_a_support_point_when_the_set_is_full():
    # two close points of opposite labels, k > (sqrt 5 - 1) / 2: after both
    # are added, F_0 = 1 - k - k^2 < 0, so pass 3 adjusts point 0 although the
    # support set is full (S_max = 2 = N): delta = 1 - F_0 = k + k^2 (Eq. 6)
    g = 10.0
    cp = _two_points(0.1)
    k = O.k_fk(cp[0], cp[1], g)
    assert k > (5 ** 0.5 - 1) / 2
    r = O.fastron_train(cp, np.array([1, -1]), g, iter_max=3, s_max=2, trace=True)
    kind, idx, delta = r.trace
    assert list(kind) == [1, 1, 1] and list(idx) == [0, 1, 0]
    assert delta[2] == pytest.approx(k + k * k, rel=1e-14)
    assert r.alpha[0] == pytest.approx(1 + k + k * k, rel=1e-14)


def test_removal_ties_go_to_the_lowest_index():
    # two pairs of coincident points (K = 1 within a pair, e between pairs),
    # all labelled +1, warm-started with every alpha = 1 and F = K alpha =
    # 2 + 2e: every removal margin y (F - alpha) is the same positive value,
    # and the removal takes the lowest index
    g = 10.0
    cp = np.zeros((4, 1, 3))
    cp[2:, 0, 0] = 0.5
    e = O.k_fk(cp[0], cp[2], g)
    r = O.fastron_train(cp, np.ones(4, dtype=np.int8), g, iter_max=1, alpha0=np.ones(4),
                        F0=np.full(4, 2.0 + 2.0 * e), trace=True)
    assert list(r.trace[0]) == [2] and list(r.trace[1]) == [0]
    assert r.alpha[0] == 0.0 and np.all(r.alpha[1:] == 1.0)


def test_two_points_same_label_keeps_one():
    cp = _two_points(0.2)
    r = O.fastron_train(cp, np.array([1, 1]), 10.0, iter_max=100, trace=True)
    assert list(r.trace[0]) == [1] and list(r.trace[1]) == [0]
    assert list(r.support) == [0] and r.converged


def test_redundant_point_is_removed():
    # four points on a line: after points 0, 3 and 1 are added, point 0 keeps a
    # positive margin without its own weight, y_0 (F_0 - alpha_0) > 0, so the
    # removal step sets alpha_0 = 0 and every margin stays positive.
    g = 10.0
    cp = np.zeros((4, 1, 3))
    cp[:, 0, 0] = [0.4, 0.73, 0.71, 0.93]
    y = np.array([-1, -1, -1, 1])
    r = O.fastron_train(cp, y, g, iter_max=100, trace=True)
    kind, idx, delta = r.trace
    assert list(kind) == [1, 1, 1, 2] and list(idx) == [0, 3, 1, 0]
    K = O.gram(cp, cp, g)
    a3 = np.zeros(4)
    for k in range(3):
        a3[idx[k]] += delta[k]
    F3 = K @ a3
    assert y[0] * (F3[0] - a3[0]) > 0
    assert delta[3] == -a3[0]
    assert r.converged and list(r.support) == [1, 3]
    assert np.all(y * r.F > 0)
    np.testing.assert_allclose(r.F, K @ r.alpha, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("beta", [1.0, 1.5])
def test_update_invariants_and_loss_decrease(beta):
    w, X, y, cp = _small_problem(120, seed=1)
    K = O.gram(cp, cp, w.gamma)
    b = np.where(y > 0, beta, 1.0)
    full = O.fastron_train(cp, y, w.gamma, beta=beta, iter_max=5000, trace=True)
    kind, idx, delta = full.trace
    assert full.converged and full.iters == len(kind)
    prev_alpha = np.zeros(len(y))
    for k in range(len(kind)):
        r = O.fastron_train(cp, y, w.gamma, beta=beta, iter_max=k + 1)
        i = idx[k]
        # the incrementally maintained F is K alpha
        np.testing.assert_allclose(r.F, K @ r.alpha, rtol=1e-10, atol=1e-10)
        if kind[k] == 1:
            # after an add step the point sits exactly at its target margin: F_i = b_i y_i
            assert r.F[i] == pytest.approx(b[i] * y[i], abs=1e-12)
            # loss L = 1/2 a'Ka - y'Ba falls by exactly 1/2 (b_i - m_i)^2 (Claim 2)
            m_i = y[i] * (K @ prev_alpha)[i]
            L0 = 0.5 * prev_alpha @ K @ prev_alpha - (y * b) @ prev_alpha
            L1 = 0.5 * r.alpha @ K @ r.alpha - (y * b) @ r.alpha
            assert L1 - L0 == pytest.approx(-0.5 * (b[i] - m_i) ** 2, rel=1e-8, abs=1e-10)
            assert m_i <= 0
        else:
            assert r.alpha[i] == 0.0 and prev_alpha[i] != 0.0
        prev_alpha = r.alpha
    assert np.all(y * full.F > 0)
    # no support point is redundant at the end
    sup = full.alpha != 0
    assert not np.any(y[sup] * (full.F[sup] - full.alpha[sup]) > 0)


def test_add_step_bound_of_claim_2():
    # number of descent steps <= y'BK^-1By + 2 L(alpha0), alpha0 = 0
    w, X, y, cp = _small_problem(150, seed=2)
    K = O.gram(cp, cp, w.gamma)
    By = y.astype(float)
    bound = By @ np.linalg.solve(K, By)
    r = O.fastron_train(cp, y, w.gamma, iter_max=100000)
    assert r.converged
    assert r.adds <= bound


def test_smax_caps_support_size_and_iter_max_stops():
    w, X, y, cp = _small_problem(200, seed=3)
    r = O.fastron_train(cp, y, w.gamma, iter_max=5000, s_max=5, trace=True)
    assert r.n_support <= 5
    r2 = O.fastron_train(cp, y, w.gamma, iter_max=3)
    assert r2.iters == 3 and not r2.converged


def test_warm_start_is_a_fixed_point():
    w, X, y, cp = _small_problem(200, seed=4)
    r = O.fastron_train(cp, y, w.gamma)
    r2 = O.fastron_train(cp, y, w.gamma, alpha0=r.alpha, F0=r.F)
    assert r2.converged and r2.iters == 0
    assert np.array_equal(r2.alpha, r.alpha)


def test_workloads_train_to_positive_margins():
    w, X, y, cp = _small_problem(1000, seed=0)
    r = O.fastron_train(cp, y, w.gamma, iter_max=w.iter_max)
    assert r.converged and np.all(y * r.F > 0)
    assert 0 < r.n_support < 1000


def test_fp32_stored_kernel_two_points_closed_form():
    # the same two passes as above with K_01 rounded to FP32
    g = 10.0
    cp = _two_points(0.3)
    k = O.k_fk(cp[0], cp[1], g)
    k32 = float(np.float32(k))
    assert k32 != k
    r = O.fastron_train(cp, np.array([1, -1]), g, iter_max=100, trace=True, store32=True)
    kind, idx, delta = r.trace
    assert list(kind) == [1, 1] and list(idx) == [0, 1]
    assert delta[1] == -1.0 - k32
    # F_0 = fma(-1 - k32, k32, 1): one rounding of the exact 1 - k32 - k32^2
    assert r.alpha[1] == -1.0 - k32 and r.F[1] == -1.0
    assert r.F[0] == pytest.approx(1.0 - k32 - k32 * k32, rel=2e-16, abs=2e-16)
    r64 = O.fastron_train(cp, np.array([1, -1]), g, iter_max=100, store32=False)
    assert r64.alpha[1] != r.alpha[1]


def test_fp32_stored_kernel_margins_are_k32_alpha():
    # F = K32 alpha throughout, with K32 the FP64 Gram rounded entry by entry
    w, X, y, cp = _small_problem(200, seed=3, name="arm7-n5000")
    K32 = O.gram(cp, cp, w.gamma).astype(np.float32).astype(np.float64)
    r = O.fastron_train(cp, y, w.gamma, iter_max=5000, store32=True)
    assert r.converged and np.all(y * r.F > 0)
    np.testing.assert_allclose(r.F, K32 @ r.alpha, rtol=1e-11, atol=1e-11)
    K = O.gram(cp, cp, w.gamma)
    assert np.max(np.abs(K32 @ r.alpha - K @ r.alpha)) > 0


def test_margins_of_a_carried_model():
    # F = K alpha0 with the first ns points weighted: against the matrix
    # product, and exactly for ns = 1 (F_j = alpha_0 K_0j)
    w, X, y, cp = _small_problem(150, seed=4, name="arm7-n5000")
    alpha = np.linspace(-2.0, 3.0, 40)
    K = O.gram(cp, cp, w.gamma)
    F = O.margins(cp, 40, alpha, w.gamma)
    np.testing.assert_allclose(F, K[:, :40] @ alpha, rtol=1e-12, atol=1e-12)
    F1 = O.margins(cp, 1, alpha[:1], w.gamma)
    assert np.array_equal(F1, alpha[0] * K[:, 0])
    F32 = O.margins(cp, 40, alpha, w.gamma, store32=True)
    np.testing.assert_allclose(F32, K[:, :40].astype(np.float32).astype(np.float64) @ alpha, rtol=1e-12,
                               atol=1e-12)
    # a carried model is a warm start: training resumes from it, and a model
    # carried onto its own training set with its own F changes nothing
    r = O.fastron_train(cp, y, w.gamma, iter_max=5000)
    order = np.concatenate([r.support, np.setdiff1d(np.arange(len(y)), r.support)])
    cpo, yo = cp[order], y[order]
    F0 = O.margins(cpo, len(r.support), r.alpha[r.support], w.gamma)
    np.testing.assert_allclose(F0, r.F[order], rtol=1e-10, atol=1e-10)
    a0 = np.zeros(len(y))
    a0[:len(r.support)] = r.alpha[r.support]
    r2 = O.fastron_train(cpo, yo, w.gamma, iter_max=5000, alpha0=a0, F0=F0)
    assert r2.converged and r2.iters == 0


def test_active_samples_layout_and_bounds():
    w = synth.workload("arm7m12-n65536")
    arm = w.scene.arm
    S = w.train_configs()[:50].astype(np.float64)
    X = O.active_samples(S, 2, 0.1, 300, arm.qlim, seed=77)
    assert X.shape == (50 + 100 + 300, 7)
    assert np.array_equal(X[:50], S)
    assert np.array_equal(X, X.astype(np.float32).astype(np.float64))  # FP32 values
    for c in range(2):
        d = X[50 + 50 * c:100 + 50 * c] - S
        assert np.all(np.abs(d) <= 0.1 + 1e-6) and np.abs(d).max() > 0.05
    assert np.all(np.abs(X) <= arm.qlim)
    U = X[150:]
    assert np.abs(U).max() > 0.9 * arm.qlim and abs(U.mean()) < 0.2
    # the draws are those of the shared generator, in the stated order
    u = synth.Stream(77).uniform(2 * 50 * 7, -0.1, 0.1).reshape(2, 50, 7)
    want = np.clip(S + u[1], -arm.qlim, arm.qlim).astype(np.float32).astype(np.float64)
    assert np.array_equal(X[100:150], want)
    assert np.array_equal(X, O.active_samples(S, 2, 0.1, 300, arm.qlim, seed=77))
