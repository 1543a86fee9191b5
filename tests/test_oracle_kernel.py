"""Pins of the oracle's RQ kernel (Eq. 3), FK kernel (Eq. 4), kernel matrix
(Sec. II-B, Claim 1) and model value f (Sec. III-B)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_06451_gb300 import synth


def test_rq_closed_forms():
    x = np.array([0.1, -0.4, 0.7])
    for g in (0.5, 10.0, 40.0):
        assert O.k_rq(x, x, g) == 1.0
        # |x - x'|^2 = 2/g  ->  (1 + 1)^-2 = 1/4 ;  6/g -> (1 + 3)^-2 = 1/16
        for d2, want in ((2.0 / g, 0.25), (6.0 / g, 1.0 / 16.0)):
            u = np.array([1.0, 2.0, -2.0]) / 3.0  # unit vector
            assert O.k_rq(x, x + math.sqrt(d2) * u, g) == pytest.approx(want, rel=1e-14)


def test_rq_symmetric_monotone_and_bounded():
    rng = np.random.default_rng(0)
    g = 10.0
    for _ in range(50):
        a, b = rng.normal(size=3), rng.normal(size=3)
        k = O.k_rq(a, b, g)
        assert k == O.k_rq(b, a, g)
        assert 0.0 < k <= 1.0
    a = np.zeros(3)
    ks = [O.k_rq(a, np.array([r, 0, 0]), g) for r in np.linspace(0, 3, 40)]
    assert all(x > y for x, y in zip(ks, ks[1:]))


def test_rq_any_dimension():
    # the RBF baseline of the paper applies Eq. 3 to joint vectors
    a = np.arange(7.0)
    b = a + 1.0
    assert O.k_rq(a, b, 2.0) == pytest.approx((1 + 7.0) ** -2, rel=1e-15)


def test_fk_kernel_is_mean_of_summands():
    rng = np.random.default_rng(1)
    g = 10.0
    A = rng.normal(size=(6, 3))
    assert O.k_fk(A, A, g) == 1.0
    B = A.copy()
    B[2] += np.array([0.0, math.sqrt(2.0 / g), 0.0])  # one summand becomes 1/4
    assert O.k_fk(A, B, g) == pytest.approx((5 + 0.25) / 6, rel=1e-15)
    C = rng.normal(size=(6, 3))
    want = np.mean([O.k_rq(A[m], C[m], g) for m in range(6)])
    assert O.k_fk(A, C, g) == pytest.approx(want, rel=1e-15)


def test_gram_symmetric_unit_diagonal_and_positive_definite():
    # Claim 1: distinct random configurations give a PD kernel matrix
    for name in ("arm3-n1000", "arm7-n5000"):
        w = synth.workload(name)
        X = w.train_configs()[:300].astype(np.float64)
        cp = O.fk_points(w.scene.arm, X)
        K = O.gram(cp, cp, w.gamma)
        assert np.array_equal(K, K.T)
        assert np.all(np.diag(K) == 1.0)
        assert np.all(K > 0) and np.all(K <= 1)
        np.linalg.cholesky(K)


def test_gram_rectangular_matches_pairs():
    w = synth.workload("arm3-n1000")
    arm = w.scene.arm
    A = O.fk_points(arm, w.train_configs()[:7].astype(np.float64))
    B = O.fk_points(arm, w.query_configs(5).astype(np.float64))
    K = O.gram(A, B, w.gamma)
    for i in range(7):
        for j in range(5):
            assert K[i, j] == O.k_fk(A[i], B[j], w.gamma)


def test_score_equals_kernel_matrix_times_alpha():
    # f(X_j) = sum_i K(X_i, X_j) alpha_i = (K alpha)_j
    w = synth.workload("arm7-n5000")
    arm = w.scene.arm
    X = w.train_configs()[:120].astype(np.float64)
    cp = O.fk_points(arm, X)
    rng = np.random.default_rng(3)
    alpha = rng.normal(size=120)
    K = O.gram(cp, cp, w.gamma)
    f = O.score_points(cp, alpha, cp, w.gamma)
    np.testing.assert_allclose(f, K @ alpha, rtol=1e-12, atol=1e-12)


def test_score_single_support_point_and_threads():
    w = synth.workload("arm3-n1000")
    arm = w.scene.arm
    Q = w.query_configs(333).astype(np.float64)
    f = O.score(arm, Q[:1], np.array([2.5]), Q[:1], w.gamma)
    assert f[0] == 2.5  # K(x, x) = 1
    S = w.train_configs()[:40].astype(np.float64)
    a = np.random.default_rng(4).normal(size=40)
    f1 = O.score(arm, S, a, Q, w.gamma, nthreads=1)
    f7 = O.score(arm, S, a, Q, w.gamma, nthreads=7)
    assert np.array_equal(f1, f7)
    assert np.array_equal(O.score(arm, S[:0], a[:0], Q, w.gamma), np.zeros(333))


def test_label_sign_rule():
    assert list(O.labels_from_f(np.array([1.0, -1.0, 0.0, -0.0, 1e-300]))) == [1, -1, 1, 1, 1]
