"""Pins of the oracle's Gaussian summand exp(-gamma/2 |x - x'|^2), the
library's non-paper alternative to the RQ kernel of Eq. 3 inside the FK
kernel of Eq. 4, and of the kernel matrix, model value and Algorithm 1 built
on it.  None of these retypes the formula: they check the semigroup property
of the exponential, its Taylor expansion, positive definiteness, the
composition with the RQ kernel as the order goes to infinity, and
Algorithm 1's own invariants."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_06451_gb300 import synth


def test_gauss_unit_diagonal_symmetry_and_bounds():
    rng = np.random.default_rng(0)
    for g in (0.5, 10.0, 40.0):
        for _ in range(20):
            a, b = rng.normal(size=3), rng.normal(size=3)
            assert O.k_gauss(a, a, g) == 1.0
            k = O.k_gauss(a, b, g)
            assert k == O.k_gauss(b, a, g)
            assert 0.0 <= k < 1.0


def test_gauss_semigroup_along_orthogonal_offsets():
    # |u + v|^2 = |u|^2 + |v|^2 for orthogonal u, v, so the summand of the sum
    # is the product of the summands (a property of exp, not of the code)
    rng = np.random.default_rng(1)
    x = rng.normal(size=3)
    for g in (2.0, 10.0, 40.0):
        u = np.array([0.3, 0.0, 0.0])
        v = np.array([0.0, -0.2, 0.1])
        lhs = O.k_gauss(x, x + u + v, g)
        rhs = O.k_gauss(x, x + u, g) * O.k_gauss(x, x + v, g)
        assert lhs == pytest.approx(rhs, rel=1e-14)


def test_gauss_taylor_expansion_near_zero():
    # 1 - k = gamma/2 |d|^2 - (gamma/2 |d|^2)^2 / 2 + O(|d|^6)
    x = np.zeros(3)
    g = 10.0
    for r in (1e-2, 3e-3, 1e-3):
        h = 0.5 * g * r * r
        k = O.k_gauss(x, np.array([0.0, r, 0.0]), g)
        assert (1.0 - k) == pytest.approx(h - h * h / 2, rel=1e-5, abs=1e-17)


def test_rq_family_tends_to_gauss():
    # (1 + gamma d^2 / (2 p))^-p -> exp(-gamma d^2 / 2) as p grows: the RQ
    # kernel of Eq. 3, (1 + gamma'/2 d^2)^-2, at gamma' = gamma / p and raised
    # to p/2 approaches the Gaussian; checked against the oracle's own RQ kernel
    x, y = np.array([0.1, 0.2, -0.3]), np.array([0.4, -0.1, 0.2])
    g = 10.0
    want = O.k_gauss(x, y, g)
    errs = []
    for p in (2, 8, 64, 4096):
        approx = O.k_rq(x, y, g / p) ** (p / 2.0)
        errs.append(abs(approx - want))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * want  # the gap shrinks like (gamma d^2 / 2)^2 / (2 p)
    assert errs[2] / errs[3] > 50


def test_fk_kernel_with_gauss_is_mean_of_summands():
    rng = np.random.default_rng(2)
    g = 40.0
    A = rng.normal(size=(8, 3))
    assert O.k_fk(A, A, g, "gauss") == 1.0
    C = rng.normal(size=(8, 3)) * 0.1 + A
    want = np.mean([O.k_gauss(A[m], C[m], g) for m in range(8)])
    assert O.k_fk(A, C, g, "gauss") == pytest.approx(want, rel=1e-15)
    # the default summand stays the paper's RQ kernel
    assert O.k_fk(A, C, g) == O.k_fk(A, C, g, "rq") != O.k_fk(A, C, g, "gauss")


def test_gauss_gram_positive_definite_and_score_is_gram_times_alpha():
    w = synth.workload("arm7-n5000")
    X = w.train_configs()[:200].astype(np.float64)
    cp = O.fk_points(w.scene.arm, X)
    K = O.gram(cp, cp, w.gamma, "gauss")
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    np.linalg.cholesky(K)
    alpha = np.random.default_rng(3).normal(size=200)
    f = O.score_points(cp, alpha, cp, w.gamma, summand="gauss")
    np.testing.assert_allclose(f, K @ alpha, rtol=1e-12, atol=1e-12)


def test_fastron_with_gauss_invariants():
    # Algorithm 1 on the Gaussian FK kernel: after convergence F = K alpha and
    # every training margin is positive; N = 1 gives alpha = b y
    w = synth.workload("arm3-n1000")
    X = w.train_configs()[:300].astype(np.float64)
    y = O.check(w.scene, X)
    cp = O.fk_points(w.scene.arm, X)
    r = O.fastron_train(cp, y, w.gamma, 1.5, 5000, summand="gauss")
    assert r.converged
    K = O.gram(cp, cp, w.gamma, "gauss")
    np.testing.assert_allclose(r.F, K @ r.alpha, rtol=1e-10, atol=1e-10)
    assert np.all(y * r.F > 0)
    # a different kernel gives a different model on the same data
    rq = O.fastron_train(cp, y, w.gamma, 1.5, 5000)
    assert not np.array_equal(rq.alpha, r.alpha)
    one = O.fastron_train(cp[:1], np.array([1], dtype=np.int8), w.gamma, 1.5, 10, summand="gauss")
    assert one.alpha[0] == 1.5


def test_gauss_score_threads_and_empty_support():
    w = synth.workload("arm3-n1000")
    arm = w.scene.arm
    Q = w.query_configs(200).astype(np.float64)
    S = w.train_configs()[:30].astype(np.float64)
    a = np.random.default_rng(4).normal(size=30)
    f1 = O.score(arm, S, a, Q, w.gamma, nthreads=1, summand="gauss")
    f5 = O.score(arm, S, a, Q, w.gamma, nthreads=5, summand="gauss")
    assert np.array_equal(f1, f5)
    assert np.array_equal(O.score(arm, S[:0], a[:0], Q, w.gamma, summand="gauss"), np.zeros(200))
    assert math.isclose(O.score(arm, S[:1], np.array([2.0]), S[:1], w.gamma, summand="gauss")[0], 2.0)
