"""Pins of the FP64 surrogate oracle: finite differences of the loss, the
closed-form first Adam step, and feature values at known configurations."""
import math

import numpy as np
import pytest

from oracle import mlp as L
from oracle import oracle as O
from paper_1910_06451_gb300 import synth


def _small(rng, n_in=5, width=6):
    p = L.init_params(rng, n_in, width)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(size=p[k].shape) * 0.3
    return p


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _small(rng)
    X = rng.normal(size=(9, 5))
    y = rng.normal(size=9)
    out, cache = L.forward(p, X)
    g = L.backward(p, cache, out, y)
    h = 1e-6
    for k, v in p.items():
        num = np.zeros_like(v)
        for idx in np.ndindex(v.shape):
            old = v[idx]
            v[idx] = old + h
            lp = L.loss(L.forward(p, X)[0], y)
            v[idx] = old - h
            lm = L.loss(L.forward(p, X)[0], y)
            v[idx] = old
            num[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[k], num, rtol=1e-5, atol=1e-8, err_msg=k)


def test_forward_is_the_composition():
    rng = np.random.default_rng(1)
    p = _small(rng)
    x = rng.normal(size=5)
    h = x
    for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        h = np.array([max(0.0, float(np.dot(p[W][o], h) + p[b][o])) for o in range(p[W].shape[0])])
    want = float(np.dot(p["w4"], h) + p["b4"][0])
    assert L.forward(p, x[None])[0][0] == pytest.approx(want, rel=1e-14)


def test_first_adam_step_closed_form():
    # with zero moments the bias-corrected first step is -lr g / (|g| + eps)
    rng = np.random.default_rng(2)
    p = _small(rng)
    g = {k: rng.normal(size=v.shape) for k, v in p.items()}
    before = {k: v.copy() for k, v in p.items()}
    st = {}
    L.adam_step(p, g, st, lr=1e-2, eps=1e-8)
    for k in p:
        np.testing.assert_allclose(p[k] - before[k], -1e-2 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12)


def test_features_at_known_configurations():
    arm = synth.arm_7dof(1001)
    q = np.zeros((1, 7))
    q[0, 2] = math.pi / 2
    f = L.features(arm, q)
    assert f.shape == (1, 64) and np.all(f[0, 56:] == 0)
    cp = O.fk_points(arm, q)[0]
    for m in range(8):
        np.testing.assert_array_equal(f[0, 7 * m:7 * m + 3], cp[m])
        qm = 0.0 if m == 0 else q[0, m - 1]
        qn = 0.0 if m == 7 else q[0, m]
        np.testing.assert_allclose(f[0, 7 * m + 3:7 * m + 7], [math.sin(qm), math.cos(qm), math.sin(qn), math.cos(qn)],
                                   atol=1e-16)
    # control point 0 is the base: constant
    assert np.all(f[0, :3] == 0)


def test_bf16_rounding():
    # representable values stay; halfway cases go to the even neighbour
    assert L.bf16_round(1.0) == 1.0 and L.bf16_round(-3.5) == -3.5
    one_ulp = 2.0 ** -7  # bf16 spacing just above 1
    assert L.bf16_round(1.0 + one_ulp / 2) == 1.0               # tie -> even (1.0)
    assert L.bf16_round(1.0 + 1.5 * one_ulp) == 1.0 + 2 * one_ulp  # tie -> even
    assert L.bf16_round(1.0 + 0.6 * one_ulp) == 1.0 + one_ulp
    assert L.bf16_round(np.float32(3.0e38)) == pytest.approx(3.0e38, rel=1e-2)


def test_bf16_storage_gradients(monkeypatch):
    rng = np.random.default_rng(8)
    p = L.init_params(rng, 8, 16)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(size=p[k].shape) * 0.1
    X = rng.normal(size=(40, 8))
    y = rng.normal(size=40)
    out, cache = L.forward(p, X)
    g = L.backward(p, cache, out, y)
    g_bf = L.backward_bf16_storage(p, X, y)
    # the storage rounding perturbs the gradients at the bfloat16 level ...
    for k in g:
        rel = np.linalg.norm(g_bf[k] - g[k]) / np.linalg.norm(g[k])
        assert rel < 5e-2, k
    assert any(np.linalg.norm(g_bf[k] - g[k]) > 0 for k in ("W1", "W2", "W3"))
    # ... and without it the storage variant is exactly the FP64 back-propagation
    monkeypatch.setattr(L, "bf16_round", lambda x: np.asarray(x, dtype=np.float64))
    g_id = L.backward_bf16_storage(p, X, y)
    for k in g:
        np.testing.assert_allclose(g_id[k], g[k], rtol=1e-13, atol=1e-15)


def test_features_of_the_twelve_point_arm_use_the_frame_origins():
    # the four link midpoints are averages of frame origins: the features
    # are those of the eight frame-origin points, as for the 8-point arm
    a12 = synth.arm_7dof_m12(4000)
    a8 = synth.arm_7dof(4000)
    q = synth.uniform_configs(3, 20, 7, a8.qlim).astype(np.float64)
    np.testing.assert_array_equal(L.features(a12, q), L.features(a8, q))
