"""The element-wise tolerances of the surrogate's GPU tests can see a
mistake: on the oracle's own values, planted mistakes of the kinds a kernel
could make (a sign, a transposed operand, a dropped ReLU mask, a row or
column off by one) move most elements of the gradient they touch beyond
their tolerance, while the FP32-accumulation-order differences the GPU is
allowed stay far inside it."""
import numpy as np
import pytest

from oracle import mlp as L
from paper_1910_06451_gb300 import synth
from tests._surrogate_ref import elementwise_reference


@pytest.fixture(scope="module")
def ref():
    w = synth.workload("arm7-n5000")
    rng = np.random.default_rng(4)
    p = L.init_params(rng)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(size=p[k].shape) * 0.05
    for k in ("W1", "W2", "W3"):
        p[k] = L.bf16_round(p[k])
    p["w4"] = p["w4"].astype(np.float32).astype(np.float64)
    q = w.query_configs(512).astype(np.float64)
    X64 = L.features(w.scene.arm, q)
    t = np.random.default_rng(5).normal(size=512)
    return p, X64, t, elementwise_reference(p, X64, t)


def _frac_caught(bad, good, tol):
    big = np.abs(good) > 0.1 * np.max(np.abs(good))
    return float(np.mean(np.abs(bad - good)[big] > tol[big]))


def _stored(p, X64, out, t):
    X = L.bf16_round(X64)
    h1 = L.bf16_round(np.maximum(X @ p["W1"].T + p["b1"], 0.0))
    h2 = L.bf16_round(np.maximum(h1 @ p["W2"].T + p["b2"], 0.0))
    h3 = L.bf16_round(np.maximum(h2 @ p["W3"].T + p["b3"], 0.0))
    d3 = L.bf16_round(np.outer(2.0 * (out - t) / len(t), p["w4"]) * (h3 > 0))
    return X, h1, h2, h3, d3


def test_accumulation_order_stays_inside(ref):
    # the W3 gradient's sums in FP32, rows in reverse order: far inside
    p, X64, t, (out, tol_out, g, tol) = ref
    X, h1, h2, h3, d3 = _stored(p, X64, out, t)
    g32 = (d3[::-1].astype(np.float32).T @ h2[::-1].astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(g32 - g["W3"]) <= 0.1 * tol["W3"])


@pytest.mark.parametrize("k", ["W1", "W2", "W3", "w4", "b1", "b2", "b3"])
def test_sign_error_is_caught(ref, k):
    p, X64, t, (out, tol_out, g, tol) = ref
    assert _frac_caught(-g[k], g[k], tol[k]) == 1.0


@pytest.mark.parametrize("k", ["W2", "W3"])
def test_transposed_gradient_is_caught(ref, k):
    p, X64, t, (out, tol_out, g, tol) = ref
    assert _frac_caught(g[k].T, g[k], tol[k]) > 0.9


def test_dropped_relu_mask_is_caught(ref):
    # the layer-2 delta without its ReLU mask changes the W2 gradient
    p, X64, t, (out, tol_out, g, tol) = ref
    X, h1, h2, h3, d3 = _stored(p, X64, out, t)
    d2_nomask = L.bf16_round(d3 @ p["W3"])
    assert _frac_caught(d2_nomask.T @ h1, g["W2"], tol["W2"]) > 0.5


def test_off_by_one_row_is_caught(ref):
    p, X64, t, (out, tol_out, g, tol) = ref
    assert _frac_caught(np.roll(g["W1"], 1, axis=0), g["W1"], tol["W1"]) > 0.9
    assert _frac_caught(np.roll(g["W3"], 1, axis=1), g["W3"], tol["W3"]) > 0.9
