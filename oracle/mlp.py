"""FP64 oracle of the learned surrogate: features, MLP forward and backward,
mean-squared-error loss and Adam.

TEST INFRASTRUCTURE ONLY (test suite, smoke check, benchmark CPU leg).  The
paper has no learned surrogate; this restates the plain definitions the GPU
kernels follow, in numpy FP64 with library matmuls as steps:

  features  per control point m < min(M, D + 1) (on frame j): its position
            (x, y, z) from the FK of Eqs. 1-2, then sin/cos of joint values
            q_j and q_{j+1} (q_0 = q_{D+1} = 0): for the 7-DOF chain
            8 x 7 = 56 values, padded with zeros to 64; further points (link
            midpoints, averages of two frame origins) are left out;
  network   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2),
            h3 = relu(h2 W3^T + b3), out = h3 w4 + b4;
  loss      mean over the batch of (out - target)^2;
  Adam      Kingma and Ba (ICLR 2015), bias-corrected moments.

Parity status: pinned by tests/test_oracle_mlp.py (central finite
differences of the loss, the closed-form first Adam step, feature values at
known configurations, bfloat16 rounding of exactly representable and halfway
values, and the BF16-storage gradients reducing to the FP64 ones when every
stored value is representable).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

N_FEAT = 56
N_IN = 64


def features(arm, q) -> np.ndarray:
    """(n, 64) feature rows for configurations q (n, D)."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, arm.D)
    n = q.shape[0]
    cp = O.fk_points(arm, q)
    qq = np.concatenate([np.zeros((n, 1)), q, np.zeros((n, 1))], axis=1)  # q_0 .. q_{D+1}
    out = np.zeros((n, N_IN))
    col = 0
    for m in range(min(arm.M, arm.D + 1)):
        j = int(arm.cp_joint[m])
        out[:, col:col + 3] = cp[:, m]
        out[:, col + 3] = np.sin(qq[:, j])
        out[:, col + 4] = np.cos(qq[:, j])
        out[:, col + 5] = np.sin(qq[:, j + 1])
        out[:, col + 6] = np.cos(qq[:, j + 1])
        col += 7
    return out


def init_params(rng: np.random.Generator, n_in=N_IN, width=256) -> dict:
    """He-uniform weights, zero biases."""
    def he(o, i):
        lim = np.sqrt(6.0 / i)
        return rng.uniform(-lim, lim, (o, i))
    return {"W1": he(width, n_in), "b1": np.zeros(width), "W2": he(width, width), "b2": np.zeros(width),
            "W3": he(width, width), "b3": np.zeros(width), "w4": he(1, width)[0] * 0.5, "b4": np.zeros(1)}


def forward(p: dict, X: np.ndarray):
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    out = h3 @ p["w4"] + p["b4"][0]
    return out, (X, h1, h2, h3)


def loss(out: np.ndarray, target: np.ndarray) -> float:
    return float(np.mean((out - target) ** 2))


def backward(p: dict, cache, out: np.ndarray, target: np.ndarray) -> dict:
    """Gradients of the mean-squared-error loss with respect to every parameter."""
    X, h1, h2, h3 = cache
    B = X.shape[0]
    dout = 2.0 * (out - target) / B
    g = {"w4": h3.T @ dout, "b4": np.array([dout.sum()])}
    d3 = np.outer(dout, p["w4"]) * (h3 > 0)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(0)
    d2 = (d3 @ p["W3"]) * (h2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"]) * (h1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return g


def bf16_round(x) -> np.ndarray:
    """Round to bfloat16 (8 exponent bits, 7 fraction bits), ties to even,
    returned as FP64: x is first rounded to FP32, then the low 16 bits of the
    FP32 pattern are rounded away."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def backward_bf16_storage(p: dict, X: np.ndarray, target: np.ndarray) -> dict:
    """The same gradients when the hidden activations h1, h2, h3 and the
    back-propagated deltas are stored in bfloat16 between layers (the
    arithmetic itself in FP64): the precision contract of the tensor-core
    path, which keeps activations and deltas in BF16 and accumulates in FP32."""
    z1 = X @ p["W1"].T + p["b1"]
    h1 = bf16_round(np.maximum(z1, 0.0))
    h2 = bf16_round(np.maximum(h1 @ p["W2"].T + p["b2"], 0.0))
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = bf16_round(np.maximum(z3, 0.0))
    out = np.maximum(z3, 0.0) @ p["w4"] + p["b4"][0]
    B = X.shape[0]
    dout = 2.0 * (out - target) / B
    g = {"w4": h3.T @ dout, "b4": np.array([dout.sum()])}
    d3 = bf16_round(np.outer(dout, p["w4"]) * (h3 > 0))
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(0)
    d2 = bf16_round((d3 @ p["W3"]) * (h2 > 0))
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = bf16_round((d2 @ p["W2"]) * (h1 > 0))
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """One Adam update in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m *= beta1
        m += (1 - beta1) * g[k]
        v *= beta2
        v += (1 - beta2) * g[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
