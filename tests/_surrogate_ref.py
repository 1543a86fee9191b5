"""Element-wise reference for the surrogate's GPU tests: the FP64 oracle with
the kernels' bfloat16 storage points (oracle/mlp.py backward_bf16_storage)
and a per-element tolerance of C_TOL units of bfloat16 roundoff times the sum
of the absolute products that form each element.  A test tolerance, not a
proven bound (see tests/test_gpu_surrogate.py)."""
import numpy as np

from oracle import mlp as L

UB = 2.0 ** -9   # bfloat16 unit roundoff (round to nearest)
C_TOL = 8.0      # units of UB per element of the absolute-product sum


def elementwise_reference(pb, X64, target=None):
    """The oracle with the kernels' BF16 storage points, evaluated in FP64 on
    the BF16 weights pb and FP64 features X64 (rounded to BF16 here), and the
    per-element tolerances of the module docstring."""
    X = L.bf16_round(X64)
    z1 = X @ pb["W1"].T + pb["b1"]
    h1 = L.bf16_round(np.maximum(z1, 0.0))
    h2 = L.bf16_round(np.maximum(h1 @ pb["W2"].T + pb["b2"], 0.0))
    z3 = h2 @ pb["W3"].T + pb["b3"]
    h3f = np.maximum(z3, 0.0)  # the output unit reads h3 in FP32
    out = h3f @ pb["w4"] + pb["b4"][0]
    tol_out = C_TOL * UB * (h3f @ np.abs(pb["w4"]) + abs(pb["b4"][0]))
    if target is None:
        return out, tol_out
    g = L.backward_bf16_storage(pb, X, target)
    h3 = L.bf16_round(h3f)
    B = X.shape[0]
    dout = 2.0 * (out - target) / B
    d3 = L.bf16_round(np.outer(dout, pb["w4"]) * (h3 > 0))
    d2 = L.bf16_round((d3 @ pb["W3"]) * (h2 > 0))
    d1 = L.bf16_round((d2 @ pb["W2"]) * (h1 > 0))
    tol = {"w4": h3.T @ np.abs(dout), "b4": np.array([np.abs(dout).sum()]),
           "W3": np.abs(d3).T @ h2, "b3": np.abs(d3).sum(0), "W2": np.abs(d2).T @ h1, "b2": np.abs(d2).sum(0),
           "W1": np.abs(d1).T @ np.abs(X), "b1": np.abs(d1).sum(0)}
    # a floor for elements with no products at all (a unit dead on every row),
    # where a ReLU at its boundary may still let one row through on the GPU
    tol = {k: C_TOL * UB * v for k, v in tol.items()}
    return out, tol_out, g, {k: np.maximum(v, 1e-3 * np.max(v)) for k, v in tol.items()}
