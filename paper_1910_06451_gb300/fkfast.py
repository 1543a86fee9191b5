"""ctypes binding of libfkfast.so (include/fkfast.h).

Argument marshalling only: every function here checks tensor placement,
dtype and shape, converts to raw pointers and calls the C function of the
same name, which runs the work in the library's CUDA kernels.  There is no
CPU path: if the library is not built or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FK_OK = 0
FK_ERR_ARG = -1
FK_ERR_CUDA = -2
FK_ERR_CAPACITY = -3
FK_ERR_TIMEOUT = -4
FK_ERR_STATE = -5
FK_F32 = 0
FK_F64 = 1
FK_F16 = 2
FK_DF64 = 3
FK_DF32 = 4
FK_LR_STEP = 0
FK_LR_COSINE = 1
FK_SUMMAND_RQ = 0      # the paper's summand (Eq. 3)
FK_SUMMAND_GAUSS = 1   # not in the paper: exp(-gamma/2 |d|^2)
FK_MAX_DOF = 16
FK_MAX_CP = 32

EXPORTS = (
    "fk_last_error", "fk_chain_create", "fk_chain_destroy", "fk_forward", "fk_forward_f64", "fk_gram",
    "fastron_model_create", "fastron_model_destroy", "fastron_train", "fastron_model_trace",
    "fastron_model_set", "fastron_model_copy", "fastron_model_get", "fk_score", "fk_score_noalloc", "fk_score_band", "fk_score_circle", "fk_set_circle_form", "fk_check_rcp", "fk_check_sincos", "fk_forward_dd", "fk_label", "fk_set_wait_limit",
    "fk_probe_pipe", "fk_tc_gemm_bf16", "surrogate_create", "surrogate_destroy", "surrogate_train", "surrogate_infer",
    "surrogate_forward", "surrogate_set_params", "surrogate_get_params", "surrogate_gradients", "surrogate_adam_step",
    "fk_batch_create", "fk_batch_destroy", "fk_score_batched", "fk_batch_tune", "fk_active_samples",
    "fk_chain_set_summand", "fk_set_gauss_poly",
)


class FkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fkfast error {code}: {msg}")
        self.code = code


class FkDh(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("alpha", ctypes.c_double), ("d", ctypes.c_double),
                ("theta0", ctypes.c_double), ("type", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class FkCp(ctypes.Structure):
    _fields_ = [("joint", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t", ctypes.c_double * 3)]


class FastronParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("beta", ctypes.c_double), ("iter_max", ctypes.c_int64),
                ("s_max", ctypes.c_int64), ("warm_start", ctypes.c_int32), ("trace", ctypes.c_int32),
                ("gram", ctypes.c_int32), ("reuse_gram", ctypes.c_int32)]


class SurrogateTrainParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("holdout", ctypes.c_float), ("reinit", ctypes.c_int32), ("schedule", ctypes.c_int32)]


class SurrogateStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("n_train", ctypes.c_int64), ("n_holdout", ctypes.c_int64),
                ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float), ("scale", ctypes.c_float),
                ("tau", ctypes.c_float), ("holdout_sign_error", ctypes.c_float), ("holdout_fallback", ctypes.c_float)]


SURROGATE_PARAMS = 148481


class FastronStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("adds", ctypes.c_int64), ("removes", ctypes.c_int64),
                ("n_support", ctypes.c_int64), ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libfkfast.so; raises if it is missing (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise FkError(FK_ERR_STATE, f"{path} is not built; run python -m paper_1910_06451_gb300.build")
            _build.build()
        lib = ctypes.CDLL(path)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "fk_last_error": ([], ctypes.c_char_p),
            "fk_chain_create": ([P, I, P, P, I, PP], I),
            "fk_chain_destroy": ([P], None),
            "fk_forward": ([P, P, I64, P, P], I),
            "fk_forward_f64": ([P, P, I64, P, P], I),
            "fk_gram": ([P, P, I64, P, I64, D, I, P, P], I),
            "fastron_model_create": ([P, PP], I),
            "fastron_model_destroy": ([P], None),
            "fastron_train": ([P, P, P, I64, P, P, P], I),
            "fastron_model_trace": ([P, P, P, P, I64, P], I),
            "fastron_model_set": ([P, P, P, I64, D], I),
            "fastron_model_get": ([P, P, P, I64, P], I),
            "fastron_model_copy": ([P, P, P], I),
            "fk_score": ([P, P, I64, I, I, D, P, P, P, P], I),
            "fk_score_noalloc": ([P, P, I64, D, P, P, P, P], I),
            "fk_score_band": ([P, I, P, P], I),
            "fk_score_circle": ([P, P], I),
            "fk_set_circle_form": ([I], I),
            "fk_check_rcp": ([I, I, P], I),
            "fk_check_sincos": ([ctypes.c_float, D, P], I),
            "fk_forward_dd": ([P, P, I64, D, P, P], I),
            "fk_label": ([P, P, I64, D, P, I64, P, P], I),
            "fk_active_samples": ([P, ctypes.c_int32, D, I64, D, ctypes.c_uint64, P, P, I64, P, P], I),
            "fk_set_wait_limit": ([ctypes.c_uint32], None),
            "fk_chain_set_summand": ([P, I], I),
            "fk_set_gauss_poly": ([I], I),
            "fk_probe_pipe": ([I, P, P], I),
            "fk_tc_gemm_bf16": ([P, I64, P, I64, I, I, I, I, P, P], I),
            "fk_batch_create": ([P, I, PP], I),
            "fk_batch_destroy": ([P], None),
            "fk_score_batched": ([P, P, P, I, P, P, P, P], I),
            "fk_batch_tune": ([P, P, P, P, P, I, P], I),
            "surrogate_create": ([P, ctypes.c_uint64, PP], I),
            "surrogate_destroy": ([P], None),
            "surrogate_train": ([P, P, P, I64, P, P, P], I),
            "surrogate_infer": ([P, P, P, I64, D, P, P, P, P], I),
            "surrogate_forward": ([P, P, I64, P, P], I),
            "surrogate_set_params": ([P, P, I64], I),
            "surrogate_get_params": ([P, P, I64, P, P], I),
            "surrogate_gradients": ([P, P, I64, P, P, P], I),
            "surrogate_adam_step": ([P, P, ctypes.c_float], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int):
    if rc != FK_OK:
        raise FkError(rc, load().fk_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- chain ---

def fk_chain_create(dh, base, cp_joint, cp_off):
    """dh: (D, 5) rows (a, alpha, d, theta0, type); base: (4, 4) or None;
    cp_joint: (M,) frames; cp_off: (M, 3) offsets.  Returns a chain handle."""
    dh = np.asarray(dh, dtype=np.float64)
    D = dh.shape[0]
    links = (FkDh * D)(*[FkDh(r[0], r[1], r[2], r[3], int(r[4]), 0) for r in dh])
    cj = np.asarray(cp_joint)
    co = np.asarray(cp_off, dtype=np.float64).reshape(-1, 3)
    M = cj.shape[0]
    cps = (FkCp * M)(*[FkCp(int(cj[m]), 0, (ctypes.c_double * 3)(*co[m])) for m in range(M)])
    bp = None
    if base is not None:
        bk, bp = _host(np.asarray(base, dtype=np.float64).reshape(16), np.float64)
    out = ctypes.c_void_p()
    _check(load().fk_chain_create(ctypes.cast(links, ctypes.c_void_p), D, bp, ctypes.cast(cps, ctypes.c_void_p), M,
                                  ctypes.byref(out)))
    return out


def chain_from_arm(arm):
    return fk_chain_create(arm.dh, arm.base, arm.cp_joint, arm.cp_off)


def fk_chain_destroy(chain):
    load().fk_chain_destroy(chain)


def fk_chain_set_summand(chain, summand: int):
    """FK_SUMMAND_RQ (the paper's kernel) or FK_SUMMAND_GAUSS (not the paper's)."""
    _check(load().fk_chain_set_summand(chain, int(summand)))


def fk_set_gauss_poly(points: int):
    """Gaussian summand on 7 points: how many points per support point use the
    FMA polynomial instead of MUFU ex2 (0, 1 or 2)."""
    _check(load().fk_set_gauss_poly(int(points)))


# ------------------------------------------------------------ kinematics --

def fk_forward(chain, q, cp, stream=None):
    """q: float32 (n, D) -> cp: float32 (M, 3, n)."""
    import torch
    n = q.shape[0]
    _check(load().fk_forward(chain, _dev(q, torch.float32, "q"), n, _dev(cp, torch.float32, "cp"), _stream(stream)))


def fk_forward_f64(chain, q, cp, stream=None):
    """q: float64 (n, D) -> cp: float64 (M, 3, n)."""
    import torch
    n = q.shape[0]
    _check(load().fk_forward_f64(chain, _dev(q, torch.float64, "q"), n, _dev(cp, torch.float64, "cp"),
                                 _stream(stream)))


def fk_gram(chain, Xa, Xb, gamma, K, stream=None, double_float=False):
    """K[i][j] = K_FK(Xa_i, Xb_j); float64 inputs -> FP64 (double-float
    arithmetic with double_float=True; a float32 K then receives each entry
    rounded to FP32), float32 -> FP32."""
    import torch
    dt = Xa.dtype
    kt = dt
    if dt == torch.float64 and double_float and K.dtype == torch.float32:
        prec, kt = FK_DF32, torch.float32
    else:
        prec = (FK_DF64 if double_float else FK_F64) if dt == torch.float64 else FK_F32
    pa = _dev(Xa, dt, "Xa")
    pb = pa if Xb is Xa else _dev(Xb, dt, "Xb")
    _check(load().fk_gram(chain, pa, Xa.shape[0], pb, Xb.shape[0], float(gamma), prec,
                          _dev(K, kt, "K", (Xa.shape[0], Xb.shape[0])), _stream(stream)))


# ---------------------------------------------------------------- model ---

def fastron_model_create(chain):
    out = ctypes.c_void_p()
    _check(load().fastron_model_create(chain, ctypes.byref(out)))
    return out


def fastron_model_destroy(model):
    load().fastron_model_destroy(model)


def fastron_train(model, X, y, gamma, beta=1.0, iter_max=5000, s_max=None, warm_start=False, trace=False,
                  gram=0, reuse_gram=False, stream=None) -> dict:
    """Algorithm 1 on device training data X (float64, (N, D)) and y (int8, (N,)).
    warm_start: False/0, True/1 (same training set), or 2 (the first |S|
    rows are the model's support points, carried with their weights).
    gram: 0 lets the library choose (FK_DF64 for the RQ summand, FK_F64 for
    the Gaussian one)."""
    import torch
    N = X.shape[0]
    p = FastronParams(float(gamma), float(beta), int(iter_max), int(N if s_max is None else s_max),
                      int(warm_start), int(bool(trace)), int(gram), int(bool(reuse_gram)))
    st = FastronStats()
    _check(load().fastron_train(model, _dev(X, torch.float64, "X"), _dev(y, torch.int8, "y", (N,)), N,
                                ctypes.byref(p), ctypes.byref(st), _stream(stream)))
    return {"iterations": st.iterations, "adds": st.adds, "removes": st.removes, "n_support": st.n_support,
            "converged": bool(st.converged)}


def fk_active_samples(model, k_near, sigma, n_uniform, qlim, seed, X, X32=None, stream=None) -> int:
    """Two-stage active-learning training set from the model's support set
    into device X (float64, (cap, D)) and optionally X32 (float32, same
    shape); returns the number of rows written."""
    import torch
    cap = X.shape[0]
    n = ctypes.c_int64()
    _check(load().fk_active_samples(model, int(k_near), float(sigma), int(n_uniform), float(qlim),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, _dev(X, torch.float64, "X"),
                                    None if X32 is None else _dev(X32, torch.float32, "X32", tuple(X.shape)), cap,
                                    ctypes.byref(n), _stream(stream)))
    return n.value


def fastron_model_trace(model, cap: int):
    kind = np.zeros(cap, dtype=np.int8)
    idx = np.zeros(cap, dtype=np.int64)
    delta = np.zeros(cap, dtype=np.float64)
    n = ctypes.c_int64()
    _check(load().fastron_model_trace(model, kind.ctypes.data_as(ctypes.c_void_p), idx.ctypes.data_as(ctypes.c_void_p),
                                      delta.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n)))
    k = min(n.value, cap)
    return kind[:k], idx[:k], delta[:k]


def fastron_model_set(model, q, alpha, gamma):
    qa, qp = _host(q, np.float64)
    aa, ap = _host(alpha, np.float64)
    _check(load().fastron_model_set(model, qp, ap, aa.shape[0], float(gamma)))


def fastron_model_copy(dst, src, stream=None):
    """Copies src's packed support set into dst (same chain) on `stream`."""
    _check(load().fastron_model_copy(dst, src, _stream(stream)))


def fastron_model_get(model):
    ns = ctypes.c_int64()
    _check(load().fastron_model_get(model, None, None, 0, ctypes.byref(ns)))
    idx = np.zeros(ns.value, dtype=np.int64)
    alpha = np.zeros(ns.value, dtype=np.float64)
    _check(load().fastron_model_get(model, idx.ctypes.data_as(ctypes.c_void_p), alpha.ctypes.data_as(ctypes.c_void_p),
                                    ns.value, ctypes.byref(ns)))
    return idx, alpha


# ---------------------------------------------------------------- score ---

def fk_score(model, q, label, f=None, rescore=True, eps=0.0, count=False, stream=None, precision=FK_F32):
    """Labels (and optionally f) of float32 queries q (n, D).  With count=True
    the call synchronises and returns the number of re-evaluated queries."""
    import torch
    n = q.shape[0]
    nr = ctypes.c_int64()
    _check(load().fk_score(model, _dev(q, torch.float32, "q"), n, int(precision), int(bool(rescore)), float(eps),
                           None if f is None else _dev(f, torch.float32, "f", (n,)),
                           _dev(label, torch.int8, "label", (n,)), ctypes.byref(nr) if count else None,
                           _stream(stream)))
    return nr.value if count else None


def fk_score_noalloc(model, q, label, f=None, eps=0.0, count=False, stream=None):
    """fk_score with FP64 re-scoring for callers that cannot allocate device
    memory: its scratch is a fixed static device array (at most 1,048,576
    queries per call).  Calls that overlap on the GPU share that array and
    race; the first call on a device must come before any stream capture."""
    import torch
    n = q.shape[0]
    nr = ctypes.c_int64()
    _check(load().fk_score_noalloc(model, _dev(q, torch.float32, "q"), n, float(eps),
                                   None if f is None else _dev(f, torch.float32, "f", (n,)),
                                   _dev(label, torch.int8, "label", (n,)), ctypes.byref(nr) if count else None,
                                   _stream(stream)))
    return nr.value if count else None


def fk_score_band(model, precision=None):
    """(eps0, eps1) of the score kernel's default band: a query is re-scored
    when |f| <= (eps0 + eps1 (|p(q)| + |s|max)) B(q), norms of control points
    scaled by sqrt(gamma/2); the bound of the kernel's whole error."""
    e0, e1 = ctypes.c_double(), ctypes.c_double()
    _check(load().fk_score_band(model, FK_F32 if precision is None else int(precision), ctypes.byref(e0),
                                ctypes.byref(e1)))
    return e0.value, e1.value


def fk_score_circle(model) -> float:
    """cnorm of the FP32 band's circle term (0: every point in the direct form):
    eps(q) = eps0 + eps1 max(|p(q)| + |s|max, cnorm)."""
    c = ctypes.c_double()
    _check(load().fk_score_circle(model, ctypes.byref(c)))
    return c.value


def fk_set_circle_form(on: bool):
    """Circle form of the first control point in the FP32 score on (default) or off."""
    _check(load().fk_set_circle_form(1 if on else 0))


def fk_check_rcp(e_lo: int, e_hi: int) -> float:
    """Max |rcp(x) x - 1| of the score kernel's MUFU reciprocal over every FP32
    mantissa of the binades [2^e_lo, 2^(e_hi+1))."""
    out = ctypes.c_double()
    _check(load().fk_check_rcp(int(e_lo), int(e_hi), ctypes.byref(out)))
    return out.value


def fk_check_sincos(hi: float, theta0: float = 0.0) -> float:
    """Max absolute error of the kernels' pair-arithmetic sine and cosine of
    x + theta0 against FP64, over every FP32 x in [-hi, hi]."""
    out = ctypes.c_double()
    _check(load().fk_check_sincos(float(hi), float(theta0), ctypes.byref(out)))
    return out.value


def fk_forward_dd(chain, q, scale, cp, stream=None):
    """Control points (Mv, 3, n) as the score kernels form them: pair-arithmetic
    kinematics times scale, rounded once to FP32."""
    import torch
    n = q.shape[0]
    _check(load().fk_forward_dd(chain, _dev(q, torch.float32, "q"), n, float(scale),
                                _dev(cp, torch.float32, "cp", (cp.shape[0], 3, n)), _stream(stream)))


def fk_label(chain, boxes, radius, q, y, stream=None):
    """Geometric labels (FP64) of float32 configurations q into int8 y."""
    import torch
    bx, bp = _host(np.asarray(boxes, dtype=np.float64).reshape(-1, 6), np.float64)
    n = q.shape[0]
    _check(load().fk_label(chain, bp, bx.shape[0], float(radius), _dev(q, torch.float32, "q"), n,
                           _dev(y, torch.int8, "y", (n,)), _stream(stream)))


def fk_set_wait_limit(polls: int):
    load().fk_set_wait_limit(int(polls))


def fk_tc_gemm_bf16(A, B, splits=1, stream=None):
    """D = A B^T on the tensor cores: A (M, K) and B (N, K) bfloat16 CUDA
    tensors (row stride may exceed K); returns float32 partials (splits, M, N)
    whose sum over the first axis is D."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or not A.is_cuda or not B.is_cuda:
        raise ValueError("A and B must be bfloat16 CUDA tensors")
    if A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("A and B rows must be contiguous")
    C = torch.empty((splits, M, N), dtype=torch.float32, device=A.device)
    _check(load().fk_tc_gemm_bf16(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                                  B.stride(0), M, N, K, splits, ctypes.c_void_p(C.data_ptr()), _stream(stream)))
    return C


def fk_probe_pipe(kind: int):
    ops = ctypes.c_double()
    sec = ctypes.c_double()
    _check(load().fk_probe_pipe(int(kind), ctypes.byref(ops), ctypes.byref(sec)))
    return ops.value, sec.value


# ------------------------------------------------------------ surrogate ---

def surrogate_create(chain, seed=0):
    out = ctypes.c_void_p()
    _check(load().surrogate_create(chain, int(seed), ctypes.byref(out)))
    return out


def surrogate_destroy(s):
    load().surrogate_destroy(s)


def surrogate_train(s, model, q, epochs=10, batch=8192, lr=1e-3, holdout=0.1, reinit=True, schedule=None,
                    stream=None) -> dict:
    """Trains the surrogate on float32 queries q (n, D); targets are the model's FP32 scores.
    schedule: FK_LR_STEP (default) or FK_LR_COSINE."""
    import torch
    p = SurrogateTrainParams(int(epochs), int(batch), float(lr), float(holdout), int(bool(reinit)),
                             FK_LR_STEP if schedule is None else int(schedule))
    st = SurrogateStats()
    _check(load().surrogate_train(s, model, _dev(q, torch.float32, "q"), q.shape[0], ctypes.byref(p),
                                  ctypes.byref(st), _stream(stream)))
    return {k: getattr(st, k) for k, _ in SurrogateStats._fields_}


def surrogate_infer(s, model, q, label, pred=None, tau=0.0, stream=None) -> int:
    """Labels of float32 queries q (n, D); returns the number of fallback queries."""
    import torch
    n = q.shape[0]
    nf = ctypes.c_int64()
    _check(load().surrogate_infer(s, model, _dev(q, torch.float32, "q"), n, float(tau), _dev(label, torch.int8, "label", (n,)),
                                  None if pred is None else _dev(pred, torch.float32, "pred", (n,)), ctypes.byref(nf),
                                  _stream(stream)))
    return nf.value


def surrogate_forward(s, q, out, stream=None):
    import torch
    n = q.shape[0]
    _check(load().surrogate_forward(s, _dev(q, torch.float32, "q"), n, _dev(out, torch.float32, "out", (n,)),
                                    _stream(stream)))


def surrogate_set_params(s, params):
    a, ap = _host(params, np.float32)
    _check(load().surrogate_set_params(s, ap, a.shape[0]))


def surrogate_get_params(s):
    a = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
    sc, tau = ctypes.c_float(), ctypes.c_float()
    _check(load().surrogate_get_params(s, a.ctypes.data_as(ctypes.c_void_p), a.shape[0], ctypes.byref(sc),
                                       ctypes.byref(tau)))
    return a, sc.value, tau.value


def surrogate_gradients(s, q, target):
    import torch
    n = q.shape[0]
    g = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(load().surrogate_gradients(s, _dev(q, torch.float32, "q"), n, _dev(target, torch.float32, "target", (n,)),
                                      g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)))
    return g, loss.value


def surrogate_adam_step(s, grad, lr):
    a, ap = _host(grad, np.float32)
    _check(load().surrogate_adam_step(s, ap, float(lr)))


# ------------------------------------------------------- batched scenes ---

def fk_batch_create(models):
    arr = (ctypes.c_void_p * len(models))(*[m.value for m in models])
    out = ctypes.c_void_p()
    _check(load().fk_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(models), ctypes.byref(out)))
    return out


def fk_batch_destroy(b):
    load().fk_batch_destroy(b)


def fk_score_batched(b, q, q_off, label, f=None, rescore=True, count=False, stream=None):
    """Scores the concatenated queries q (total, D) of all scenes; q_off (host
    int64, n_scenes + 1) gives each scene's rows."""
    import torch
    off, offp = _host(q_off, np.int64)
    total = int(off[-1])
    nr = ctypes.c_int64()
    _check(load().fk_score_batched(b, _dev(q, torch.float32, "q"), offp, int(bool(rescore)),
                                   None if f is None else _dev(f, torch.float32, "f", (total,)),
                                   _dev(label, torch.int8, "label", (total,)), ctypes.byref(nr) if count else None,
                                   _stream(stream)))
    return nr.value if count else None


def fk_batch_tune(b, q, q_off, label):
    import torch
    off, offp = _host(q_off, np.int64)
    ms = np.zeros(16, dtype=np.float32)
    best = ctypes.c_int()
    _check(load().fk_batch_tune(b, _dev(q, torch.float32, "q"), offp, _dev(label, torch.int8, "label"),
                                ms.ctypes.data_as(ctypes.c_void_p), 16, ctypes.byref(best)))
    return best.value, ms
