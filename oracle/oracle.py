"""Python face of the FP64 CPU oracle (fk_oracle.c) plus the small pieces that
are plainest in numpy (classification metrics).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path; both read their inputs from the seeded generator.

Every function cites the passage of Das and Yip, arXiv 1910.06451, that it
states.  Parity status: every function here is pinned by tests/test_oracle_*.py
against closed forms, invariants or brute force; nothing is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from paper_1910_06451_gb300 import synth  # the seeded generator (draws only)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def _elf_matches_host(path: str) -> bool:
    import platform
    want = {"x86_64": 0x3E, "aarch64": 0xB7, "arm64": 0xB7}.get(platform.machine())
    with open(path, "rb") as fh:
        head = fh.read(20)
    return len(head) == 20 and head[:4] == b"\x7fELF" and (want is None or int.from_bytes(head[18:20], "little") == want)


def build(force: bool = False) -> str:
    """Compile fk_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH) and _elf_matches_host(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        Dbl = ctypes.c_double
        lib.orc_frames.argtypes = [I, P, P, P, P]
        lib.orc_frames.restype = None
        lib.orc_fk_points.argtypes = [I, P, P, I, P, P, I64, P, P]
        lib.orc_fk_points.restype = I
        lib.orc_k_rq.argtypes = [I, P, P, Dbl]
        lib.orc_k_rq.restype = Dbl
        lib.orc_k_fk.argtypes = [I, P, P, Dbl]
        lib.orc_k_fk.restype = Dbl
        lib.orc_gram.argtypes = [I, Dbl, I64, P, I64, P, P]
        lib.orc_gram.restype = None
        lib.orc_score.argtypes = [I, Dbl, I64, P, P, I64, P, P, I]
        lib.orc_score.restype = I
        lib.orc_k_gauss.argtypes = [I, P, P, Dbl]
        lib.orc_k_gauss.restype = Dbl
        lib.orc_k_fk_s.argtypes = [I, P, P, Dbl, I]
        lib.orc_k_fk_s.restype = Dbl
        lib.orc_gram_s.argtypes = [I, Dbl, I64, P, I64, P, P, I]
        lib.orc_gram_s.restype = None
        lib.orc_score_s.argtypes = [I, Dbl, I64, P, P, I64, P, P, I, I]
        lib.orc_score_s.restype = I
        lib.orc_fastron_train_kind.argtypes = [I, Dbl, I64, P, P, Dbl, I64, I64, P, P, P, P, P, P, I, I]
        lib.orc_fastron_train_kind.restype = I
        lib.orc_fastron_train_mt.argtypes = [I, Dbl, I64, P, P, Dbl, I64, I64, P, P, P, P, P, P, I, I, I]
        lib.orc_fastron_train_mt.restype = I
        lib.orc_fastron_train.argtypes = [I, Dbl, I64, P, P, Dbl, I64, I64, P, P, P, P, P, P]
        lib.orc_fastron_train.restype = I
        lib.orc_fastron_train_store.argtypes = [I, Dbl, I64, P, P, Dbl, I64, I64, P, P, P, P, P, P, I]
        lib.orc_fastron_train_store.restype = I
        lib.orc_margins.argtypes = [I, Dbl, I64, P, I64, P, I, P]
        lib.orc_margins.restype = None
        lib.orc_seg_box_dist2.argtypes = [P, P, P, P]
        lib.orc_seg_box_dist2.restype = Dbl
        lib.orc_check.argtypes = [I, P, P, I64, P, Dbl, I64, P, P]
        lib.orc_check.restype = I
        _lib = lib
        return lib


def _d(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ FK ----

def frames(dh, base, q) -> np.ndarray:
    """Frame poses wA_0 .. wA_D of one configuration (Sec. II-A, Eqs. 1-2)."""
    dh, base, q = _d(dh), _d(base), _d(q)
    D = dh.shape[0]
    T = np.empty((D + 1, 4, 4))
    _load().orc_frames(D, _p(dh), _p(base), _p(q), _p(T))
    return T


def fk_points(arm, q) -> np.ndarray:
    """Control-point positions FK_m(x) for every configuration (Eq. 2): (n, M, 3)."""
    dh, base = _d(arm.dh), _d(arm.base)
    q = _d(q).reshape(-1, arm.D)
    cj = np.ascontiguousarray(arm.cp_joint, dtype=np.int32)
    co = _d(arm.cp_off)
    out = np.empty((q.shape[0], arm.M, 3))
    rc = _load().orc_fk_points(arm.D, _p(dh), _p(base), arm.M, _p(cj), _p(co), q.shape[0], _p(q), _p(out))
    if rc != 0:
        raise ValueError(f"orc_fk_points failed ({rc})")
    return out


# -------------------------------------------------------------- kernels ---

def k_rq(x, xp, gamma: float) -> float:
    """Rational quadratic kernel, Eq. 3."""
    x, xp = _d(x), _d(xp)
    return _load().orc_k_rq(x.shape[0], _p(x), _p(xp), float(gamma))


# Summand of the FK kernel: "rq" is the paper's (Eq. 3); "gauss" is the
# library's non-paper alternative exp(-gamma/2 |x - x'|^2) in the same mean
# over control points (Eq. 4 with exp in place of the RQ term).
SUMMANDS = {"rq": 0, "gauss": 1}


def k_gauss(x, xp, gamma: float) -> float:
    """Gaussian summand exp(-gamma/2 |x - x'|^2) (not in the paper)."""
    x, xp = _d(x), _d(xp)
    return _load().orc_k_gauss(x.shape[0], _p(x), _p(xp), float(gamma))


def k_fk(cpa, cpb, gamma: float, summand: str = "rq") -> float:
    """FK kernel, Eq. 4, between two (M, 3) control-point sets."""
    cpa, cpb = _d(cpa), _d(cpb)
    return _load().orc_k_fk_s(cpa.shape[0], _p(cpa), _p(cpb), float(gamma), SUMMANDS[summand])


def gram(cpa, cpb, gamma: float, summand: str = "rq") -> np.ndarray:
    """Kernel matrix K_ij = K_FK(a_i, b_j) (Sec. II-B)."""
    cpa, cpb = _d(cpa), _d(cpb)
    na, M = cpa.shape[0], cpa.shape[1]
    nb = cpb.shape[0]
    K = np.empty((na, nb))
    _load().orc_gram_s(M, float(gamma), na, _p(cpa), nb, _p(cpb), _p(K), SUMMANDS[summand])
    return K


def score_points(cps, alpha, cpq, gamma: float, nthreads: int = 1, summand: str = "rq") -> np.ndarray:
    """Fastron model value f(x) = sum_s alpha_s K_FK(S_s, x) (Sec. III-B) from control points."""
    cps, alpha, cpq = _d(cps), _d(alpha), _d(cpq)
    f = np.empty(cpq.shape[0])
    rc = _load().orc_score_s(cps.shape[1] if cps.ndim == 3 else cpq.shape[1], float(gamma), cps.shape[0],
                             _p(cps), _p(alpha), cpq.shape[0], _p(cpq), _p(f), int(nthreads), SUMMANDS[summand])
    if rc != 0:
        raise RuntimeError("orc_score failed")
    return f


def score(arm, support_q, alpha, query_q, gamma: float, nthreads: int = 1, summand: str = "rq") -> np.ndarray:
    """f for query configurations against a support set given as configurations."""
    return score_points(fk_points(arm, support_q), alpha, fk_points(arm, query_q), gamma, nthreads, summand)


def labels_from_f(f) -> np.ndarray:
    """Sign rule (Sec. III-B): f > 0 -> C_obs (+1), f < 0 -> C_free (-1); f = 0 is read as +1."""
    return np.where(np.asarray(f) >= 0.0, 1, -1).astype(np.int8)


# -------------------------------------------------------------- Fastron ---

class TrainResult:
    def __init__(self, alpha, F, stats, trace):
        self.alpha = alpha
        self.F = F
        self.iters, self.adds, self.removes, conv, self.n_support = (int(v) for v in stats)
        self.converged = bool(conv)
        self.trace = trace

    @property
    def support(self) -> np.ndarray:
        """removeNonsupportPoints: ascending training indices with alpha != 0."""
        return np.flatnonzero(self.alpha != 0.0)


def fastron_train(cpX, y, gamma: float, beta: float = 1.0, iter_max: int = 5000, s_max: int | None = None,
                  alpha0=None, F0=None, trace: bool = False, store32: bool = False,
                  summand: str = "rq", nthreads: int = 1) -> TrainResult:
    """Algorithm 1 (Sec. III-B) on training control points cpX (N, M, 3) and labels y in {+1, -1}.

    alpha0/F0 warm-start the model (loadPreviousModel); zeros otherwise.
    store32: kernel-matrix entries rounded to the nearest FP32 value (the
    matrix held in single precision); margins and weights stay FP64.
    summand: "rq" (the paper's kernel) or "gauss" (see SUMMANDS).
    nthreads: threads sharing the entries of each kernel-matrix column (the
    result does not depend on it)."""
    cpX = _d(cpX)
    N, M = cpX.shape[0], cpX.shape[1]
    y = np.ascontiguousarray(y, dtype=np.int8)
    alpha = np.zeros(N) if alpha0 is None else _d(alpha0).copy()
    F = np.zeros(N) if F0 is None else _d(F0).copy()
    stats = np.zeros(5, dtype=np.int64)
    s_max = N if s_max is None else int(s_max)
    if trace:
        tk = np.zeros(iter_max, dtype=np.int8)
        ti = np.full(iter_max, -1, dtype=np.int64)
        td = np.zeros(iter_max)
        tr = (_p(tk), _p(ti), _p(td))
    else:
        tr = (None, None, None)
    rc = _load().orc_fastron_train_mt(M, float(gamma), N, _p(cpX), _p(y), float(beta), int(iter_max), s_max,
                                      _p(alpha), _p(F), _p(stats), *tr, int(bool(store32)), SUMMANDS[summand],
                                      int(nthreads))
    if rc != 0:
        raise RuntimeError("orc_fastron_train failed")
    tr_out = None
    if trace:
        k = int(stats[0])
        tr_out = (tk[:k].copy(), ti[:k].copy(), td[:k].copy())
    return TrainResult(alpha, F, stats, tr_out)


def margins(cpX, ns: int, alpha_s, gamma: float, store32: bool = False) -> np.ndarray:
    """F = K alpha0 for a training set whose first ns points carry weights
    alpha_s and the rest 0 (loadPreviousModel on a changed training set),
    summed in ascending support order."""
    cpX = _d(cpX)
    N, M = cpX.shape[0], cpX.shape[1]
    a = _d(alpha_s)
    assert a.shape[0] == ns <= N
    F = np.empty(N)
    _load().orc_margins(M, float(gamma), N, _p(cpX), int(ns), _p(a), int(bool(store32)), _p(F))
    return F


def active_samples(support_q, k_near: int, sigma: float, n_uniform: int, qlim: float, seed: int) -> np.ndarray:
    """Two-stage active learning (Sec. III-B, after Algorithm 1): the support
    configurations, then k_near random samples near each of them (uniform in
    +-sigma per joint, clipped to the joint limits), then n_uniform samples
    uniform in the joint limits.  Draw ((c ns + s) D + d) of SplitMix64 stream
    `seed` perturbs joint d of support point s in copy c; draw
    (k_near ns D + i D + d) gives joint d of uniform sample i.  Every new
    value is computed in FP64 (lo + (hi - lo) u, then the sum and the clip)
    and rounded to FP32 once."""
    S = _d(support_q)
    ns, D = S.shape
    st = synth.Stream(seed)
    near = st.uniform(k_near * ns * D, -sigma, sigma).reshape(k_near, ns, D)
    out = [S]
    for c in range(k_near):
        v = np.clip(S + near[c], -qlim, qlim)
        out.append(v.astype(np.float32).astype(np.float64))
    uni = st.uniform(n_uniform * D, -qlim, qlim).reshape(n_uniform, D)
    out.append(uni.astype(np.float32).astype(np.float64))
    return np.concatenate(out, axis=0)


# -------------------------------------------------------------- checker ---

def seg_box_dist2(p0, p1, lo, hi) -> float:
    """Squared distance between a segment and an axis-aligned box."""
    p0, p1, lo, hi = _d(p0), _d(p1), _d(lo), _d(hi)
    return _load().orc_seg_box_dist2(_p(p0), _p(p1), _p(lo), _p(hi))


def check(scene, q) -> np.ndarray:
    """Ground-truth labels from sphere-swept links vs boxes (stands in for FCL, Sec. IV)."""
    arm = scene.arm
    dh, base, boxes = _d(arm.dh), _d(arm.base), _d(scene.boxes)
    q = _d(q).reshape(-1, arm.D)
    y = np.empty(q.shape[0], dtype=np.int8)
    rc = _load().orc_check(arm.D, _p(dh), _p(base), boxes.shape[0], _p(boxes), float(scene.radius),
                           q.shape[0], _p(q), _p(y))
    if rc != 0:
        raise RuntimeError("orc_check failed")
    return y


# -------------------------------------------------------------- metrics ---

def metrics(y_true, y_pred) -> dict:
    """Accuracy, TPR and TNR, Eqs. 10-12 (positive class = C_obs = +1)."""
    yt, yp = np.asarray(y_true), np.asarray(y_pred)
    tp = int(np.sum((yt == 1) & (yp == 1)))
    tn = int(np.sum((yt == -1) & (yp == -1)))
    fp = int(np.sum((yt == -1) & (yp == 1)))
    fn = int(np.sum((yt == 1) & (yp == -1)))
    tot = tp + tn + fp + fn
    return {
        "accuracy": (tp + tn) / tot if tot else float("nan"),
        "tpr": tp / (tp + fn) if tp + fn else float("nan"),
        "tnr": tn / (tn + fp) if tn + fp else float("nan"),
        "tp": tp, "tn": tn, "fp": fp, "fn": fn,
    }
