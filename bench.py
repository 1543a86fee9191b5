"""Benchmark: proxy collision checks per second on the 7-DOF workload
(7-DOF arm, 8 control points, 10 boxes, N = 5000 training configurations,
4,194,304 uniform query configurations, FK kernel with gamma = 40).

One step is one pass of the whole path over one batch:
  ground-truth labels of the N training configurations (GPU checker),
  FP64 control points and FP64 kernel matrix, Fastron Algorithm 1,
  support packing, then FK + FP32 score + FP64 re-score of the band for
  every query of the batch, whose labels are the output.
value = queries per second of steps (each query is one proxy collision check).
The K timed steps are pipelined: step s's update runs beside step s-1's
query pass (two streams, two models), so the SMs that Algorithm 1's single
cluster leaves idle score queries meanwhile; every step still does all of
its work, and the last labels are checked against a sequential step's.
e2e (host buffers, copies inside the timed region) runs the same pipeline:
each update copies the training set in, each query pass copies the batch in
and its labels out.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1910_06451_gb300 import shard, synth  # noqa: E402

WORKLOAD = "arm7-n5000"
N_QUERY = 1 << 22
# DRAM bytes read + written by one launch of the FP32 score kernel on this
# workload (4,194,304 queries, 800 support points), from an ncu capture of
# the kernel as it stands (dram__bytes_read.sum + dram__bytes_write.sum:
# 117,847,040 + 4,649,472): the queries in and the labels out, no re-reads.
SCORE_TRAFFIC_BYTES = 122496512
METRIC = "proxy collision checks/s (7-DOF): half2+surrogate vs plain FP32, oracle-exact labels"
UNIT = "checks/s"
L2_FLUSH_BYTES = 512 << 20


def _dist():
    ws, rank, _ = shard.world()
    return ws, rank


class ClockSampler:
    """Samples SM clocks and throttle reasons while the timed steps run: one
    nvidia-smi process streaming a line every 50 ms (its own child process,
    ended by terminate()); start() returns once the first line has arrived,
    and only lines that arrive after that are kept."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0, period_ms: int = 50):
        self.index = index
        self.period_ms = period_ms
        self.samples = []  # (time, fields)
        self.t0 = None
        self._proc = None
        self._th = None
        self._first = threading.Event()

    def start(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                           "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return

        def run():
            for line in self._proc.stdout:
                line = line.strip()
                if line:
                    self.samples.append((time.time(), [x.strip() for x in line.split(",")]))
                    self._first.set()
        self._th = threading.Thread(target=run, daemon=True)
        self._th.start()
        self._first.wait(5.0)
        self.t0 = time.time()

    def stop(self) -> dict:
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._th:
            self._th.join(timeout=5)
        during = [f for t, f in self.samples if self.t0 is not None and t >= self.t0]
        if not during and self.samples:
            during = [self.samples[-1][1]]
        if not during:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(f[0]) for f in during if f[0].replace(".", "").isdigit()]
        mx = [float(f[1]) for f in during if f[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for f in during for i in range(4) if len(f) > 4 + i and "Active" in f[4 + i]
                          and "Not" not in f[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(during)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def oracle_cpu_baseline(w, sample_queries: int, threads: int) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample: labels + training on
    the full training set, scoring of `sample_queries` queries; the per-query
    time is scaled to the full batch."""
    from oracle import oracle as O
    arm = w.scene.arm
    X = w.train_configs().astype(np.float64)
    t0 = time.perf_counter()
    y = O.check(w.scene, X)
    r = O.fastron_train(O.fk_points(arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max)
    t1 = time.perf_counter()
    Q = w.query_configs(sample_queries).astype(np.float64)
    S = X[r.support]
    f = O.score(arm, S, r.alpha[r.support], Q, w.gamma, nthreads=threads)
    O.labels_from_f(f)
    t2 = time.perf_counter()
    per_q = (t2 - t1) / sample_queries
    step = (t1 - t0) + per_q * N_QUERY
    # one core, for the per-check time beside the paper's (Table I)
    n1 = max(1, min(2048, sample_queries))
    t3 = time.perf_counter()
    O.score(arm, S, r.alpha[r.support], Q[:n1], w.gamma, nthreads=1)
    per_q1 = (time.perf_counter() - t3) / n1
    return {"value": N_QUERY / step, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"labels+Algorithm 1 on all {w.n_train} training configs ({t1 - t0:.2f} s), "
                      f"FP64 scoring of {sample_queries} of {N_QUERY} queries ({t2 - t1:.2f} s) scaled to the batch",
            "train_s": t1 - t0, "score_us_per_query": per_q * 1e6, "score_us_per_query_1core": per_q1 * 1e6,
            "n_support": int(r.n_support)}


def run_pipelined(update, query, steps: int) -> None:
    """Runs update(0); then, for s = 1 .. steps - 1, update(s) beside
    query(s - 1), one host thread each, both finished before the next pair
    starts; then query(steps - 1).  So step s's query pass always follows its
    own update, and update(s + 1) never starts before query(s - 1) has ended
    (two models can alternate).  An exception raised by either call is
    re-raised once both threads of its pair have finished."""
    errors = []

    def guarded(fn, s):
        try:
            fn(s)
        except BaseException as e:  # re-raised by the calling thread
            errors.append(e)

    if steps <= 0:
        return
    update(0)
    for s in range(1, steps):
        ta = threading.Thread(target=guarded, args=(update, s))
        tb = threading.Thread(target=guarded, args=(query, s - 1))
        ta.start()
        tb.start()
        ta.join()
        tb.join()
        if errors:
            raise errors[0]
    query(steps - 1)


def label_checksum(lab) -> dict:
    """Count of +1 labels and a position-weighted sum of them (mod 2^61 - 1):
    two arms with these equal labelled the batch alike."""
    lab = np.asarray(lab).astype(np.int64)
    pos = np.flatnonzero(lab == 1).astype(np.int64)
    h = int(np.sum((pos * 2654435761 + 97) % 2305843009213693951) % 2305843009213693951)
    return {"positive": int(pos.size), "weighted": h}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands runs the whole step on
    the host cores - labels of the training set, Algorithm 1, and the FP64
    score of every query of the batch - timed step by step."""
    ws, rank = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    w = synth.workload(WORKLOAD)
    arm = w.scene.arm
    threads = os.cpu_count() or 1
    X = w.train_configs().astype(np.float64)
    nq = args.queries
    Q = w.query_configs(nq).astype(np.float64)
    times, train_s = [], []
    lab = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        y = O.check(w.scene, X)
        r = O.fastron_train(O.fk_points(arm, X), y, w.gamma, w.beta, w.iter_max, w.s_max)
        t1 = time.perf_counter()
        f = O.score(arm, X[r.support], r.alpha[r.support], Q, w.gamma, nthreads=threads)
        lab = O.labels_from_f(f)
        t2 = time.perf_counter()
        if i >= args.warmup:
            times.append(t2 - t0)
            train_s.append(t1 - t0)
    ms = statistics.mean(times) * 1e3
    value = nq / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_train": w.n_train, "n_query": nq, "gamma": w.gamma,
                       "l2": "host CPU run", "step": "labels + Algorithm 1 + FP64 score of every query, timed"},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value, "unit": UNIT,
                             "sample": f"the whole {nq}-query step (labels and training "
                                       f"{statistics.mean(train_s):.2f} s of it)"},
            "labels_checksum": label_checksum(lab),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def small_3dof(fk, dev, rank, flush, steps=20):
    """The small 3-DOF workload (3-DOF arm, 4 control points, 6 boxes, N = 1000
    training configurations, 10,000 queries, gamma = 10): the same step
    (labels, kernel matrix, Algorithm 1, score with the band re-score), timed
    over `steps` steps.  At this size the step is bound by launch and
    synchronisation latency, not by the kernels' throughput."""
    import torch
    w = synth.workload("arm3-n1000", trial=rank)
    ch = fk.chain_from_arm(w.scene.arm)
    m = fk.fastron_model_create(ch)
    try:
        X = torch.from_numpy(w.train_configs().astype(np.float64)).to(dev)
        X32 = X.float()
        Q = torch.from_numpy(w.query_configs()).to(dev)
        y = torch.empty(w.n_train, dtype=torch.int8, device=dev)
        lab = torch.empty(Q.shape[0], dtype=torch.int8, device=dev)

        def step():
            fk.fk_label(ch, w.scene.boxes, w.scene.radius, X32, y)
            st = fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max)
            fk.fk_score(m, Q, lab, rescore=True)
            return st

        for _ in range(3):
            st = step()
        torch.cuda.synchronize()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            step()
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        fk.fk_score(m, Q, lab, rescore=True)
        e[1].record()
        e[1].synchronize()
        return {"workload": w.name, "support": st["n_support"], "iterations": st["iterations"], "ms_per_step": ms,
                "checks_per_s": Q.shape[0] / ms * 1e3, "query_ms": e[0].elapsed_time(e[1])}
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


def gaussian_summand(fk, dev, rank, Q, X32, X, flush, peak):
    """The same 7-DOF workload with the library's non-paper Gaussian summand
    (FK_SUMMAND_GAUSS): labels, FP64 kernel matrix and Algorithm 1, then the
    query batch scored in FP32 on MUFU ex2, with 1 or 2 of the 7 summands per
    support point on the FMA polynomial instead, and in packed half
    (ex2.f16x2); every path with its band re-scored, labels compared with the
    FP32 path's.  Roofline as for the RQ score: one transcendental and five
    FP32 operations per evaluation."""
    import torch
    w = synth.workload(WORKLOAD, trial=rank)
    ch = fk.chain_from_arm(w.scene.arm)
    fk.fk_chain_set_summand(ch, fk.FK_SUMMAND_GAUSS)
    m = fk.fastron_model_create(ch)
    nq = Q.shape[0]
    y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
    ref = torch.empty(nq, dtype=torch.int8, device=dev)
    lab = torch.empty(nq, dtype=torch.int8, device=dev)

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    try:
        fk.fk_label(ch, w.scene.boxes, w.scene.radius, X32, y)
        t_train = timed(lambda: fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max), reps=1)
        st = fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max)
        evals = st["n_support"] * int(np.sum(w.scene.arm.cp_joint != 0)) * nq
        fk.fk_score(m, Q, ref, rescore=True)
        out = {"summand": "exp(-gamma/2 |d|^2) (not the paper's kernel)", "support": st["n_support"],
               "iterations": st["iterations"], "update_ms": t_train}
        for poly in (0, 1, 2):
            fk.fk_set_gauss_poly(poly)
            t_raw = timed(lambda: fk.fk_score(m, Q, lab, rescore=False))
            nb = fk.fk_score(m, Q, lab, rescore=True, count=True)
            t_all = timed(lambda: fk.fk_score(m, Q, lab, rescore=True))
            out[f"fp32_poly{poly}"] = {"score_ms": t_raw, "teval_per_s": evals / t_raw / 1e9,
                                       "roofline_frac": evals / t_raw / 1e9 / peak, "rescored": nb,
                                       "with_rescore_ms": t_all, "checks_per_s": nq / t_all * 1e3,
                                       "label_mismatch": int((lab != ref).sum().item())}
        fk.fk_set_gauss_poly(0)
        t_raw = timed(lambda: fk.fk_score(m, Q, lab, rescore=False, precision=fk.FK_F16))
        nb = fk.fk_score(m, Q, lab, rescore=True, count=True, precision=fk.FK_F16)
        t_all = timed(lambda: fk.fk_score(m, Q, lab, rescore=True, precision=fk.FK_F16))
        out["half2"] = {"score_ms": t_raw, "teval_per_s": evals / t_raw / 1e9, "band_to_fp32": nb / nq,
                        "with_rescore_ms": t_all, "checks_per_s": nq / t_all * 1e3,
                        "label_mismatch": int((lab != ref).sum().item())}
        return out
    finally:
        fk.fk_set_gauss_poly(0)
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


def obstacle_sweep(fk, dev, rank, counts, Q, X32, X, flush):
    """Query cost of the proxy check against the geometric checker as the
    number of boxes grows (the sweep of Sec. IV-A, 1-50 random boxes): per box
    count, the 7-DOF arm's 5000 training configurations are labelled and the
    model trained; then the query batch is labelled by the checker and scored
    by the model (FP32 with the band re-score), each timed alone; the model's
    labels are compared with the checker's (accuracy, TPR, TNR of Sec. IV-A)."""
    import torch
    w = synth.workload(WORKLOAD, trial=rank)
    ch = fk.chain_from_arm(w.scene.arm)
    m = fk.fastron_model_create(ch)
    nq = Q.shape[0]
    y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
    truth = torch.empty(nq, dtype=torch.int8, device=dev)
    lab = torch.empty(nq, dtype=torch.int8, device=dev)

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = []
    try:
        for nb in counts:
            boxes = synth.random_boxes(w.seed * 97 + nb, nb)
            fk.fk_label(ch, boxes, w.scene.radius, X32, y)
            st = fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max)
            t_chk = timed(lambda: fk.fk_label(ch, boxes, w.scene.radius, Q, truth))
            t_fk = timed(lambda: fk.fk_score(m, Q, lab, rescore=True))
            pos, pred = truth == 1, lab == 1
            tp = int((pos & pred).sum().item())
            tn = int((~pos & ~pred).sum().item())
            npos = int(pos.sum().item())
            out.append({"boxes": nb, "in_collision": npos / nq, "support": st["n_support"],
                        "iterations": st["iterations"], "proxy_checks_per_s": nq / t_fk * 1e3,
                        "checker_checks_per_s": nq / t_chk * 1e3, "accuracy": (tp + tn) / nq,
                        "tpr": tp / max(npos, 1), "tnr": tn / max(nq - npos, 1)})
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)
    return out


def changing_environment(fk, dev, rank, frames, nq, modes=("warm", "cold", "active", "pipelined", "surrogate"),
                         short=None):
    """The 12-control-point arm among moving boxes: a fixed training set of
    65,536 configurations relabelled every frame, Algorithm 1 on the stored
    FP32 kernel matrix (built once), then the query batch scored.  Each frame
    runs twice over the same box path: warm-started from the previous frame's
    model (loadPreviousModel) and from zero; then a third time as the paper's
    loop, two-stage active learning: the next training set (65,536 rows) is
    the support set, one copy of it moved by up to 0.1 rad per joint, and
    uniform samples; it is relabelled, its kernel matrix rebuilt, and
    Algorithm 1 starts from the carried weights.  A fourth pass adds the
    learned surrogate: after each cold update it is fine-tuned (one epoch on
    a fixed 1M-query set scored by the new model, threshold recalibrated) and
    answers the frame's queries, falling back to the exact score below the
    threshold; its labels are compared with the exact path's.  A fifth pass
    repeats the cold mode with each frame's update overlapped with the
    previous frame's query pass (pipelined_frames).  Per-frame device times.
    The cold, pipelined and surrogate modes run `frames` frames, the
    warm-start and active-learning modes `short` (default: the same)."""
    import torch
    wd = synth.workload("arm7m12-n65536", trial=rank)
    ch = fk.chain_from_arm(wd.scene.arm)
    m = fk.fastron_model_create(ch)
    try:
        X = torch.from_numpy(wd.train_configs().astype(np.float64)).to(dev)
        X32 = X.float()
        Q = torch.from_numpy(wd.query_configs(nq)).to(dev)
        boxes = synth.moving_boxes(wd.seed, wd.scene.boxes, frames)
        y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
        lab = torch.empty(nq, dtype=torch.int8, device=dev)

        def ev():
            e = torch.cuda.Event(enable_timing=True)
            e.record()
            return e

        torch.cuda.synchronize()
        e0 = ev()
        fk.fk_label(ch, boxes[0], wd.scene.radius, X32, y)
        st0 = fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max, gram=fk.FK_DF32)
        e1 = ev()
        torch.cuda.synchronize()
        setup_ms = e0.elapsed_time(e1)
        out = {"workload": wd.name, "n_train": X.shape[0], "control_points": wd.scene.arm.M, "queries_per_frame": nq,
               "frames": frames, "kernel_matrix": "fp32 (double-float entries rounded once), built once",
               "frame0_cold_with_matrix_ms": setup_ms, "frame0_support": st0["n_support"],
               "frame0_iterations": st0["iterations"]}
        n_max = X.shape[0]
        cold_sums = []
        Xa = torch.empty_like(X)
        Xa32 = torch.empty_like(X32)
        for mode in [m for m in ("warm", "cold", "active") if m in modes]:
            # every mode starts from the frame-0 model; the stored matrix is X's
            # here (the active mode, which replaces it, runs last of the three)
            fk.fk_label(ch, boxes[0], wd.scene.radius, X32, y)
            fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max, gram=fk.FK_DF32, reuse_gram=True)
            ns = st0["n_support"]
            upd, qry, its, sup, conv, nres = [], [], [], [], [], []
            nf = frames if mode == "cold" or short is None else min(frames, short)
            for k in range(1, nf):
                torch.cuda.synchronize()
                a = ev()
                if mode == "active":
                    kn = 1 if 2 * ns <= n_max else 0
                    nu = max(0, n_max - (1 + kn) * ns)
                    n = fk.fk_active_samples(m, kn, 0.1, nu, wd.scene.arm.qlim, wd.seed * 7919 + k, Xa, Xa32)
                    fk.fk_label(ch, boxes[k], wd.scene.radius, Xa32[:n], y[:n])
                    st = fk.fastron_train(m, Xa[:n], y[:n], wd.gamma, wd.beta, wd.iter_max, wd.s_max, warm_start=2,
                                          gram=fk.FK_DF32)
                    ns = st["n_support"]
                else:
                    fk.fk_label(ch, boxes[k], wd.scene.radius, X32, y)
                    st = fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max,
                                          warm_start=mode == "warm", gram=fk.FK_DF32, reuse_gram=True)
                b = ev()
                nr = fk.fk_score(m, Q, lab, rescore=True, count=True)
                c = ev()
                torch.cuda.synchronize()
                upd.append(a.elapsed_time(b))
                qry.append(b.elapsed_time(c))
                if mode == "cold":
                    cold_sums.append(label_checksum(lab.cpu().numpy()))
                its.append(st["iterations"])
                sup.append(st["n_support"])
                conv.append(bool(st["converged"]))
                nres.append(nr)
            tot = [u + q for u, q in zip(upd, qry)]
            out[mode] = {"update_ms_p50": float(np.percentile(upd, 50)), "update_ms_p99": float(np.percentile(upd, 99)),
                         "query_ms_p50": float(np.percentile(qry, 50)), "query_ms_p99": float(np.percentile(qry, 99)),
                         "frame_ms_p50": float(np.percentile(tot, 50)), "frame_ms_p99": float(np.percentile(tot, 99)),
                         "frames": nf, "iterations": its, "support": sup, "converged": conv, "rescored": nres,
                         "checks_per_s_p50": nq / (float(np.percentile(tot, 50)) * 1e-3)}
        if "pipelined" in modes:
            out["pipelined"] = pipelined_frames(fk, dev, wd, ch, m, X, X32, y, Q, boxes, frames, cold_sums)
        if "surrogate" in modes:
            out["surrogate"] = surrogate_frames(fk, dev, wd, ch, m, X, X32, y, Q, lab, boxes, ev)
        return out
    finally:
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


def pipelined_frames(fk, dev, wd, ch, m, X, X32, y, Q, boxes, frames, cold_sums):
    """The cold mode's frames with the update and the query pass overlapped:
    while Algorithm 1 runs for frame k (one 16-CTA cluster, on a
    higher-priority stream, from one host thread), frame k-1's queries are
    scored with a snapshot of frame k-1's model (fastron_model_copy) on the
    other SMs (another stream and thread).  A frame's labels come out one
    update later; the frame period is the wall time of one such step.  Each
    frame's label checksum is compared with the sequential cold mode's."""
    import threading
    import torch
    nq = Q.shape[0]
    snaps = [fk.fastron_model_create(ch), fk.fastron_model_create(ch)]
    U = torch.cuda.Stream(priority=-1)
    S = torch.cuda.Stream(priority=0)
    lab = torch.empty(nq, dtype=torch.int8, device=dev)
    sums, period, errors = [None] * frames, [], []
    try:
        def update(k):
            try:
                with torch.cuda.stream(U):
                    fk.fk_label(ch, boxes[k], wd.scene.radius, X32, y, stream=U)
                    fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max, gram=fk.FK_DF32,
                                     reuse_gram=True, stream=U)
                    fk.fastron_model_copy(snaps[k % 2], m, stream=U)
                    U.synchronize()
            except Exception as e:  # re-raised by the main thread
                errors.append(e)

        def query(k):
            try:
                with torch.cuda.stream(S):
                    fk.fk_score(snaps[k % 2], Q, lab, rescore=True, stream=S)
                    S.synchronize()
                    sums[k] = label_checksum(lab.cpu().numpy())
            except Exception as e:
                errors.append(e)

        # the stored matrix is X's again (the active mode replaced it)
        fk.fk_label(ch, boxes[0], wd.scene.radius, X32, y)
        fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max, gram=fk.FK_DF32)
        torch.cuda.synchronize()
        fk.fastron_model_copy(snaps[0], m)
        for k in range(1, frames):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ta = threading.Thread(target=update, args=(k,))
            tb = threading.Thread(target=query, args=(k - 1,))
            ta.start()
            tb.start()
            ta.join()
            tb.join()
            period.append((time.perf_counter() - t0) * 1e3)
            if errors:
                raise errors[0]
        query(frames - 1)
        if errors:
            raise errors[0]
        # frames 1.. of the cold mode are the same updates in the same order
        same = [sums[k] == cold_sums[k - 1] for k in range(1, frames) if k - 1 < len(cold_sums)]
        return {"frames": frames, "frame_period_ms_p50": float(np.percentile(period, 50)),
                "frame_period_ms_p99": float(np.percentile(period, 99)),
                "checks_per_s_p50": nq / (float(np.percentile(period, 50)) * 1e-3),
                "labels_equal_cold": bool(same) and all(same), "frames_compared": len(same),
                "overlap": "update k (cluster kernel, priority stream) beside the query pass of k-1"}
    finally:
        for x in snaps:
            fk.fastron_model_destroy(x)


def surrogate_frames(fk, dev, wd, ch, m, X, X32, y, Q, lab, boxes, ev):
    import torch
    nq = Q.shape[0]
    sur = fk.surrogate_create(ch, seed=11)
    try:
        qtr = torch.from_numpy(synth.uniform_configs(wd.seed + 9, 1 << 20, wd.scene.arm.D, wd.scene.arm.qlim)).to(dev)
        # the matrix is rebuilt: an earlier mode may have left another training set's
        fk.fk_label(ch, boxes[0], wd.scene.radius, X32, y)
        fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max, gram=fk.FK_DF32)
        torch.cuda.synchronize()
        a = ev()
        fk.surrogate_train(sur, m, qtr, epochs=96, batch=8192, lr=3e-3, holdout=0.0625, reinit=True,
                           schedule=fk.FK_LR_COSINE)
        b = ev()
        torch.cuda.synchronize()
        first = a.elapsed_time(b)
        exact = torch.empty(nq, dtype=torch.int8, device=dev)
        upd, tune, qry, fb, mism = [], [], [], [], []
        for k in range(1, len(boxes)):
            torch.cuda.synchronize()
            e0 = ev()
            fk.fk_label(ch, boxes[k], wd.scene.radius, X32, y)
            fk.fastron_train(m, X, y, wd.gamma, wd.beta, wd.iter_max, wd.s_max, gram=fk.FK_DF32, reuse_gram=True)
            e1 = ev()
            fk.surrogate_train(sur, m, qtr, epochs=1, batch=8192, lr=3e-4, holdout=0.0625, reinit=False)
            e2 = ev()
            nfb = fk.surrogate_infer(sur, m, Q, lab)
            e3 = ev()
            torch.cuda.synchronize()
            upd.append(e0.elapsed_time(e1))
            tune.append(e1.elapsed_time(e2))
            qry.append(e2.elapsed_time(e3))
            fb.append(nfb / nq)
            fk.fk_score(m, Q, exact, rescore=True)
            mism.append(int((lab != exact).sum().item()))
        tot = [u + t + q for u, t, q in zip(upd, tune, qry)]
        return {"first_train_ms": first, "update_ms_p50": float(np.percentile(upd, 50)),
                "finetune_ms_p50": float(np.percentile(tune, 50)), "query_ms_p50": float(np.percentile(qry, 50)),
                "query_ms_p99": float(np.percentile(qry, 99)), "frame_ms_p50": float(np.percentile(tot, 50)),
                "frame_ms_p99": float(np.percentile(tot, 99)), "fallback": fb, "label_mismatch": mism,
                "checks_per_s_p50": nq / (float(np.percentile(tot, 50)) * 1e-3)}
    finally:
        fk.surrogate_destroy(sur)


def metric_paths(fk, dev, chain, model, sur, w, nq, flush, train_s):
    """The comparison the headline metric names, on the surrogate
    configuration: the 7-DOF scene with 16,777,216 uniform queries.  Three
    query paths over the same batch - the exact FP32 path (labels equal the
    FP64 oracle's), the half-precision pass (its band through the FP32
    path, labels exact as well), and the learned surrogate with exact
    fallback - each timed alone (median of three, L2 flushed), with the
    surrogate's training time and the number of batches after which it pays
    for itself, its fallback fraction, and accuracy, TPR and TNR of every
    path against the geometric checker (fk_label) on the same queries."""
    import torch
    Q = torch.from_numpy(synth.uniform_configs(w.seed + 31, nq, w.scene.arm.D, w.scene.arm.qlim)).to(dev)
    truth = torch.empty(nq, dtype=torch.int8, device=dev)
    fk.fk_label(chain, w.scene.boxes, w.scene.radius, Q, truth)

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def quality(lab):
        t, p = truth == 1, lab == 1
        tp, tn = int((t & p).sum().item()), int((~t & ~p).sum().item())
        npos, nneg = int(t.sum().item()), nq - int(t.sum().item())
        return {"accuracy": (tp + tn) / nq, "tpr": tp / max(npos, 1), "tnr": tn / max(nneg, 1)}

    out = {"workload": f"{WORKLOAD} scene, {nq} uniform queries (surrogate configuration)", "queries": nq}
    exact = torch.empty(nq, dtype=torch.int8, device=dev)
    nb = fk.fk_score(model, Q, exact, rescore=True, count=True)
    t_exact = timed(lambda: fk.fk_score(model, Q, exact, rescore=True))
    out["fp32_exact"] = {"ms": t_exact, "checks_per_s": nq / (t_exact * 1e-3), "rescored": nb,
                         "label_mismatch_vs_exact": 0} | quality(exact)
    lab = torch.empty(nq, dtype=torch.int8, device=dev)
    nb16 = fk.fk_score(model, Q, lab, rescore=True, count=True, precision=fk.FK_F16)
    t_half = timed(lambda: fk.fk_score(model, Q, lab, rescore=True, precision=fk.FK_F16))
    out["half2_exact"] = {"ms": t_half, "checks_per_s": nq / (t_half * 1e-3), "band_to_fp32": nb16 / nq,
                          "speedup_vs_fp32": t_exact / t_half,
                          "label_mismatch_vs_exact": int((lab != exact).sum().item())} | quality(lab)
    if sur is not None:
        nfb = fk.surrogate_infer(sur, model, Q, lab)
        t_sur = timed(lambda: fk.surrogate_infer(sur, model, Q, lab))
        saved = t_exact - t_sur
        out["surrogate"] = {"ms": t_sur, "checks_per_s": nq / (t_sur * 1e-3), "fallback": nfb / nq,
                            "speedup_vs_fp32": t_exact / t_sur, "train_s": train_s,
                            "break_even_batches": (train_s * 1e3 / saved) if saved > 0 else None,
                            "label_mismatch_vs_exact": int((lab != exact).sum().item())} | quality(lab)
    out["note"] = ("labels of fp32_exact and half2_exact equal the FP64 oracle's (derived band + re-score); "
                   "the surrogate's confident answers are the network's")
    del Q, truth, exact, lab
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fkfast")
    ap.add_argument("--cpu-sample", type=int, default=16384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--queries", type=int, default=N_QUERY, help="query batch size (profiling runs use a smaller one)")
    ap.add_argument("--surrogate-train", type=int, default=1 << 21, help="surrogate training queries (0: skip)")
    ap.add_argument("--surrogate-epochs", type=int, default=192)
    ap.add_argument("--surrogate-lr", type=float, default=3e-3, help="peak of the cosine learning-rate schedule")
    ap.add_argument("--metric-queries", type=int, default=1 << 24,
                    help="queries of the metric-paths comparison (surrogate configuration; 0: skip)")
    ap.add_argument("--batch-scenes", type=int, default=256, help="scenes of the multi-scene measurement (0: skip)")
    ap.add_argument("--dynamic-frames", type=int, default=100,
                    help="frames of the changing-environment measurement, cold and surrogate modes (0: skip)")
    ap.add_argument("--dynamic-frames-short", type=int, default=8,
                    help="frames of the warm-start and active-learning modes")
    ap.add_argument("--dynamic-queries", type=int, default=1 << 24, help="queries per frame of that measurement")
    ap.add_argument("--dynamic-modes", default="warm,cold,active,pipelined,surrogate",
                    help="update modes of that measurement (comma-separated)")
    ap.add_argument("--gauss", type=int, default=1, help="measure the non-paper Gaussian summand (0: skip)")
    ap.add_argument("--small", type=int, default=1, help="measure the 3-DOF workload's step (0: skip)")
    ap.add_argument("--obstacle-sweep", default="1,2,5,10,20,35,50",
                    help="box counts of the obstacle sweep (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank = _dist()
    local = shard.world()[2]
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1910_06451_gb300 import build, fkfast as fk
    build.build()
    fk.load()

    # every rank runs an independent scene (trial = rank): the path shards by
    # scene and by query batch with no exchange
    w = synth.workload(WORKLOAD, trial=shard.rank_trial(rank))
    arm = w.scene.arm
    X = torch.from_numpy(w.train_configs().astype(np.float64)).to(dev)
    Xq32 = torch.from_numpy(w.train_configs()).to(dev)
    nq = args.queries
    Q = torch.from_numpy(w.query_configs(nq)).to(dev)
    ytr = torch.empty(w.n_train, dtype=torch.int8, device=dev)
    lab = torch.empty(nq, dtype=torch.int8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    chain = fk.chain_from_arm(arm)
    model = fk.fastron_model_create(chain)
    stream = torch.cuda.current_stream()

    def step(q_dev, x_dev, xq32_dev, lab_dev):
        fk.fk_label(chain, w.scene.boxes, w.scene.radius, xq32_dev, ytr)
        st = fk.fastron_train(model, x_dev, ytr, w.gamma, w.beta, w.iter_max, w.s_max)
        fk.fk_score(model, q_dev, lab_dev, rescore=True)
        return st

    # phase timing (untimed run): update vs query pass, band size
    st = step(Q, X, Xq32, lab)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    fk.fk_label(chain, w.scene.boxes, w.scene.radius, Xq32, ytr)
    st = fk.fastron_train(model, X, ytr, w.gamma, w.beta, w.iter_max, w.s_max)
    e[1].record()
    nres = fk.fk_score(model, Q, lab, rescore=True, count=True)
    e[2].record()
    fk.fk_score(model, Q, lab, rescore=False)
    e[3].record()
    torch.cuda.synchronize()
    update_ms = e[0].elapsed_time(e[1])
    query_ms = e[1].elapsed_time(e[2])
    score_only_ms = e[2].elapsed_time(e[3])

    for _ in range(args.warmup):
        flush.zero_()
        step(Q, X, Xq32, lab)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    # nvidia-smi numbers GPUs physically: map the local device through
    # CUDA_VISIBLE_DEVICES (an index or a UUID) when it is set
    visible = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    # The timed steps, pipelined: step s's update (labels, kernel matrix,
    # Algorithm 1 on one 16-CTA cluster, packing) runs on a high-priority
    # stream while step s-1's query pass (L2 flush, FP32 score, band
    # re-score) runs on another, each issued from its own host thread.  Two
    # models alternate, so a query pass reads a finished model while the next
    # one is trained.  Every step does all of its work; the overlap only puts
    # the SMs that Algorithm 1 leaves idle to use.  The region is timed with
    # CUDA events on the issuing stream, both work streams joined into it.
    ref_lab = lab.clone()  # the sequential step's labels
    models = [model, fk.fastron_model_create(chain)]
    labs = [lab, torch.empty_like(lab)]
    U = torch.cuda.Stream(device=dev, priority=-1)
    S = torch.cuda.Stream(device=dev, priority=0)

    def upd(s):
        with torch.cuda.stream(U):
            fk.fk_label(chain, w.scene.boxes, w.scene.radius, Xq32, ytr, stream=U)
            fk.fastron_train(models[s % 2], X, ytr, w.gamma, w.beta, w.iter_max, w.s_max, stream=U)
            U.synchronize()

    def qry(s):
        with torch.cuda.stream(S):
            flush.zero_()
            fk.fk_score(models[s % 2], Q, labs[s % 2], rescore=True, stream=S)
            S.synchronize()

    # two untimed pipelined steps: the second model's buffers are allocated
    # here, not in the timed region
    run_pipelined(upd, qry, 2)
    sampler = ClockSampler(visible[local].strip() if local < len(visible) else local)
    sampler.start()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    U.wait_event(a)
    S.wait_event(a)
    run_pipelined(upd, qry, args.steps)
    for st_ in (U, S):
        done = torch.cuda.Event()
        done.record(st_)
        torch.cuda.current_stream().wait_event(done)
    b.record()
    b.synchronize()
    clocks = sampler.stop()
    pipelined_equal = all(torch.equal(x, ref_lab) for x in labs[: min(2, args.steps)])
    lab = labs[(args.steps - 1) % 2]
    total_ms = shard.max_over_ranks(a.elapsed_time(b), dev)  # the slowest rank's time
    ms_per_step = total_ms / args.steps
    value = shard.aggregate_rate(nq, ws, ms_per_step)
    # kernels of this library per step: label; FK, pair split, kernel
    # matrix, Algorithm 1, compaction, packing; FP32 score, then band FK,
    # double-float summands, their finish and the FP64 re-score when the band
    # is not empty
    launches = 8 + (4 if nres > 0 else 0)

    # roofline of the dominant kernel: the FP32 score, one launch per step.
    # Algorithmic work = |S| * Mv RQ evaluations per query.
    Mv = int(np.sum(arm.cp_joint != 0))
    evals = st["n_support"] * Mv * nq
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    score_times = []
    for _ in range(5):
        flush.zero_()
        ev[0].record()
        fk.fk_score(model, Q, lab, rescore=False)
        ev[1].record()
        ev[1].synchronize()
        score_times.append(ev[0].elapsed_time(ev[1]))
    score_ms = statistics.median(score_times)
    achieved = evals / (score_ms * 1e-3) / 1e12
    # peak: the slower of the reciprocal (MUFU: 16 lanes/clk/SM, one per
    # evaluation) and the FP32 pipe (128 lanes/clk/SM, five operations per
    # evaluation: three products and two sums); the second, stricter figure
    # ignores the reciprocal altogether
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(clocks.get("sm_max_mhz") or _peaks().get("sm_max_mhz") or 2070.0)
    sm_clk = props.multi_processor_count * sm_max * 1e6
    peak_fp32_floor = sm_clk * 128 / 5 / 1e12
    peak = min(sm_clk * 16 / 1, sm_clk * 128 / 5) / 1e12

    # end to end through the public API with host buffers
    Qh = Q.cpu().pin_memory()
    Xh = X.cpu().pin_memory()
    X32h = Xq32.cpu().pin_memory()
    labh = torch.empty(nq, dtype=torch.int8).pin_memory()
    qd = torch.empty_like(Q)
    xd = torch.empty_like(X)
    x32d = torch.empty_like(Xq32)
    # pipelined like the timed steps: update(s) copies the training set in,
    # labels it and trains; query(s) copies the query batch in, scores it and
    # copies the labels out (the caller's host buffer), while the next update
    # runs.  L2 is flushed before every query pass.

    def upd_e(s):
        with torch.cuda.stream(U):
            xd.copy_(Xh, non_blocking=True)
            x32d.copy_(X32h, non_blocking=True)
            fk.fk_label(chain, w.scene.boxes, w.scene.radius, x32d, ytr, stream=U)
            fk.fastron_train(models[s % 2], xd, ytr, w.gamma, w.beta, w.iter_max, w.s_max, stream=U)
            U.synchronize()

    def qry_e(s):
        with torch.cuda.stream(S):
            qd.copy_(Qh, non_blocking=True)
            flush.zero_()
            fk.fk_score(models[s % 2], qd, labs[s % 2], rescore=True, stream=S)
            labh.copy_(labs[s % 2], non_blocking=True)
            S.synchronize()

    run_pipelined(upd_e, qry_e, args.warmup)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    U.wait_event(a)
    S.wait_event(a)
    run_pipelined(upd_e, qry_e, args.steps)
    for st_ in (U, S):
        done = torch.cuda.Event()
        done.record(st_)
        torch.cuda.current_stream().wait_event(done)
    b.record()
    b.synchronize()
    e2e_ms = shard.max_over_ranks(a.elapsed_time(b) / max(args.steps, 1), dev)
    e2e_equal = torch.equal(labh, ref_lab.cpu())
    fk.fastron_model_destroy(models[1])
    lab = labs[(args.steps - 1) % 2]
    # the step's labels as the caller receives them (exact: the oracle's),
    # for comparison with the reference arm's
    checksum = label_checksum(labh.numpy()) if nq == N_QUERY else None
    h2d = Qh.numel() * 4 + Xh.numel() * 8 + X32h.numel() * 4
    d2h = labh.numel()

    # query-pass alternatives on the same batch (not part of the step):
    # the learned surrogate with exact fallback, against the exact path
    paths = {"fp32_exact": {"checks_per_s": nq / (query_ms * 1e-3), "ms": query_ms, "label_mismatch": 0,
                            "rescored": nres}}
    # packed-half distances, band through the FP32 path and its FP64 re-score
    hlab = torch.empty(nq, dtype=torch.int8, device=dev)
    ex16 = torch.empty(nq, dtype=torch.int8, device=dev)
    fk.fk_score(model, Q, ex16, rescore=True)
    nb16 = fk.fk_score(model, Q, hlab, rescore=True, count=True, precision=fk.FK_F16)
    ht = []
    for _ in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fk.fk_score(model, Q, hlab, rescore=True, precision=fk.FK_F16)
        b.record()
        b.synchronize()
        ht.append(a.elapsed_time(b))
    hms = statistics.median(ht)
    paths["half2_exact"] = {"checks_per_s": nq / (hms * 1e-3), "ms": hms, "band_to_fp32": nb16 / nq,
                            "label_mismatch": int((hlab != ex16).sum().item()),
                            "speedup_vs_fp32_exact": query_ms / hms}
    del hlab, ex16
    sur, train_s = None, None
    if args.surrogate_train > 0:
        sur = fk.surrogate_create(chain, seed=rank + 1)
        qtr = torch.from_numpy(synth.uniform_configs(w.seed + 7, args.surrogate_train, arm.D, arm.qlim)).to(dev)
        t0 = time.perf_counter()
        sst = fk.surrogate_train(sur, model, qtr, epochs=args.surrogate_epochs, batch=8192,
                                 lr=args.surrogate_lr, holdout=0.0625, schedule=fk.FK_LR_COSINE)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del qtr
        slab = torch.empty(nq, dtype=torch.int8, device=dev)
        ex = torch.empty(nq, dtype=torch.int8, device=dev)
        fk.fk_score(model, Q, ex, rescore=True)
        nfb = fk.surrogate_infer(sur, model, Q, slab)
        times_s = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fk.surrogate_infer(sur, model, Q, slab)
            b.record()
            b.synchronize()
            times_s.append(a.elapsed_time(b))
        sms = statistics.median(times_s)
        mism = int((slab != ex).sum().item())
        paths["surrogate"] = {"checks_per_s": nq / (sms * 1e-3), "ms": sms, "fallback": nfb / nq,
                              "label_mismatch": mism, "label_mismatch_rate": mism / nq,
                              "tau": sst["tau"], "holdout_fallback": sst["holdout_fallback"],
                              "holdout_sign_error": sst["holdout_sign_error"], "train_s": train_s,
                              "train_rows": sst["n_train"], "epochs": args.surrogate_epochs,
                              "lr_schedule": f"cosine from {args.surrogate_lr:g}",
                              "loss_last": sst["loss_last"], "speedup_vs_fp32_exact": query_ms / sms}
        del slab, ex
    metric = None
    try:
        if args.metric_queries > 0:
            metric = metric_paths(fk, dev, chain, model, sur, w, args.metric_queries, flush, train_s)
    finally:
        if sur is not None:
            fk.surrogate_destroy(sur)

    # many scenes: one persistent graph-captured launch (tuned) against one
    # fk_score call per scene, same queries, same exact labels
    batched = None
    if args.batch_scenes > 0:
        scenes = synth.batch_scenes(100 + rank, args.batch_scenes)
        bchains, bmodels = [], []
        for sc in scenes:
            ch = fk.chain_from_arm(sc.scene.arm)
            m = fk.fastron_model_create(ch)
            fk.fastron_model_set(m, sc.support.astype(np.float64), sc.alpha, sc.gamma)
            bchains.append(ch)
            bmodels.append(m)
        bb = fk.fk_batch_create(bmodels)
        try:
            off = np.concatenate([[0], np.cumsum([len(sc.queries) for sc in scenes])]).astype(np.int64)
            bq = torch.from_numpy(np.concatenate([sc.queries for sc in scenes])).to(dev)
            btot = int(off[-1])
            blab = torch.empty(btot, dtype=torch.int8, device=dev)
            best, tms = fk.fk_batch_tune(bb, bq, off, blab)
            fk.fk_score_batched(bb, bq, off, blab)
            def timed(fn, reps=5):
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    fn()
                    b.record()
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                return statistics.median(ts)
            t_batch = timed(lambda: fk.fk_score_batched(bb, bq, off, blab))
            plab = torch.empty(btot, dtype=torch.int8, device=dev)
            views = [(bq[off[i]:off[i + 1]], plab[off[i]:off[i + 1]]) for i in range(len(scenes))]
            def per_scene():
                for m, (qv, lv) in zip(bmodels, views):
                    if qv.shape[0]:
                        fk.fk_score(m, qv, lv, rescore=True)
            per_scene()
            t_per = timed(per_scene)
            same = bool(torch.equal(blab, plab))
            evals_b = sum(len(sc.support) * len(sc.queries) for sc in scenes) * Mv
            batched = {"scenes": len(scenes), "queries": btot, "support_min": min(len(sc.support) for sc in scenes),
                       "support_max": max(len(sc.support) for sc in scenes), "ms_persistent_graph": t_batch,
                       "ms_per_scene_launches": t_per, "speedup": t_per / t_batch,
                       "checks_per_s": btot / (t_batch * 1e-3), "teval_per_s": evals_b / (t_batch * 1e-3) / 1e12,
                       "tuned_variant": best, "variant_ms": [float(x) for x in tms[:6]], "labels_identical": same}
        finally:
            fk.fk_batch_destroy(bb)
            for m in bmodels:
                fk.fastron_model_destroy(m)
            for ch in bchains:
                fk.fk_chain_destroy(ch)

    small = small_3dof(fk, dev, rank, flush) if args.small else None

    gauss = None
    if args.gauss:
        gauss = gaussian_summand(fk, dev, rank, Q, Xq32, X, flush, peak)

    sweep = None
    counts = [int(x) for x in args.obstacle_sweep.split(",") if x.strip() and int(x) > 0]
    if counts:
        sweep = obstacle_sweep(fk, dev, rank, counts, Q, Xq32, X, flush)

    dynamic = None
    if args.dynamic_frames > 1:
        dynamic = changing_environment(fk, dev, rank, args.dynamic_frames, args.dynamic_queries,
                                       [m.strip() for m in args.dynamic_modes.split(",") if m.strip()],
                                       short=args.dynamic_frames_short)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_cpu_baseline(w, args.cpu_sample, os.cpu_count() or 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 score; double-float then f64 band re-score; f64 training (double-float kernel matrix)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dof": arm.D, "control_points": arm.M, "boxes": len(w.scene.boxes),
                       "n_train": w.n_train, "n_query": nq, "gamma": w.gamma,
                       "support": st["n_support"], "iterations": st["iterations"],
                       "l2": "flushed before every query pass (512 MiB write)", "path": "fp32+df+fp64-rescore",
                       "pipeline": "update of step s (priority stream) overlapped with the query pass of step "
                                   "s-1; two models alternate",
                       "pipelined_labels_equal_sequential": pipelined_equal,
                       "e2e_labels_equal_sequential": e2e_equal,
                       "headline": "value is the exact FP32 step (labels equal the FP64 oracle's); the "
                                   "half2 and surrogate paths the metric compares are in metric_paths"},
            "phases_ms": {"update": update_ms, "query": query_ms, "score_fp32": score_only_ms,
                          "rescored_queries": nres},
            "query_only_checks_per_s": nq / (query_ms * 1e-3),
            "query_paths": paths,
            "metric_paths": metric,
            "labels_checksum": checksum,
            "batched_scenes": batched,
            "changing_environment": dynamic,
            "obstacle_sweep": sweep,
            "gaussian_summand": gauss,
            "small_3dof": small,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Teval/s",
                         "frac": achieved / peak,
                         "peak_basis": "min(MUFU 16/clk/SM x 1 reciprocal, FP32 128/clk/SM / 5 ops) per evaluation "
                                       "x SMs x max SM clock",
                         "peak_fp32_floor": peak_fp32_floor, "frac_fp32_floor": achieved / peak_fp32_floor,
                         "traffic": SCORE_TRAFFIC_BYTES if SCORE_TRAFFIC_BYTES and nq == N_QUERY and Mv == 7 else None,
                         "kernel": "score_f32_kernel", "evals_per_launch": evals, "launch_ms": score_ms},
            "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                                         "score_us_per_query_1core")},
            "e2e": {"value": shard.aggregate_rate(nq, ws, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line))
    fk.fastron_model_destroy(model)
    fk.fk_chain_destroy(chain)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
