"""fk_score_noalloc: the scoring entry point for callers that cannot allocate
device memory while they run (for example a planner loop that must never wait
on the allocator).  It must give the same labels and scores as fk_score, call
after call, although all its calls share one static scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_QUERIES = 1 << 20


@pytest.fixture(scope="module")
def trained(fk):
    # the FP64 oracle's model of the 7-DOF workload (Algorithm 1 on the
    # checker's labels), loaded into the library with fastron_model_set
    dev = torch.device("cuda:0")
    w = synth.workload("arm7-n5000")
    X = w.train_configs().astype(np.float64)
    r = O.fastron_train(O.fk_points(w.scene.arm, X), O.check(w.scene, X), w.gamma, w.beta, w.iter_max, w.s_max)
    S, alpha = X[r.support], r.alpha[r.support]
    chain = fk.chain_from_arm(w.scene.arm)
    model = fk.fastron_model_create(chain)
    fk.fastron_model_set(model, S, alpha, w.gamma)
    yield w, model, dev, float(np.sum(np.abs(alpha))), (S, alpha)
    fk.fastron_model_destroy(model)
    fk.fk_chain_destroy(chain)


def _both(fk, model, q):
    n = q.shape[0]
    f_ref = torch.empty(n, dtype=torch.float32, device=q.device)
    l_ref = torch.empty(n, dtype=torch.int8, device=q.device)
    n_ref = fk.fk_score(model, q, l_ref, f_ref, rescore=True, count=True)
    f_na = torch.full((n,), float("nan"), dtype=torch.float32, device=q.device)
    l_na = torch.zeros(n, dtype=torch.int8, device=q.device)
    n_na = fk.fk_score_noalloc(model, q, l_na, f_na, count=True)
    torch.cuda.synchronize()
    return f_ref.cpu().numpy(), l_ref.cpu().numpy(), n_ref, f_na.cpu().numpy(), l_na.cpu().numpy(), n_na


def test_noalloc_matches_fk_score_on_consecutive_calls(fk, trained):
    w, model, dev, sum_alpha, (S, alpha) = trained
    Q = w.query_configs(1 << 19)
    # two calls in a row: a large batch, then a different, smaller one, so a
    # band list left over from the first call would show up in the second
    for q in (Q[: 1 << 19], Q[1000:1000 + 70001]):
        tq = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
        f_ref, l_ref, n_ref, f_na, l_na, n_na = _both(fk, model, tq)
        assert n_na == n_ref and n_ref > 0
        assert np.array_equal(l_na, l_ref)
        np.testing.assert_allclose(f_na, f_ref, rtol=0, atol=1e-4 * sum_alpha)
        # and the labels are the oracle's (the sign of the FP64 model value)
        want = O.score(w.scene.arm, S, alpha, q.astype(np.float64), w.gamma, nthreads=os.cpu_count() or 1)
        assert np.array_equal(l_na, O.labels_from_f(want))


def test_noalloc_reports_a_tile_wait_timeout(fk, trained):
    # a tile wait that gives up at once is reported whether or not the
    # caller asks for the band count (the call reads its error word back
    # every time); the next call with the normal limit is correct again
    w, model, dev, sum_alpha, _ = trained
    tq = torch.from_numpy(w.query_configs(4096)).to(dev)
    lab = torch.empty(4096, dtype=torch.int8, device=dev)
    fk.fk_set_wait_limit(0)
    try:
        for count in (False, True):
            with pytest.raises(fk.FkError) as e:
                fk.fk_score_noalloc(model, tq, lab, count=count)
            assert e.value.code == fk.FK_ERR_TIMEOUT
    finally:
        fk.fk_set_wait_limit(1 << 22)
    f_ref, l_ref, n_ref, f_na, l_na, n_na = _both(fk, model, tq)
    assert n_na == n_ref and np.array_equal(l_na, l_ref)


def test_noalloc_rejects_batches_above_its_scratch(fk, trained):
    w, model, dev, _, _ = trained
    q = torch.zeros((MAX_QUERIES + 1, w.scene.arm.D), dtype=torch.float32, device=dev)
    lab = torch.empty(MAX_QUERIES + 1, dtype=torch.int8, device=dev)
    with pytest.raises(fk.FkError) as e:
        fk.fk_score_noalloc(model, q, lab)
    assert e.value.code == fk.FK_ERR_CAPACITY and "scratch" in str(e.value)
    # the largest allowed batch still works
    q = torch.from_numpy(w.query_configs(MAX_QUERIES)).to(dev)
    lab = torch.empty(MAX_QUERIES, dtype=torch.int8, device=dev)
    fk.fk_score_noalloc(model, q, lab, count=True)
