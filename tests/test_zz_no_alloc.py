"""fk_score_noalloc: the scoring entry point for callers that cannot allocate
device memory while they run (for example a planner loop that must never wait
on the allocator).  It must give the same labels and scores as fk_score, call
after call, although all its calls share one static scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest
import torch

from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_QUERIES = 1 << 20


@pytest.fixture(scope="module")
def trained(fk):
    dev = torch.device("cuda:0")
    w = synth.workload("arm7-n5000")
    chain = fk.chain_from_arm(w.scene.arm)
    model = fk.fastron_model_create(chain)
    X = w.train_configs()
    y = torch.empty(w.n_train, dtype=torch.int8, device=dev)
    fk.fk_label(chain, w.scene.boxes, w.scene.radius, torch.from_numpy(X).to(dev), y)
    fk.fastron_train(model, torch.from_numpy(X.astype(np.float64)).to(dev), y, w.gamma, w.beta, w.iter_max, w.s_max)
    _, alpha = fk.fastron_model_get(model)
    yield w, model, dev, float(np.sum(np.abs(alpha)))
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
    w, model, dev, sum_alpha = trained
    Q = w.query_configs(1 << 19)
    # two calls in a row: a large batch, then a different, smaller one, so a
    # band list left over from the first call would show up in the second
    for q in (Q[: 1 << 19], Q[1000:1000 + 70001]):
        tq = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
        f_ref, l_ref, n_ref, f_na, l_na, n_na = _both(fk, model, tq)
        assert n_na == n_ref and n_ref > 0
        assert np.array_equal(l_na, l_ref)
        np.testing.assert_allclose(f_na, f_ref, rtol=0, atol=1e-4 * sum_alpha)


def test_noalloc_rejects_batches_above_its_scratch(fk, trained):
    w, model, dev, _ = trained
    q = torch.zeros((MAX_QUERIES + 1, w.scene.arm.D), dtype=torch.float32, device=dev)
    lab = torch.empty(MAX_QUERIES + 1, dtype=torch.int8, device=dev)
    with pytest.raises(fk.FkError) as e:
        fk.fk_score_noalloc(model, q, lab)
    assert e.value.code == fk.FK_ERR_CAPACITY and "scratch" in str(e.value)
    # the largest allowed batch still works
    q = torch.from_numpy(w.query_configs(MAX_QUERIES)).to(dev)
    lab = torch.empty(MAX_QUERIES, dtype=torch.int8, device=dev)
    fk.fk_score_noalloc(model, q, lab, count=True)
