"""fastron_model_copy: a snapshot of a trained model's support set for
scoring while the model itself trains again (the double buffer of a
pipelined changing-environment loop: Algorithm 1 for frame k + 1 on one
stream while frame k's queries are scored with frame k's model on another).

The snapshot must score exactly as its source did (same labels, same f, bit
for bit), must not change when the source is retrained, and the pipelined
loop must give every frame the labels of the sequential update-then-score
loop."""
import threading

import numpy as np
import pytest
import torch

from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu


def _scene(fk):
    w = synth.workload("arm7-n5000")
    ch = fk.chain_from_arm(w.scene.arm)
    dev = torch.device("cuda:0")
    X = torch.from_numpy(w.train_configs()[:2048].astype(np.float64)).to(dev)
    Q = torch.from_numpy(w.query_configs(1 << 16)).to(dev)
    return w, ch, dev, X, Q


def _score(fk, m, Q, stream=None):
    lab = torch.empty(Q.shape[0], dtype=torch.int8, device=Q.device)
    f = torch.empty(Q.shape[0], dtype=torch.float32, device=Q.device)
    fk.fk_score(m, Q, lab, f=f, rescore=True, stream=stream)
    return lab, f


def test_copy_scores_like_its_source_and_outlives_retraining(fk):
    w, ch, dev, X, Q = _scene(fk)
    m, snap = fk.fastron_model_create(ch), fk.fastron_model_create(ch)
    try:
        boxes = synth.moving_boxes(w.seed, w.scene.boxes, 2)
        y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
        fk.fk_label(ch, boxes[0], w.scene.radius, X.float(), y)
        fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max)
        lab0, f0 = _score(fk, m, Q)
        fk.fastron_model_copy(snap, m)
        lab1, f1 = _score(fk, snap, Q)
        torch.cuda.synchronize()
        assert torch.equal(lab0, lab1)
        assert torch.equal(f0.view(torch.int32), f1.view(torch.int32))
        i0, a0 = fk.fastron_model_get(m)
        i1, a1 = fk.fastron_model_get(snap)
        assert np.array_equal(i0, i1) and np.array_equal(a0, a1)
        # the source retrained on the next frame's labels: the snapshot keeps
        # the old model's labels, a new snapshot takes the new model's
        fk.fk_label(ch, boxes[1], w.scene.radius, X.float(), y)
        fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max)
        lab2, _ = _score(fk, snap, Q)
        labm, fm = _score(fk, m, Q)
        assert torch.equal(lab2, lab0)
        assert not torch.equal(labm, lab0)  # the boxes moved: some labels change
        fk.fastron_model_copy(snap, m)
        lab3, f3 = _score(fk, snap, Q)
        assert torch.equal(lab3, labm) and torch.equal(f3.view(torch.int32), fm.view(torch.int32))
    finally:
        fk.fastron_model_destroy(snap)
        fk.fastron_model_destroy(m)
        fk.fk_chain_destroy(ch)


def test_copy_rejects_bad_arguments(fk):
    w, ch, dev, X, Q = _scene(fk)
    w3 = synth.workload("arm3-n1000")
    ch3 = fk.chain_from_arm(w3.scene.arm)
    m, snap, other = fk.fastron_model_create(ch), fk.fastron_model_create(ch), fk.fastron_model_create(ch3)
    try:
        with pytest.raises(fk.FkError) as e:
            fk.fastron_model_copy(snap, m)  # m untrained
        assert e.value.code == fk.FK_ERR_STATE
        y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
        fk.fk_label(ch, w.scene.boxes, w.scene.radius, X.float(), y)
        fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max)
        with pytest.raises(fk.FkError) as e:
            fk.fastron_model_copy(m, m)
        assert e.value.code == fk.FK_ERR_ARG
        with pytest.raises(fk.FkError) as e:
            fk.fastron_model_copy(other, m)  # another chain
        assert e.value.code == fk.FK_ERR_ARG
    finally:
        for x in (other, snap, m):
            fk.fastron_model_destroy(x)
        fk.fk_chain_destroy(ch3)
        fk.fk_chain_destroy(ch)


def test_pipelined_update_and_query_give_the_sequential_labels(fk):
    # frames 1..F-1: Algorithm 1 for frame k on stream U (a host thread)
    # while frame k-1's queries are scored with its snapshot on stream S
    # (another thread); every frame's labels must equal those of the
    # sequential loop (update k, then score k)
    w, ch, dev, X, Q = _scene(fk)
    F = 5
    boxes = synth.moving_boxes(w.seed, w.scene.boxes, F)
    m = fk.fastron_model_create(ch)
    snaps = [fk.fastron_model_create(ch), fk.fastron_model_create(ch)]
    try:
        y = torch.empty(X.shape[0], dtype=torch.int8, device=dev)
        want = []
        for k in range(F):
            fk.fk_label(ch, boxes[k], w.scene.radius, X.float(), y)
            fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max, warm_start=k > 0)
            want.append(_score(fk, m, Q)[0])
        U = torch.cuda.Stream(priority=-1)
        S = torch.cuda.Stream(priority=0)
        got = [None] * F
        errors = []

        def update(k):
            try:
                with torch.cuda.stream(U):
                    fk.fk_label(ch, boxes[k], w.scene.radius, X.float(), y, stream=U)
                    fk.fastron_train(m, X, y, w.gamma, w.beta, w.iter_max, w.s_max, warm_start=k > 0, stream=U)
                    fk.fastron_model_copy(snaps[k % 2], m, stream=U)
                    U.synchronize()
            except Exception as e:  # reported by the main thread
                errors.append(e)

        def query(k):
            try:
                with torch.cuda.stream(S):
                    got[k] = _score(fk, snaps[k % 2], Q, stream=S)[0]
                    S.synchronize()
            except Exception as e:
                errors.append(e)

        update(0)
        for k in range(1, F):
            ta = threading.Thread(target=update, args=(k,))
            tb = threading.Thread(target=query, args=(k - 1,))
            ta.start()
            tb.start()
            ta.join()
            tb.join()
            assert not errors, errors
        query(F - 1)
        assert not errors, errors
        torch.cuda.synchronize()
        for k in range(F):
            assert torch.equal(got[k], want[k]), k
    finally:
        for x in snaps + [m]:
            fk.fastron_model_destroy(x)
        fk.fk_chain_destroy(ch)
