"""Many scenes in one persistent launch: labels equal those of per-scene
fk_score calls and of the FP64 oracle, f within the FP32 bound, for uneven
scenes including empty query batches and single support points; every
autotuner variant gives the same labels."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1910_06451_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch(fk):
    scenes = synth.batch_scenes(7, 9, support=(1, 700), queries=(1, 3000))
    scenes[2].queries = scenes[2].queries[:0]       # a scene without queries
    scenes[4].support = scenes[4].support[:1]       # a single support point
    scenes[4].alpha = scenes[4].alpha[:1]
    chains, models = [], []
    for sc in scenes:
        ch = fk.chain_from_arm(sc.scene.arm)
        m = fk.fastron_model_create(ch)
        fk.fastron_model_set(m, sc.support.astype(np.float64), sc.alpha, sc.gamma)
        chains.append(ch)
        models.append(m)
    b = fk.fk_batch_create(models)
    off = np.concatenate([[0], np.cumsum([len(sc.queries) for sc in scenes])]).astype(np.int64)
    q = torch.from_numpy(np.concatenate([sc.queries for sc in scenes])).cuda()
    yield scenes, models, b, off, q
    fk.fk_batch_destroy(b)
    for m in models:
        fk.fastron_model_destroy(m)
    for ch in chains:
        fk.fk_chain_destroy(ch)


def test_batched_matches_per_scene_and_oracle(fk, batch):
    scenes, models, b, off, q = batch
    total = int(off[-1])
    lab = torch.empty(total, dtype=torch.int8, device="cuda")
    f = torch.empty(total, dtype=torch.float32, device="cuda")
    fk.fk_score_batched(b, q, off, lab, f, count=True)
    # the second call replays the captured graph
    lab2 = torch.empty_like(lab)
    fk.fk_score_batched(b, q, off, lab2, f)
    torch.cuda.synchronize()
    lab, lab2, f = lab.cpu().numpy(), lab2.cpu().numpy(), f.cpu().numpy()
    for i, (sc, m) in enumerate(zip(scenes, models)):
        a, z = off[i], off[i + 1]
        if z == a:
            continue
        qi = q[a:z].contiguous()
        ref = torch.empty(z - a, dtype=torch.int8, device="cuda")
        fk.fk_score(m, qi, ref, rescore=True)
        want = O.score(sc.scene.arm, sc.support.astype(np.float64), sc.alpha, sc.queries.astype(np.float64),
                       sc.gamma, nthreads=8)
        B = O.score(sc.scene.arm, sc.support.astype(np.float64), np.abs(sc.alpha), sc.queries.astype(np.float64),
                    sc.gamma, nthreads=8)
        assert np.array_equal(lab[a:z], ref.cpu().numpy()), i
        assert np.array_equal(lab[a:z], O.labels_from_f(want)), i
        assert np.array_equal(lab2[a:z], lab[a:z])
        assert np.all(np.abs(f[a:z] - want) <= 3e-6 * B + 1e-30), i


def test_every_tuned_variant_agrees(fk, batch):
    scenes, models, b, off, q = batch
    total = int(off[-1])
    ref = torch.empty(total, dtype=torch.int8, device="cuda")
    fk.fk_score_batched(b, q, off, ref)
    tuned = torch.empty(total, dtype=torch.int8, device="cuda")
    best, ms = fk.fk_batch_tune(b, q, off, tuned)
    assert 0 <= best < 6 and np.all(ms[:6] > 0)
    # the tuner scores every variant into its label buffer in turn: the last
    # one (one query per thread, compiled for three CTAs per SM) is left there
    torch.cuda.synchronize()
    assert torch.equal(tuned, ref)
    lab = torch.empty(total, dtype=torch.int8, device="cuda")
    fk.fk_score_batched(b, q, off, lab)
    torch.cuda.synchronize()
    assert torch.equal(lab, ref)


def test_batched_band_reaches_fp64_for_cancelling_scene(fk):
    # one scene whose two support points coincide with weights +1 and -1
    # (f = 0 for every query) among ordinary scenes: inside the captured graph
    # its queries pass the FP32 band and the double-float tier to the FP64
    # re-score, which returns f = 0 and the label +1; the other scenes keep
    # their own labels
    scenes = synth.batch_scenes(11, 3, support=(50, 300), queries=(200, 800))
    x = scenes[1].support[:1]
    scenes[1].support = np.concatenate([x, x])
    scenes[1].alpha = np.array([1.0, -1.0])
    chains, models = [], []
    try:
        for sc in scenes:
            ch = fk.chain_from_arm(sc.scene.arm)
            m = fk.fastron_model_create(ch)
            fk.fastron_model_set(m, sc.support.astype(np.float64), sc.alpha, sc.gamma)
            chains.append(ch)
            models.append(m)
        b = fk.fk_batch_create(models)
        try:
            off = np.concatenate([[0], np.cumsum([len(sc.queries) for sc in scenes])]).astype(np.int64)
            q = torch.from_numpy(np.concatenate([sc.queries for sc in scenes])).cuda()
            lab = torch.zeros(int(off[-1]), dtype=torch.int8, device="cuda")
            f = torch.full((int(off[-1]),), 7.0, dtype=torch.float32, device="cuda")
            fk.fk_score_batched(b, q, off, lab, f)
            torch.cuda.synchronize()
            lab, f = lab.cpu().numpy(), f.cpu().numpy()
            a, z = off[1], off[2]
            assert np.all(f[a:z] == 0.0) and np.all(lab[a:z] == 1)
            for i in (0, 2):
                sc = scenes[i]
                want = O.score(sc.scene.arm, sc.support.astype(np.float64), sc.alpha,
                               sc.queries.astype(np.float64), sc.gamma, nthreads=8)
                assert np.array_equal(lab[off[i]:off[i + 1]], O.labels_from_f(want))
        finally:
            fk.fk_batch_destroy(b)
    finally:
        for m in models:
            fk.fastron_model_destroy(m)
        for ch in chains:
            fk.fk_chain_destroy(ch)


def test_batched_circle_form(fk):
    # every scene with at least 128 support points: each takes the circle form
    # of its first control point with its own cnorm; switched off, the same
    # batch takes the direct form; both give the oracle's labels
    scenes = synth.batch_scenes(11, 6, support=(128, 700), queries=(500, 3000))
    chains, models = [], []
    try:
        for sc in scenes:
            ch = fk.chain_from_arm(sc.scene.arm)
            m = fk.fastron_model_create(ch)
            fk.fastron_model_set(m, sc.support.astype(np.float64), sc.alpha, sc.gamma)
            chains.append(ch)
            models.append(m)
            assert fk.fk_score_circle(m) > 0
        off = np.concatenate([[0], np.cumsum([len(sc.queries) for sc in scenes])]).astype(np.int64)
        q = torch.from_numpy(np.concatenate([sc.queries for sc in scenes])).cuda()
        total = int(off[-1])
        out = {}
        for on in (True, False):
            fk.fk_set_circle_form(on)
            try:
                b = fk.fk_batch_create(models)
                try:
                    lab = torch.empty(total, dtype=torch.int8, device="cuda")
                    f = torch.empty(total, dtype=torch.float32, device="cuda")
                    fk.fk_score_batched(b, q, off, lab, f, count=True)
                    torch.cuda.synchronize()
                    out[on] = (lab.cpu().numpy(), f.cpu().numpy())
                finally:
                    fk.fk_batch_destroy(b)
            finally:
                fk.fk_set_circle_form(True)
        for i, sc in enumerate(scenes):
            a, z = off[i], off[i + 1]
            want = O.score(sc.scene.arm, sc.support.astype(np.float64), sc.alpha, sc.queries.astype(np.float64),
                           sc.gamma, nthreads=8)
            B = O.score(sc.scene.arm, sc.support.astype(np.float64), np.abs(sc.alpha), sc.queries.astype(np.float64),
                        sc.gamma, nthreads=8)
            for on in (True, False):
                lab, f = out[on]
                assert np.array_equal(lab[a:z], O.labels_from_f(want)), (i, on)
                assert np.all(np.abs(f[a:z] - want) <= 3e-6 * B + 1e-30), (i, on)
        assert not np.array_equal(out[True][1], out[False][1])  # the forms round differently
    finally:
        for m in models:
            fk.fastron_model_destroy(m)
        for ch in chains:
            fk.fk_chain_destroy(ch)
