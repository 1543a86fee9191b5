"""Host-side logic of the multi-GPU run, with two gloo processes on CPU: each
rank gets its own scene, the ranks share nothing but the max of their step
times, and the reported rate is the whole job's."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1910_06451_gb300 import shard, synth


def test_contiguous_ranges_cover_everything_once():
    for n in (0, 1, 7, 100, 4_194_304):
        for ws in (1, 2, 3, 8):
            got = [shard.contiguous_range(n, r, ws) for r in range(ws)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[r][1] == got[r + 1][0] for r in range(ws - 1))
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1


def test_single_process_is_the_identity():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.aggregate_rate(1000, 1, 2.0) == pytest.approx(5e5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = shard.world()
        w = synth.workload("arm7-n5000", trial=shard.rank_trial(got_rank))
        my_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        worst = shard.max_over_ranks(my_ms)
        out[rank] = (got_ws, got_rank, w.seed, worst, shard.aggregate_rate(1000, got_ws, worst))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_scene_and_take_the_max_time():
    ws = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    seeds = {res[r][2] for r in res}
    assert len(seeds) == 2  # a different scene per rank
    for r in res:
        assert res[r][0] == ws and res[r][1] == r
        assert res[r][3] == 15.0  # every rank sees the slowest time
        assert res[r][4] == pytest.approx(2 * 1000 / 15e-3)
