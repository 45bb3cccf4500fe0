"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2): each rank estimates its own
data (disjoint seeds), the job time is the slowest rank's, the throughput counts every rank's
units.  No data-path collective exists: the estimator shards into independent map sets."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    tot = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(64 * 10, world, tot)
    seeds = bench.rank_seeds(rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    dist.barrier()
    out[rank] = (tot, rate, gathered)
    dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        tot, rate, gathered = res[r]
        assert tot == 150.0                              # max over ranks
        assert abs(rate - world * 640 / 0.150) < 1e-9    # all ranks' units / slowest time
        assert not set(gathered[0]) & set(gathered[1])   # disjoint data per rank


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(10, 1, 500.0) == 20.0
