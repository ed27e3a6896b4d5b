"""The benchmark's multi-rank path (independent replicas, one per GPU): the
job's time is the slowest rank's, taken by an all-reduce MAX; checked with
two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, w, "cpu")
    out[rank] = (r, w, loc, ms, bench.job_seconds_per_compression(ms, 4, w))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_ranks_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
        got = dict(out)
    for rank in range(world):
        r, w, loc, ms, v = got[rank]
        assert (r, w, loc) == (rank, world, rank)
        assert ms == 150.0                      # max over ranks
        assert v == 150.0 / 1e3 / (4 * world)   # all ranks' compressions in that time


def test_single_rank_is_its_own_clock():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_seconds_per_compression(1000.0, 5, 1) == 0.2
