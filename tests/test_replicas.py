"""The multi-GPU path of the benchmark is replicas only: every rank runs its own ensemble from its
own seed, and the ranks meet once, at the end, to take the maximum time and the total work. Checked
here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

import bench                              # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 3.0 - rank]          # (step time, e2e time) of this rank
        work = [1000.0 * (rank + 1)]               # particles of this rank's replica
        mx, sm = bench.combine_ranks(dist, times, work, "cpu")
        out[rank] = (mx, sm, bench.replica_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_replicas_combine_by_max_time_and_total_work():
    port = _free_port()
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, sm, seed = res[r]
        assert mx == [11.0, 3.0]                   # the slowest rank sets the job's times
        assert sm == [3000.0]                      # the work of both replicas
    assert res[0][2] != res[1][2]                  # independent seeds


def test_single_rank_passes_through():
    mx, sm = bench.combine_ranks(None, [5.0, 2.0], [7.0], "cpu")
    assert mx == [5.0, 2.0] and sm == [7.0]
