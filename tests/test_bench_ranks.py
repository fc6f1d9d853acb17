"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.

Each GPU runs an independent replica (the lattice does not shard), so the
only cross-rank steps are the barrier and the max of the timed regions;
the job's throughput counts every rank's node updates over the slowest
rank's time.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        ms = bench._max_over_ranks(10.0 + 3.0 * rank, ws, "cpu")  # rank 1 is the slow one
        out[rank] = (ms, bench._job_mlups(ws, 1000, 50, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 13.0
    # 2 ranks x 1000 nodes x 50 steps in 13 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 50 / 13e-3 / 1e6)


def test_one_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench._job_mlups(1, 4096 * 4096, 200, 46.2) == pytest.approx(4096 * 4096 * 200 / 46.2e-3 / 1e6)
