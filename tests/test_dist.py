"""bench.py's multi-process plumbing on CPU: two gloo ranks (no GPU).

Replicas only: the learner has no exchange step, so the only collectives are the
timing barrier and the max over ranks of the timed interval.  This runs both as
two spawned processes and checks that every rank sees the slowest rank's time and
that a rank that raises is reported as a failure, not a hang.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out, fail_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    if rank == fail_rank:
        dist.destroy_process_group()
        raise RuntimeError("rank failed on purpose (host-side failure)")
    bench.barrier(w)
    out[rank] = bench.max_over_ranks(times[rank], w)
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    times = [3.5, 7.25]
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, port, times, out, -1), nprocs=world, start_method="spawn",
                       join=True)
    assert [out[r] for r in range(world)] == [max(times)] * world


def test_a_failing_rank_is_reported():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    ctx = mp.start_processes(_rank_main, args=(world, port, [1.0, 2.0], out, 1), nprocs=world,
                             start_method="spawn", join=False)
    with pytest.raises(Exception):
        while not ctx.join(timeout=60):
            pass
    for p in ctx.processes:
        if p.is_alive():
            p.kill()
