"""The benchmark's multi-process path on CPU: world size 2 over gloo.

Every rank advances its own replica of the chip (the chips exchange no
data), so the only collective is the reduction of the timings: the
whole-job figure is all ranks' units over the slowest rank's time.
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 3.0][rank]          # rank 1 is the slow one
    slowest = bench.reduce_max(seconds, world)
    glups = bench.aggregate_glups(1e9, seconds, world)
    dist.barrier()
    out[rank] = (slowest, glups)
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(2):
        slowest, glups = res[r]
        assert slowest == 3.0
        assert abs(glups - 2 * 1e9 / 3.0 / 1e9) < 1e-12


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(1.5, 1) == 1.5
    assert bench.aggregate_glups(3e9, 1.5, 1) == pytest.approx(2.0)
