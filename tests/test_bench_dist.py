"""The multi-rank host logic of bench.py (replicas, barrier, max over ranks) on CPU ranks
over gloo (world size 2): the job value divides the slowest rank's time by all solves."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, loc = bench.dist_setup()
    bench.barrier(w)
    t = 10.0 + 5.0 * r                       # per-rank timed region (ms)
    out[r] = (w, r, loc, bench.barrier_max(t, w))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    assert res[0][3] == res[1][3] == 15.0
    # bench.py reports whole-job ms per solve: max time / (steps * world)
    steps = 3
    assert res[0][3] / (steps * 2) == pytest.approx(2.5)
