"""The multi-rank logic of bench.py on CPU: two gloo ranks, each a replica
of the timed job.  The job's time is the slowest rank's, its throughput the
units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.dist_init("gloo")
    bench.barrier(w)
    ms = 10.0 * (r + 1)            # rank 1 is the slow one
    units = 1000.0 * (r + 1)
    tmax = bench.max_over_ranks(ms, w)
    tot = bench.sum_over_ranks(units, w)
    q.put((r, w, tmax, tot, tot / (tmax / 1000.0)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, tmax, tot, val in out:
        assert w == 2 and tmax == 20.0 and tot == 3000.0 and val == 150000.0


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
