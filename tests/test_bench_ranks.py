"""The multi-rank logic of bench.py on CPU: two gloo ranks, the timed
region reduced to its maximum over ranks, and the whole-job throughput
counting the updates of every replica."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + rank, dist)          # rank 1 is the slowest
    glups = bench.whole_job_glups(1000, 50, world, ms * 1e-3)
    out.put((rank, ms, glups))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, glups in res:
        assert ms == 11.0
        assert glups == pytest.approx(1000 * 50 * 2 / 11e-3 / 1e9)


def test_single_rank_without_group():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_glups(10, 2, 1, 1.0) == pytest.approx(2e-8)
