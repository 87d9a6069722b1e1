"""The multi-rank path of bench.py on CPU (gloo, world size 2): the step time
is the maximum over ranks, throughput is the whole job's, and the reference
arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_init()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(10.0 + 5.0 * r, w)  # rank 1 is the slow one
        value = bench.job_throughput(1000, w, ms)
        ran = bench.run_reference(None, r, w) if r != 0 else "skipped"
        q.put((r, w, local, ms, value, ran))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, w, local, ms, value, ran in res:
        assert w == 2 and local == r
        assert ms == 15.0                 # both ranks see the slowest rank's time
        assert value == pytest.approx(2 * 1000 / 0.015)
    assert res[1][5] is None              # the reference arm does no work off rank 0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10, 1, 2.0) == pytest.approx(5000.0)
