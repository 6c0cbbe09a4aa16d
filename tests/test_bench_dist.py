"""Multi-rank logic of bench.py on the CPU (gloo, world size 2): the path runs
as independent replicas (no data-path collective), so what the ranks share is
the start barrier and the maximum of the per-rank step times, from which rank
0 reports the whole-job throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    ws, r, local = bench.dist_setup(None)
    try:
        bench.barrier(ws)
        step_ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
        worst = bench.max_over_ranks(step_ms, ws)
        value = ws * 2.0 * 1e9 / (worst * 1e-3) / 1e9  # whole-job GB/s of 1 GB fields, as run_ours reports
        q.put((r, ws, local, worst, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [x[0] for x in res] == [0, 1]
    for r, ws, local, worst, value in res:
        assert ws == 2 and local == r
        assert worst == 15.0  # the slowest rank's step time, on every rank
        assert abs(value - 2 * 2.0 / 0.015) < 1e-9
