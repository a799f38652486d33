"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

Every rank registers its own independent problem (weak scaling, no data-path
collective); the only collective is the max over ranks of the step times, and
the job's rate is all ranks' units over the slowest rank's time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]
        ms, e2e = bench.reduce_max(local, ws, "cpu")
        out.put((rank, ms, e2e, bench.rank_seed(2, rank), bench.job_throughput(1e9, ws, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_distinct_problems():
    import torch.multiprocessing as mp
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
    (r0, ms0, e0, s0, v0), (r1, ms1, e1, s1, v1) = res
    assert ms0 == ms1 == 15.0 and e0 == e1 == 20.0  # max over the ranks
    assert s0 != s1  # every rank registers its own pair
    assert v0 == v1 == pytest.approx(2 * 1e9 / 0.015)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.job_throughput(100.0, 1, 1000.0) == pytest.approx(100.0)
