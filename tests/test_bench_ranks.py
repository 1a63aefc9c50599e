"""The benchmark's multi-rank host logic on CPU with the gloo backend (world size 2, two
processes on 127.0.0.1): the barrier lines the ranks up, the timing taken is the slowest rank's
(max over ranks) on every rank, and the whole-job throughput counts the units of all ranks over
that time. The GPU runs use the same functions over NCCL."""
import os
import socket
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(ws, sync_device=False)
    t0 = time.perf_counter()
    time.sleep(0.05 + 0.15 * rank)  # rank 1 is the slow one
    bench.barrier(ws, sync_device=False)
    mine = time.perf_counter() - t0
    slow = bench.max_over_ranks(0.05 + 0.15 * rank, ws, device="cpu")
    longest = bench.max_over_ranks(mine, ws, device="cpu")
    q.put((rank, mine, slow, longest, bench.whole_job_rate(1000.0, ws, slow)))
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo():
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, m0, s0, l0, v0), (_, m1, s1, l1, v1) = out
    # the barrier after the sleeps makes both ranks measure at least the slow rank's sleep
    assert m0 >= 0.2 - 0.01 and m1 >= 0.2 - 0.01
    assert s0 == s1 == pytest.approx(0.2)
    assert l0 == l1 == max(m0, m1)
    assert v0 == v1 == pytest.approx(2 * 1000.0 / 0.2)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
