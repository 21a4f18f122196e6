"""The multi-rank bench path on CPU: two gloo ranks, each timing its own shot,
reduce to the slowest rank's time; the whole-job rate counts every rank's work.
The reference arm runs on rank 0 only; other ranks leave without work."""

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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 10.0 + 5.0 * rank                      # rank 1 is the slowest
    slowest = bench.reduce_max(mine)
    rate = bench.whole_job_rate(1000.0, world, slowest)
    out.put((rank, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_and_whole_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in res:
        assert slowest == 15.0
        assert rate == pytest.approx(2 * 1000.0 / 15.0)


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:  # the reference arm needs only these fields before it returns
        impl, steps, warmup, workload, so, nt = "reference", 1, 0, "acoustic256", None, None
    assert bench.run_reference(A()) == 0
