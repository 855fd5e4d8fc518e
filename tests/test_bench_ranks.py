"""Host logic of the multi-process benchmark, on CPU: two gloo ranks agree on the
slowest rank's timings (the step time of a weak-scaling job) and the whole-job
throughput counts the samples of every rank; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r is slower in the forward, rank 0 in the adjoint
        mine = [10.0 + rank, 4.0 + 2.0 * rank, 6.0 - rank]
        got = bench.max_over_ranks(mine, dist, "cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, world = _free_port(), 2
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(world))
    assert res[0] == res[1] == [11.0, 6.0, 6.0]


def test_single_rank_and_whole_job_value():
    import bench
    assert bench.max_over_ranks([3.0, 1.0], None, "cpu") == [3.0, 1.0]
    # 36.1 G samples per rank and step, 2 ranks, slowest rank 51.3 ms
    assert bench.whole_job_value(36.1e9, 2, 51.3) == pytest.approx(2 * 36.1e9 / 0.0513 / 1e9)
    assert bench.whole_job_value(36.1e9, 1, 51.3) == pytest.approx(36.1e9 / 0.0513 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    def no_work(*a, **k):
        raise AssertionError("a non-zero rank must not run the CPU checker")

    monkeypatch.setattr(bench, "cpu_reference", no_work)
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(None) == 0
    assert capsys.readouterr().out == ""
