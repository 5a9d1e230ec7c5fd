"""The multi-GPU (replica) host logic of bench.py on two CPU ranks (gloo, 127.0.0.1).

The path does not shard across GPUs here: `bench.py --gpus N` runs N independent replicas of
the whole workload.  Its host logic is checked without a GPU: every rank must see the
slowest rank's step time, the job's value must count every rank's rows over that time, and
the reference arm must run on rank 0 only (the other ranks return without work or output).
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


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
        slow = bench.slowest_rank_ms(ms, dist, "cpu")
        value = bench.job_rows_per_s(1000, world, slow)
        queue.put((rank, slow, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time_and_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, queue)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(queue.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, slow, value in out:
        assert slow == pytest.approx(15.0)              # max over ranks, on every rank
        assert value == pytest.approx(2 * 1000 / 0.015)  # both ranks' rows over the job time


def test_single_rank_is_the_local_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5) == 12.5
    assert bench.job_rows_per_s(480, 1, 60.0) == pytest.approx(8000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, cpu_nside, eps, degree = 1, 0, 32, 1e-2, 2
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
