"""Host logic of bench.py's multi-rank run, on CPU with two gloo ranks: the job time is
the slowest rank's (max over ranks), the rate counts every rank's units, and under the
reference arm only rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]                      # this rank's time for the timed steps
        m = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.whole_job_rate(1000, 4, world, m / 1e3)
        q.put((rank, m, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, rate in got:
        assert m == 17.25                               # the slowest rank's time on every rank
        assert rate == pytest.approx(1000 * 4 * 2 / 17.25e-3)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.whole_job_rate(10, 2, 1, 0.5) == 40.0


def test_reference_arm_other_ranks_print_nothing(capsys):
    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A(), rank=1)
    assert capsys.readouterr().out == ""
