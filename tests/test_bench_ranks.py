"""The N > 1 logic of bench.py on CPU: world-size-2 gloo ranks agree on the
slowest rank's time, the whole-job value counts every rank's steps, and the
reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank_ms(100.0 * (rank + 1), world, "cpu")
        out[rank] = (ms, bench.job_throughput(world, 10, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, v = out[r]
        assert ms == 200.0
        assert v == pytest.approx(2 * 10 / 0.2)


def test_single_rank_value():
    assert bench.slowest_rank_ms(50.0, 1, "cpu") == 50.0
    assert bench.job_throughput(1, 100, 50.0) == pytest.approx(2000.0)


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    def no_oracle(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "run_oracle", no_oracle)
    args = type("A", (), {"steps": 3, "warmup": 1, "gpus": 2})()
    bench.reference_arm(args)
    assert capsys.readouterr().out == ""
