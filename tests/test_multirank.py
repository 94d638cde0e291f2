"""The N > 1 path of bench.py (one independent replica per GPU, "replicas
only": no data-path collective) on CPU ranks with the gloo backend: the job
time is the slowest rank's (max over ranks), whole-job throughput counts the
samples of every rank, and under torchrun the comparison arm runs on rank 0
only."""
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


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [10.0, 25.0, 17.5][rank]
        m = bench._max_over_ranks(ms, world, "cpu")
        v = bench._job_throughput(1 << 28, 50, m, world)
        out.put((rank, m, v))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_job_throughput_on_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(world, _free_port(), q), nprocs=world, join=True, start_method="spawn")
    res = sorted(q.get() for _ in range(world))
    slowest = max([10.0, 25.0, 17.5][:world])
    for rank, m, v in res:
        assert m == slowest
        assert v == pytest.approx(world * (1 << 28) * 50 / (slowest / 1e3) / 1e9)


def test_single_rank_needs_no_process_group():
    assert bench._max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench._job_throughput(1000, 4, 2.0, 1) == pytest.approx(1000 * 4 / 2e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "3", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""
