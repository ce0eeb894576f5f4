"""Host logic of bench.py's multi-GPU path on CPU: two gloo ranks agree on the slowest rank's
time (all-reduce MAX) and the whole-job rate counts every rank's steps; the reference arm returns
on ranks other than 0 without doing any work."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [1250.0, 1310.5][rank]
    out[rank] = bench.max_over_ranks(local_ms, world, "cpu")
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == 1310.5
    # 2 ranks x 3 steps in 1.3105 s of the slowest rank
    assert bench.whole_job_rate(world, 3, out[0]) == pytest.approx(6 / 1.3105)


def test_single_rank_is_its_own_max():
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.whole_job_rate(1, 5, 2000.0) == pytest.approx(2.5)


def test_reference_arm_other_ranks_exit(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    called = []
    monkeypatch.setattr(bench, "run_oracle_sample", lambda *a, **k: called.append(a))
    assert bench.main() == 0
    assert not called
