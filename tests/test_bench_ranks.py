"""The bench's multi-rank host logic on CPU (gloo, world size 2): every rank gets the slowest
rank's step time, the whole-job rate counts every replica, and the reference arm runs on
rank 0 only.  No GPU is needed: the collectives run on CPU tensors."""
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
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        out[rank] = ms
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_whole_job_rate_and_single_rank():
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    one = bench.whole_job_rate(1, 4097 ** 2, 53, 20.0)
    assert bench.whole_job_rate(2, 4097 ** 2, 53, 20.0) == pytest.approx(2 * one)
    assert one == pytest.approx(4097 ** 2 * 53 / 0.02)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        N, kappa, shape, steps, warmup, gpus = 4096, 1.0, "flower", 1, 3, 2
    assert bench.run_reference(A()) == 0     # returns at once, without work or output
