"""Host logic of the multi-process bench: on the GPU machine one process per GPU
(NCCL), here world size 2 over gloo on the CPU.  Every rank renders its own
replica; the job's time is its slowest rank's and its throughput counts the
frames of every rank.  The reference arm runs on rank 0 only."""
import socket
import types

import pytest
import torch.multiprocessing as mp

import bench
from _rank_worker import job_rate_worker


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=job_rate_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(queue.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, slowest, rate, env in res:
        assert slowest == 150.0
        assert rate == pytest.approx(8 * 2 / 0.150)
        assert env == (rank, 2, rank)


def test_single_process_rate_is_local():
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.job_rate(10, 250.0) == pytest.approx(40.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) is None     # returns at once: no oracle work, no output
