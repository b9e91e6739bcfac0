"""The N > 1 benchmark path on CPU: world size 2 over gloo (no GPU).

Queries are independent, so N GPUs run N replicas of the workload with no
data-path collective; the only communication is the barrier around the timed
region and the max over ranks of the step time, from which rank 0 reports the
whole-job throughput.  These tests run that host-side logic in two processes.
"""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = [120.0, 150.0][rank]            # the second rank is slower
        step_ms = bench.max_over_ranks(local_ms, dist)
        value = bench.job_throughput(2_000_000, world, step_ms)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"step_ms": step_ms, "value": value, "env": bench._dist()}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    for k in range(2):
        assert r[k]["step_ms"] == 150.0                              # max over ranks, on every rank
        assert r[k]["value"] == pytest.approx(2 * 2_000_000 / 0.150)   # whole-job queries/s
        assert r[k]["env"] == [2, k, k]


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.job_throughput(1000, 1, 500.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle; other ranks exit 0 with no work."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    import argparse
    ns = argparse.Namespace(impl="reference", workload="soup8", n_query=None, gpus=2, steps=1, warmup=1)
    assert bench.run_reference(ns) == 0
    assert capsys.readouterr().out == ""
