"""The N > 1 launch of bench.py on the CPU: world_size-2 gloo process groups (127.0.0.1) stand in for the
one-process-per-GPU torchrun launch.  Every rank runs its own replica (no data-path collective); the job's time is
the slowest rank's (max over ranks) and its value the units of all ranks over that time; the reference arm runs on
rank 0 alone and the other ranks return without work."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]          # the second rank is the slower one
    dist.barrier()
    total = bench.max_over_ranks(local_ms)
    value = bench.job_value(world, 10, 50, total)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"total": total, "value": value}, f)


def test_max_over_ranks_and_job_value_with_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["total"] == 150.0                      # the slowest rank's time, seen by every rank
        assert r["value"] == pytest.approx(2 * 10 * 50 / 0.150)


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 4, 50, 100.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
