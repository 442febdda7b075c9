"""The benchmark's multi-rank logic on CPU: two gloo ranks (127.0.0.1) reduce
their timings to the slowest rank, the whole-job throughput counts every
rank's replica, and the reference arm does its work on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 10 ms: every rank must see the slowest, 20 ms
    got = bench.max_over_ranks(torch, (rank + 1) * 10.0)
    env = bench.dist_env()
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"max": got, "env": list(env)}, fh)


def test_two_gloo_ranks_reduce_to_the_slowest(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.loads((tmp_path / f"rank{r}.json").read_text())
        assert d["max"] == 20.0
        assert d["env"] == [world, r, r]


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(torch, 3.5) == 3.5


def test_job_throughput_counts_every_replica():
    import bench
    # 2 GB per rank-step, 4 ranks, 10 steps in 1 s -> 80 GB/s
    assert bench.job_throughput(2e9, 4, 10, 1000.0) == pytest.approx(80.0)


def test_reference_arm_works_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--edge", "8",
                                      "--steps", "1", "--warmup", "0"])
    assert bench.reference_arm(bench.parse_args()) == 0
    assert capsys.readouterr().out == ""          # rank 1 prints nothing
    monkeypatch.setenv("RANK", "0")
    assert bench.reference_arm(bench.parse_args()) == 0
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
