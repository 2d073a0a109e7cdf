"""The N > 1 path of the benchmark on the CPU: replicas only, so the one
collective is the maximum of the ranks' times (gloo, world size 2), and
each rank's inputs are its own seeded replica of the workload."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from paper_1812_03689_gb300 import inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 10 solves
        value, slow = bench.job_rate(1.0 + rank, 10, world, device="cpu")
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"value": value, "slow": slow}, f)
    finally:
        dist.destroy_process_group()


def test_job_rate_one_rank():
    value, slow = bench.job_rate(2.0, 10, 1)
    assert slow == 2.0 and value == 5.0


def test_job_rate_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for g in got:
        # the slowest rank's time; all ranks' solves over it
        assert g["slow"] == 2.0
        assert g["value"] == world * 10 / 2.0


def test_replicas_are_seeded_and_distinct():
    w = inputs.workload("c1_small")
    a0 = w.particles(request_index=0)
    a0b = w.particles(request_index=0)
    a1 = w.particles(request_index=1)
    for u, v in zip(a0, a0b):
        assert np.array_equal(u, v)
    assert not np.array_equal(a0[0], a1[0])
    assert len(a0[0]) == len(a1[0])


def test_dist_env(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (1, 2, 1)
