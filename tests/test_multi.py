"""The multi-process path on CPU: two gloo ranks (127.0.0.1) split work and form the job-level
throughput (all ranks' points over the slowest rank's time)."""
from __future__ import annotations

import os
import socket

import pytest

from paper_2008_06972_gb300 import multi

torch = pytest.importorskip("torch")


def test_shard_is_disjoint_and_complete():
    for world in (1, 2, 3, 8):
        parts = [multi.shard(64, r, world) for r in range(world)]
        flat = sorted(u for p in parts for u in p)
        assert flat == list(range(64))
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        multi.shard(4, 2, 2)


def test_job_value_without_a_group():
    v, sec, pts = multi.job_value(2e6, 0.5)
    assert (v, sec, pts) == (4.0, 0.5, 2e6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r encodes 1e6 * (r + 1) points in 0.1 * (r + 1) seconds
    v, sec, pts = multi.job_value(1e6 * (rank + 1), 0.1 * (rank + 1), dist, "cpu")
    out[rank] = (v, sec, pts, multi.shard(10, rank, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_form_the_job_value():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        v, sec, pts, units = out[r]
        assert abs(sec - 0.2) < 1e-12 and abs(pts - 3e6) < 1e-6
        assert abs(v - 3e6 / 0.2 / 1e6) < 1e-9
    assert sorted(out[0][3] + out[1][3]) == list(range(10))
