"""Multi-rank behaviour on CPU (gloo, world size 2).

The page-crypto path shards by contiguous ranges of data units: rank r handles
units [r*U/W, (r+1)*U/W) with the unit numbering continuing from the first
unit of its range, and there is no exchange step.  Each rank here computes its
slice with the oracle; the gathered result must equal the single-rank result.
A rank that fails before the join is detected by the other rank's collective
timing out with an error (host-side failure detection, no GPU involved).
"""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist

    import oracle
    import workloads as w
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    du, units = 4096, 96
    data = w.seeded_bytes(31, w.STREAM_DATA, du * units)
    key = w.xts_key(31, 256)
    u0, u1 = units * rank // world, units * (rank + 1) // world
    mine = oracle.xts(key, 0, data[u0 * du:u1 * du], du, 1000 + u0, nthreads=1)
    parts = [torch.zeros(0, dtype=torch.uint8)] * world
    dist.all_gather_object(parts, torch.from_numpy(mine))
    if rank == 0:
        whole = np.concatenate([p.numpy() for p in parts])
        np.save(out_path, whole)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_xts_equals_whole(tmp_path):
    import oracle
    import workloads as w
    out = str(tmp_path / "whole.npy")
    mp.start_processes(_shard_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    data = w.seeded_bytes(31, w.STREAM_DATA, 4096 * 96)
    ref = oracle.xts(w.xts_key(31, 256), 0, data, 4096, 1000)
    assert np.array_equal(got, ref)


def _failing_worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise SystemExit(3)  # this rank dies before the join
    t = torch.ones(4)
    try:
        dist.all_reduce(t)
        open(out_path, "w").write("completed")
    except Exception as e:  # the survivor sees the failure as an error, not a hang
        open(out_path, "w").write("detected: " + type(e).__name__)


def test_dead_rank_is_detected_by_the_survivor(tmp_path):
    out = str(tmp_path / "survivor.txt")
    ctx = mp.start_processes(_failing_worker, args=(2, _free_port(), out), nprocs=2, join=False,
                             start_method="spawn")
    for p in ctx.processes:
        p.join(120)
    assert all(p.exitcode is not None for p in ctx.processes), "a rank hung"
    assert open(out).read().startswith("detected")
