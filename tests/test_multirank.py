"""The benchmark's multi-rank path (replicas, one per GPU) on CPU: two gloo
ranks combine their timings as the max over ranks and their work as the sum
over ranks, exactly as bench.py does under torchrun with NCCL."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 20.0 - rank]          # ms: max over ranks
        work = [100 + rank, 7 * (rank + 1)]          # iterations: sum over ranks
        maxed, summed = bench.reduce_across_ranks(dist, torch, torch.device("cpu"), times, work)
        out[rank] = (maxed, summed)
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            maxed, summed = out[r]
            assert maxed == [11.0, 20.0]
            assert summed == [201.0, 21.0]


def test_single_process_is_identity():
    import bench
    maxed, summed = bench.reduce_across_ranks(dist, torch, torch.device("cpu"), [3.0], [4])
    assert maxed == [3.0] and summed == [4]
