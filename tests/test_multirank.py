"""The bench's multi-rank host logic on CPU: two processes over gloo.

Events are independent, so every rank processes its own seeded batch (weak
scaling) with no data-path collective; the only collective is the max of
the per-rank times, and the job's throughput is world x events x steps over
that max.  The reference arm runs on rank 0 alone.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    b = bench.make_batch("tiny", rank, n_events=4)
    seconds = [0.5, 0.8][rank]
    worst = bench.max_over_ranks(seconds, dist, device="cpu")
    value = bench.job_events_per_s(world, b.n_events, 10, worst)
    digest = int(np.asarray(b.raw, np.uint64).sum() % (1 << 61))
    out[rank] = (worst, value, b.n_events, digest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_events_and_take_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    (w0, v0, e0, d0), (w1, v1, e1, d1) = res[0], res[1]
    assert w0 == w1 == 0.8                       # max over ranks, seen by every rank
    assert v0 == v1 == world * e0 * 10 / 0.8     # whole-job events/s
    assert e0 == e1 == 4 and d0 != d1            # same shape, different seeded events


def _ref_main(rank, world, port, out):
    import sys
    import types
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    calls = []
    bench.make_batch = lambda *a, **k: calls.append(a) or (_ for _ in ()).throw(RuntimeError("rank 0 only"))
    try:
        bench.run_reference(types.SimpleNamespace(workload="tiny", warmup=1, steps=1, gpus=world))
        out[rank] = ("returned", len(calls))
    except RuntimeError as e:
        out[rank] = (str(e), len(calls))


def test_reference_arm_runs_on_rank_zero_only():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_ref_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[1] == ("returned", 0)             # rank 1: no work
    assert res[0] == ("rank 0 only", 1)          # rank 0 starts the oracle run
