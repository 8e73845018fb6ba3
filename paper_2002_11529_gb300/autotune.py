"""Autotuner for the batched form's launch shape.

Sweeps tracks per warp {1, 2, 4, 8} and block size {128, 256, 512}, plus,
at 8 tracks per warp, large blocks of one per SM: 640, 768, 800 threads and
the block whose warps cover the batch's median event in one round of warp
calls (32 x ceil(median tracks / 8) threads, when above 512 and at most
800).  The per-event shared-memory tile of hit x stays at 8192 hits.  Each
shape runs on the caller's batch (device resident), timed with CUDA events
over several passes (L2 flushed before each pass); the fastest
LaunchConfig is returned with the table.
Results can be cached in a JSON file keyed by the batch's shape.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

import torch

from . import LaunchConfig

TRACKS_PER_WARP = (1, 2, 4, 8)
BLOCKS = (128, 256, 512)
X_CAPS = (8192,)
LARGE_BLOCKS = (640, 768, 800)   # tracks_per_warp 8 only
LARGE_BLOCK_MAX = 800


def round_block(pipe) -> int | None:
    """Threads of a block whose warps (8 tracks each) cover the median
    event's tracks in one round, if that is a large block."""
    per_event = torch.diff(pipe.velo.trk_off.to("cpu", torch.int64))
    if per_event.numel() == 0:
        return None
    med = int(per_event.median())
    block = 32 * max(1, -(-med // 8))
    return block if 512 < block <= LARGE_BLOCK_MAX else None


def candidates(pipe) -> list:
    """Launch shapes the autotuner times for this batch."""
    cfgs = [LaunchConfig(t, b, x) for t, b, x in itertools.product(TRACKS_PER_WARP, BLOCKS, X_CAPS)]
    large = set(LARGE_BLOCKS)
    rb = round_block(pipe)
    if rb is not None:
        large.add(rb)
    cfgs += [LaunchConfig(8, b, x) for b in sorted(large) for x in X_CAPS]
    return cfgs


def shape_key(pipe) -> str:
    hits = int(pipe.ev_off.numel())
    return f"E{pipe.n_events}_T{pipe.velo.n_tracks}_W{pipe.n_words}_S{pipe.ctx.geom.n_sectors}_{hits}"


def time_config(pipe, cfg, reps=5, flush=None, stream=None):
    stream = stream or torch.cuda.current_stream()
    pipe.run_batched(cfg, stream)
    ms = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pipe.run_batched(cfg, stream)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def autotune(pipe, reps=5, cache_path=None, flush=None, configs=None):
    """Return (best LaunchConfig, [(cfg, ms), ...])."""
    key = shape_key(pipe)
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return LaunchConfig(**cache[key]["best"]), [(LaunchConfig(**c), m) for c, m in cache[key]["table"]]
    if configs is None:
        configs = candidates(pipe)
    table = []
    for cfg in configs:
        table.append((cfg, time_config(pipe, cfg, reps, flush)))
    pipe.ctx.check(what="autotune")
    best = min(table, key=lambda r: r[1])[0]
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[key] = {"best": best.__dict__, "table": [(c.__dict__, m) for c, m in table]}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, table
