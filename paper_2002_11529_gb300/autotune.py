"""Autotuner for the batched form's launch shape.

Sweeps tracks per warp {1, 2, 4, 8} and block size {128, 256, 512} (the
per-event shared-memory tile of hit x stays at 8192 hits) on the caller's
batch (device resident), times each with CUDA events over several passes
(L2 flushed before each pass), and returns the fastest LaunchConfig with
the table.
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
        configs = [LaunchConfig(t, b, x) for t, b, x in itertools.product(TRACKS_PER_WARP, BLOCKS, X_CAPS)]
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
