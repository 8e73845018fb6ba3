"""Launch shapes the autotuner sweeps (host logic, CPU): the large block
sized so that one round of warp calls (8 tracks per warp) covers the median
event."""
import types

import numpy as np
import torch

from paper_2002_11529_gb300 import LaunchConfig, autotune


def fake_pipe(tracks_per_event):
    off = np.concatenate([[0], np.cumsum(np.asarray(tracks_per_event, np.int64))])
    return types.SimpleNamespace(velo=types.SimpleNamespace(trk_off=torch.tensor(off, dtype=torch.int32)))


def test_round_block_covers_the_median_event():
    assert autotune.round_block(fake_pipe([200] * 10)) == 800          # 25 warps x 8
    assert autotune.round_block(fake_pipe([150, 149, 160])) == 32 * 19  # ceil(150 / 8) warps
    assert autotune.round_block(fake_pipe([7, 200, 200, 5000, 200])) == 800
    assert autotune.round_block(fake_pipe([100] * 5)) is None          # 416 threads: not a large block
    assert autotune.round_block(fake_pipe([300] * 5)) is None          # beyond 800 threads
    assert autotune.round_block(fake_pipe([])) is None


def test_candidates():
    small = len(autotune.TRACKS_PER_WARP) * len(autotune.BLOCKS) * len(autotune.X_CAPS)
    c = autotune.candidates(fake_pipe([200] * 4))
    assert len(c) == small + len(autotune.LARGE_BLOCKS) and LaunchConfig(8, 800) in c
    c = autotune.candidates(fake_pipe([150] * 4))
    assert len(c) == small + len(autotune.LARGE_BLOCKS) + 1 and LaunchConfig(8, 608) in c
    for cfg in c:
        if cfg.block > 512:
            assert cfg.tracks_per_warp == 8 and cfg.block % 32 == 0 and cfg.block <= autotune.LARGE_BLOCK_MAX
        else:
            assert cfg.block in autotune.BLOCKS
    assert len(set(c)) == len(c)
