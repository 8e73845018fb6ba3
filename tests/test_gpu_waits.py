"""Bounded device waits that run out (failure detection without a GPU fault).

The cause is made on the host: the context's first work ticket is set to 1,
so event 0 is never decoded and every later event's look-back waits for a
predecessor that never publishes.  With a short wait limit each such wait
runs out: the kernel records UT_ERR_TIMEOUT at the first waiting event and
returns, and the context stays usable (a normal run afterwards matches the
oracle bit for bit).  No kernel traps, faults or waits without a limit."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

P = synth.CompassParams()


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    assert torch.cuda.is_available()
    return g


def _check_normal_run(g, ctx, pipe, batch, run):
    ctx.set_first_ticket(0)
    ctx.set_wait_limit(0)
    ctx.reset()
    pipe.hits_a.x.fill_(-1.0)
    run()
    ctx.check(what="normal run after the timeout")
    oh, ot = oracle.run_batch(batch, P)
    hits = g.hits_to_numpy(pipe.hits_a)
    assert np.array_equal(hits["hit_off"], oh.hit_off)
    assert np.array_equal(hits["x"].view(np.uint32), oh.x.view(np.uint32))
    return ot


@pytest.mark.parametrize("sorted_", [True, False])
def test_decode_lookback_wait_runs_out(g, sorted_):
    batch = synth.generate(n_events=8, n_sectors=64, tracks=50, hits=800, seed=71)
    ctx = g.Context(batch.geom)
    pipe = g.Pipeline(ctx, batch, P)
    ctx.set_wait_limit(2000)
    ctx.set_first_ticket(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, batch.n_events, pipe.hits_a, sorted_, pipe.workspace)
    code, ev, bank = ctx.status()
    dt = time.perf_counter() - t0
    assert code == g.UT_ERR_TIMEOUT and ev == 1 and bank == -1
    assert dt < 5.0                                   # the kernel returned
    run = lambda: g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, batch.n_events, pipe.hits_a, True,
                              pipe.workspace)
    _check_normal_run(g, ctx, pipe, batch, run)
    ctx.close()


@pytest.mark.parametrize("shape", [(8, 800), (4, 256)])
def test_persistent_kernel_lookback_wait_runs_out(g, shape):
    batch = synth.generate(n_events=12, n_sectors=64, tracks=50, hits=800, seed=72)
    ctx = g.Context(batch.geom)
    pipe = g.Pipeline(ctx, batch, P)
    cfg = g.LaunchConfig(tracks_per_warp=shape[0], block=shape[1])
    ctx.set_wait_limit(2000)
    ctx.set_first_ticket(1)
    pipe.run_batched(cfg)
    code, ev, bank = ctx.status()
    assert code == g.UT_ERR_TIMEOUT and ev == 1 and bank == -1
    ot = _check_normal_run(g, ctx, pipe, batch, lambda: pipe.run_batched(cfg))
    tr = g.tracks_to_numpy(pipe.tracks, batch.n_tracks)
    assert np.array_equal(tr["hit"], ot.hit)
    ctx.close()


def test_wait_limit_arguments(g):
    batch = synth.generate(n_events=2, n_sectors=64, tracks=5, hits=100, seed=73)
    ctx = g.Context(batch.geom)
    with pytest.raises(g.UtError):
        ctx.set_first_ticket(-1)
    ctx.set_wait_limit(-5)          # restores the default
    ctx.set_wait_limit(0)
    ctx.close()
