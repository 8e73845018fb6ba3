"""The batched persistent form (one launch for decode + Compass over a
batch of uneven events, CUDA-graph capturable) against the oracle."""
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
    return g


def check_against_oracle(g, pipe, b, params=P):
    hits = g.hits_to_numpy(pipe.hits_a)
    tr = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    oh, ot = oracle.run_batch(b, params)
    assert np.array_equal(hits["hit_off"], oh.hit_off)
    n = oh.n
    for k in ("x", "z"):
        assert np.array_equal(hits[k][:n].view(np.uint32), getattr(oh, k).view(np.uint32)), k
    for k in ("sector", "layer", "id"):
        assert np.array_equal(hits[k][:n], getattr(oh, k)), k
    assert np.array_equal(tr["hit"], ot.hit)
    assert np.array_equal(tr["nhits"], ot.nhits) and np.array_equal(tr["found"], ot.found)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(tr[k].view(np.uint32), getattr(ot, k).view(np.uint32)), k
    return ot


def test_batched_matches_oracle(g):
    b = synth.generate_config("batched", n_events=300)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched()
    ctx.check(what="batched")
    check_against_oracle(g, pipe, b)


@pytest.mark.parametrize("tpw", [1, 2, 4, 8])
@pytest.mark.parametrize("block", [128, 256, 512])
def test_batched_launch_shapes(g, tpw, block):
    b = synth.generate_config("batched", n_events=60, seed=31)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched(g.LaunchConfig(tpw, block, 8192, 8192))
    ctx.check(what="batched")
    check_against_oracle(g, pipe, b)


@pytest.mark.parametrize("tpw,block", [(4, 256), (8, 800)])
def test_batched_more_than_1024_banks(g, tpw, block):
    """600 sectors per layer (2400 banks per event): the sorted decode maps of
    the persistent kernel hold banks above 1023."""
    b = synth.generate(n_events=8, n_sectors=600, tracks=100, hits=6000, seed=17)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched(g.LaunchConfig(tpw, block, 8192, 8192))
    ctx.check(what="batched")
    check_against_oracle(g, pipe, b)
    ctx.close()


@pytest.mark.parametrize("block", [544, 672, 800])
def test_batched_large_blocks(g, block):
    """One block per SM of up to 25 warps (8 tracks per warp), on uneven
    events (many need several rounds of warp calls) and on events of 200
    tracks (one round at 800 threads)."""
    for b in (synth.generate_config("batched", n_events=60, seed=37),
              synth.generate_config("plain", n_events=64)):
        ctx = g.Context(b.geom)
        pipe = g.Pipeline(ctx, b, P)
        pipe.run_batched(g.LaunchConfig(8, block, 8192, 8192))
        ctx.check(what="batched")
        check_against_oracle(g, pipe, b)
        ctx.close()


@pytest.mark.parametrize("tpw,block,x_cap", [(4, 800, 8192), (8, 816, 8192), (8, 600, 8192),
                                             (8, 1024, 8192), (8, 800, 32768)])
def test_batched_rejects_unsupported_shapes(g, tpw, block, x_cap):
    """Large blocks exist for 8 tracks per warp only, as multiples of 32 up
    to 800 threads, and the shape must fit the block's shared memory: the
    call returns UT_ERR_ARG before any launch."""
    b = synth.generate_config("tiny")
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    with pytest.raises(g.UtError) as err:
        pipe.run_batched(g.LaunchConfig(tpw, block, x_cap, 8192))
    assert err.value.code == g.UT_ERR_ARG
    pipe.run_batched(g.LaunchConfig(8, 800, 8192, 8192))  # the context stays usable
    ctx.check(what="batched")
    check_against_oracle(g, pipe, b)


@pytest.mark.parametrize("x_cap,stage", [(256, 8192), (8192, 64), (0, 0)])
def test_batched_global_fallbacks(g, x_cap, stage):
    """Events larger than the shared-memory tiles are read from global memory."""
    b = synth.generate_config("batched", n_events=40, seed=32)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched(g.LaunchConfig(4, 256, x_cap, stage))
    ctx.check(what="batched")
    check_against_oracle(g, pipe, b)


def test_batched_parameter_sweep(g):
    b = synth.generate_config("batched", n_events=40, seed=33)
    ctx = g.Context(b.geom)
    for n_sec, n_cand in ((1, 1), (3, 2), (5, 16)):
        params = P.replace(n_sectors=n_sec, n_candidates=n_cand)
        pipe = g.Pipeline(ctx, b, params)
        pipe.run_batched()
        ctx.check(what="batched")
        check_against_oracle(g, pipe, b, params)


def test_batched_graph_replay(g):
    b = synth.generate_config("batched", n_events=200, seed=34)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    runner = g.GraphRunner(pipe)
    for _ in range(2):
        pipe.tracks.qop.fill_(123.0)
        pipe.hits_a.x.fill_(-1.0)
        runner.replay()
        torch.cuda.synchronize()
        ctx.check(what="graph")
        check_against_oracle(g, pipe, b)


def test_batched_reports_decode_errors(g):
    b = synth.generate_config("batched", n_events=50, seed=35)
    bad = b.raw.copy()
    base = int(b.ev_off[17])
    d = base + int(bad[base + 300])
    bad[d] = (bad[d] & 0xFFFF) | (301 << 16)
    bb = synth.generator.Batch(**{**b.__dict__, "raw": bad})
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, bb, P)
    pipe.run_batched()
    code, e, bank = ctx.status()
    rc, _, where = oracle.decode(bad, b.ev_off, b.n_events, b.geom, raise_on_error=False)
    assert (code, (e, bank)) == (rc, where) == (g.UT_ERR_HEADER, (17, 300))


def test_autotuner_picks_a_valid_config(g):
    from paper_2002_11529_gb300 import autotune
    b = synth.generate_config("batched", n_events=100, seed=36)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    best, table = autotune.autotune(pipe, reps=1)
    n_small = len(autotune.TRACKS_PER_WARP) * len(autotune.BLOCKS) * len(autotune.X_CAPS)
    assert len(table) == len(autotune.candidates(pipe)) >= n_small + len(autotune.LARGE_BLOCKS)
    assert all(ms > 0 for _, ms in table) and best in [c for c, _ in table]
    assert {128, 256, 512, *autotune.LARGE_BLOCKS} <= {c.block for c, _ in table}
    pipe.run_batched(best)
    ctx.check(what="autotuned")
    check_against_oracle(g, pipe, b)


def test_full_batched_workload_matches_oracle(g):
    """All 20000 events of the uneven-occupancy workload in one launch."""
    b = synth.generate_config("batched")
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched()
    ctx.check(what="batched")
    ot = check_against_oracle(g, pipe, b)
    m = ot.found.astype(bool)
    rel = np.abs(ot.qop[m].astype(np.float64) - ot.qop64[m]) / np.maximum(np.abs(ot.qop64[m]), 1e-2)
    print(f"\n20000 events: {b.n_tracks} tracks, found {int(m.sum())}, near-cut {int((ot.near <= 1e-5).sum())}, "
          f"float q/p vs double: max rel {rel.max():.2e}")
    assert rel.max() <= 1e-5


def test_full_plain_workload_every_tuned_shape(g):
    """The 1000-event, 256-sector workload in the benchmark's default launch:
    the persistent kernel captured in a CUDA graph and replayed, for every
    launch shape the autotuner can pick, each compared with the oracle."""
    from paper_2002_11529_gb300 import autotune
    b = synth.generate_config("plain")
    oh, ot = oracle.run_batch(b, P)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    shapes = autotune.candidates(pipe)
    assert g.LaunchConfig(8, 800) in shapes      # 200 tracks per event: one round of 25 warps
    for cfg in shapes:
        t, blk = cfg.tracks_per_warp, cfg.block
        runner = g.GraphRunner(pipe, cfg)
        for _ in range(2):
            pipe.tracks.qop.fill_(123.0)
            pipe.tracks.hit.fill_(-7)
            pipe.hits_a.x.fill_(-1.0)
            runner.replay()
            torch.cuda.synchronize()
            ctx.check(what=f"graph tpw={t} block={blk}")
        hits = g.hits_to_numpy(pipe.hits_a)
        tr = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
        assert np.array_equal(hits["hit_off"], oh.hit_off)
        assert np.array_equal(hits["x"][:oh.n].view(np.uint32), oh.x.view(np.uint32))
        assert np.array_equal(hits["id"][:oh.n], oh.id)
        assert np.array_equal(tr["hit"], ot.hit), (t, blk)
        assert np.array_equal(tr["found"], ot.found) and np.array_equal(tr["nhits"], ot.nhits)
        for k in ("qop", "chi2", "x", "tx"):
            assert np.array_equal(tr[k].view(np.uint32), getattr(ot, k).view(np.uint32)), (k, t, blk)
    ctx.close()
