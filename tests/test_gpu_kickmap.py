"""The kick map (ut_ctx_set_kick_map, the field look-up tables of Sec.
III-C) on the GPU against the oracle: compass_find, compass_fit and the
persistent kernel on hits made with a direction-dependent field; a constant
map equal to no map; removing the map; maps the ABI refuses."""
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


def _tracks_equal(gpu, orc, report=""):
    assert np.array_equal(gpu["hit"], orc.hit), report
    assert np.array_equal(gpu["nhits"], orc.nhits) and np.array_equal(gpu["found"], orc.found), report
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(gpu[k].view(np.uint32), getattr(orc, k).view(np.uint32)), (k, report)
    m = orc.found.astype(bool)
    rel = np.abs(gpu["qop"][m].astype(np.float64) - orc.qop64[m]) / np.maximum(np.abs(orc.qop64[m]), 1e-2)
    assert rel.max() <= 1e-5


@pytest.mark.parametrize("tpw", [1, 8])
def test_compass_find_with_map(g, tpw):
    b = synth.generate_config("fieldmap", n_events=64)
    km = synth.kick_map()
    ctx = g.Context(b.geom)
    ctx.set_kick_map(km)
    pipe = g.Pipeline(ctx, b, P)
    win = torch.full((b.n_tracks, 4, P.n_sectors, 2), 7, dtype=torch.int16, device="cuda")
    g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, b.n_events, pipe.hits_a, True, pipe.workspace)
    g.compass_find(ctx, pipe.hits_a, pipe.velo, b.n_events, P, pipe.tracks, win=win, tracks_per_warp=tpw)
    ctx.check(what="compass_find with map")
    _, orc = oracle.run_batch(b, P, want_windows=True, kick_map=km)
    _tracks_equal(g.tracks_to_numpy(pipe.tracks, b.n_tracks), orc)
    assert np.array_equal(win.cpu().numpy(), orc.win)
    _, plain = oracle.run_batch(b, P, want_windows=True)
    assert not np.array_equal(plain.win, orc.win)  # the map changed the windows
    ctx.close()


@pytest.mark.parametrize("tpw,block", [(8, 800), (8, 512), (4, 256), (1, 128)])
def test_persistent_kernel_with_map(g, tpw, block):
    b = synth.generate_config("fieldmap", n_events=96, seed=16)
    km = synth.kick_map(9, 13)
    ctx = g.Context(b.geom)
    ctx.set_kick_map(km)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched(g.LaunchConfig(tpw, block))
    ctx.check(what="batched with map")
    _, orc = oracle.run_batch(b, P, kick_map=km)
    _tracks_equal(g.tracks_to_numpy(pipe.tracks, b.n_tracks), orc, (tpw, block))
    ctx.close()


def test_compass_fit_with_map(g):
    b = synth.generate_config("fieldmap", n_events=32, seed=17)
    km = synth.kick_map()
    ctx = g.Context(b.geom)
    ctx.set_kick_map(km)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_fused()
    hit = pipe.tracks.hit.clone()
    hit[::7, 1] = -1
    pipe.tracks.hit.copy_(hit)
    g.compass_fit(ctx, pipe.hits_a, pipe.velo, P, pipe.tracks)
    ctx.check(what="compass_fit with map")
    out = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    _, hits = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, True)[:2]
    ref = oracle.fit_tracks(hits.x, b.geom, oracle.Velo(b), hit.cpu().numpy(), P, kick_map=km)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(out[k].view(np.uint32), ref[k].view(np.uint32)), k
    ctx.close()


def test_constant_map_and_removal(g):
    b = synth.generate_config("tiny", seed=12)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched(g.LaunchConfig(8, 512))
    ref = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    ctx.set_kick_map(synth.KickMap(2, 2, 0.3, 0.25, np.full((2, 2), P.kick_k, np.float32)))
    pipe.run_batched(g.LaunchConfig(8, 512))
    same = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    ctx.set_kick_map(synth.kick_map())
    pipe.run_batched(g.LaunchConfig(8, 512))
    moved = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    ctx.set_kick_map(None)
    pipe.run_batched(g.LaunchConfig(8, 512))
    back = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    ctx.check(what="maps")
    for k in ref:
        assert np.array_equal(ref[k], same[k]) and np.array_equal(ref[k], back[k]), k
    assert not np.array_equal(ref["qop"], moved["qop"])
    _, orc = oracle.run_batch(b, P)
    _tracks_equal(back, orc)
    ctx.close()


@pytest.mark.parametrize("nx,ny,tx,ty,fill", [(1, 4, 0.3, 0.25, 1.0), (4, 300, 0.3, 0.25, 1.0),
                                              (4, 4, 0.0, 0.25, 1.0), (4, 4, 0.3, 0.25, -1.0),
                                              (4, 4, 0.3, 0.25, float("nan"))])
def test_refused_maps(g, nx, ny, tx, ty, fill):
    b = synth.generate_config("tiny")
    ctx = g.Context(b.geom)
    km = synth.KickMap(nx, ny, tx, ty, np.full((ny, nx), fill, np.float32))
    with pytest.raises(g.UtError) as err:
        ctx.set_kick_map(km)
    assert err.value.code == g.UT_ERR_ARG
    ctx.close()


def test_full_fieldmap_workload(g):
    """All 1000 events of the field workload, persistent form at the
    benchmark's shape, with the map."""
    b = synth.generate_config("fieldmap")
    km = synth.kick_map()
    ctx = g.Context(b.geom)
    ctx.set_kick_map(km)
    pipe = g.Pipeline(ctx, b, P)
    g.GraphRunner(pipe, g.LaunchConfig(8, 800)).replay()
    torch.cuda.synchronize()
    ctx.check(what="fieldmap")
    oh, orc = oracle.run_batch(b, P, kick_map=km)
    hits = g.hits_to_numpy(pipe.hits_a)
    assert np.array_equal(hits["hit_off"], oh.hit_off)
    _tracks_equal(g.tracks_to_numpy(pipe.tracks, b.n_tracks), orc)
    ctx.close()
