"""compass_find_groups (Compass on the sector-group layout: windows over the
x regions with two binary searches in y, Sec. V-A; tracklet search and
selection, Sec. V-B) against the oracle's group search, bit for bit: hit
indices, q/p, chi2, x, tx, nhits and found of every track, on several
detector shapes (up to 1000 events), y tolerances, parameter sets, the kick
map and the Global Event Cut.  Tracks whose smallest decision margin is
within 1e-5 of a cut are counted and printed, and must match too (both
sides decide in float with the same operations)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from synth.grouped import generate_grouped

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    assert torch.cuda.is_available()
    return g


def run_gpu(g, b, params, tol_y, kick_map=None, vy=None, vty=None):
    ctx, gh = g.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    if kick_map is not None:
        ctx.set_kick_map(kick_map)
    bb = b if vy is None else dataclasses.replace(b, velo_y=vy, velo_ty=vty)
    velo = g.upload_velo(bb)
    out = g.TrackBuffers.allocate(b.n_tracks)
    out.hit.fill_(-7)
    g.compass_find_groups(ctx, gh, b.geom, velo, b.n_events, params, out, tol_y)
    ctx.check(what="compass_find_groups")
    tr = g.tracks_to_numpy(out, b.n_tracks)
    ctx.close()
    return tr


def compare(g, b, params, tol_y, kick_map=None, vy=None, vty=None, min_found=1):
    ref_gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    ref = oracle.compass_groups(ref_gh, b, params, tol_y=tol_y, kick_map=kick_map, vy=vy, vty=vty)
    got = run_gpu(g, b, params, tol_y, kick_map, vy, vty)
    near = int(np.sum(ref.near <= 1e-5))
    print(f"tracks {b.n_tracks}, found {int(ref.found.sum())}, near-cut {near}")
    assert np.array_equal(got["found"], ref.found)
    assert np.array_equal(got["nhits"], ref.nhits)
    assert np.array_equal(got["hit"], ref.hit)
    for k, r in (("qop", ref.qop), ("chi2", ref.chi2), ("x", ref.x), ("tx", ref.tx)):
        assert np.array_equal(got[k].view(np.uint32), r.view(np.uint32)), k
    assert int(ref.found.sum()) >= min_found
    # q/p within 1e-5 of the double fit (floor 1e-2 GeV^-1)
    f = ref.found.astype(bool)
    assert np.all(np.abs(got["qop"][f] - ref.qop64[f]) <= 1e-5 * np.maximum(np.abs(ref.qop64[f]), 1e-2))
    return ref


SHAPES = {
    "default": dict(n_events=16, seed=51),
    "rows3_groups10": dict(n_events=12, n_columns=8, rows=3, n_groups=10, seed=52),
    "one_row": dict(n_events=10, rows=1, n_groups=6, seed=53),
    "max_groups": dict(n_events=6, n_columns=32, rows=7, n_groups=128, tracks=100, hits=2500, seed=54),
}


@pytest.mark.parametrize("name", list(SHAPES))
@pytest.mark.parametrize("tol_y", [5.0, 60.0])
def test_group_search_matches_oracle(g, name, tol_y):
    compare(g, generate_grouped(**SHAPES[name]), synth.CompassParams(), tol_y, min_found=20)


def test_group_search_1000_events(g):
    """The benchmark's grouped workload: 1000 events, 48 columns x 4 rows of
    sensors, 84 groups, 200 tracks and 4000 hits per event."""
    b = generate_grouped(1000, n_columns=48, rows=4, n_groups=84, tracks=200, hits=4000, seed=21)
    compare(g, b, synth.CompassParams(), 5.0, min_found=100000)


@pytest.mark.parametrize("ns,nc", [(1, 1), (3, 2), (5, 16), (5, 1)])
def test_group_search_parameters(g, ns, nc):
    b = generate_grouped(20, tracks=80, hits=2000, seed=55)
    compare(g, b, synth.CompassParams(n_sectors=ns, n_candidates=nc), 20.0)


def test_group_search_without_y_cut(g):
    """tol_y beyond the plane: every row is searched (more candidates per
    layer, more valid tracklets than n_candidates)."""
    b = generate_grouped(12, tracks=60, hits=1500, seed=56)
    compare(g, b, synth.CompassParams(), 1e6, min_found=100)


def test_group_search_on_row_boundaries(g):
    """Tracks flat in y whose y window ends exactly on a row boundary (y = 130
    and 120 mm, tol_y = 130: y - tol_y = 0 and y + tol_y = 250 exactly): the
    boundary rows are in the window on both sides."""
    b = generate_grouped(10, tracks=60, hits=1500, seed=57)
    T = b.n_tracks
    vty = np.zeros(T, np.float32)
    for y in (130.0, 120.0):
        ref = compare(g, b, synth.CompassParams(), 130.0, vy=np.full(T, y, np.float32), vty=vty, min_found=0)
        assert np.all(ref.near[ref.found.astype(bool)] == 0.0)


def test_group_search_kick_map_and_event_cut(g):
    b = generate_grouped(16, tracks=60, hits=1500, seed=58)
    compare(g, b, synth.CompassParams(), 10.0, kick_map=synth.kick_map(), min_found=50)
    per_event = np.bincount(b.truth_event, minlength=b.n_events)
    P = synth.CompassParams(gec_max_hits=int(np.median(per_event)))
    ref = compare(g, b, P, 10.0)
    over = np.repeat(per_event > P.gec_max_hits, np.diff(b.trk_off.astype(np.int64)))
    assert over.any() and not ref.found[over].any()


def test_group_search_events_without_tracks_and_backward_tracks(g):
    """Events whose VELO tracks are removed (no tracks at all), and backward
    tracks (never searched)."""
    b = generate_grouped(8, tracks=30, hits=900, seed=59, backward_frac=0.2)
    keep_ev = np.array([0, 1, 0, 1, 1, 0, 1, 1], bool)
    n_ev = np.diff(b.trk_off.astype(np.int64))
    keep = np.repeat(keep_ev, n_ev)
    trk_off = np.zeros(b.n_events + 1, np.uint32)
    trk_off[1:] = np.cumsum(n_ev * keep_ev)
    sub = dataclasses.replace(b, velo_x=b.velo_x[keep], velo_y=b.velo_y[keep], velo_tx=b.velo_tx[keep],
                              velo_ty=b.velo_ty[keep], velo_flags=b.velo_flags[keep], trk_off=trk_off,
                              qop_true=b.qop_true[keep])
    assert (sub.velo_flags & 1).any()
    ref = compare(g, sub, synth.CompassParams(), 10.0, min_found=10)
    assert not ref.found[(sub.velo_flags & 1).astype(bool)].any()


def test_group_search_refused_arguments(g):
    b = generate_grouped(4, seed=60)
    ctx, gh = g.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    velo = g.upload_velo(b)
    out = g.TrackBuffers.allocate(b.n_tracks)
    bad = dataclasses.replace(b.geom, edges=np.array([0.0, 1.0, 1.0, 2.0], np.float32), n_groups=3)
    for gg, tol in ((bad, 5.0), (b.geom, float("nan"))):
        with pytest.raises(g.UtError) as err:
            g.compass_find_groups(ctx, gh, gg, velo, b.n_events, synth.CompassParams(), out, tol)
        assert err.value.code == g.UT_ERR_ARG
    with pytest.raises(g.UtError):
        g.compass_find_groups(ctx, gh, b.geom, velo, b.n_events, synth.CompassParams(n_sectors=6), out, 5.0)
    ctx.check(what="refused")
    ctx.close()


def test_group_search_dense_layers_walk_the_y_windows(g):
    """Dense events without a y cut: layers with more candidates than the
    per-warp list holds (64) take the walking form; same results."""
    b = generate_grouped(6, tracks=40, hits=6000, seed=62)
    compare(g, b, synth.CompassParams(), 1e6, min_found=50)
    compare(g, b, synth.CompassParams(n_candidates=3), 1e6, min_found=50)
