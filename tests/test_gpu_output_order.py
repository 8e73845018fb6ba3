"""The paper's output order (Sec. V-B: a found track's index inside its event
comes from an atomic counter), compass_params.output_order = 1, against the
oracle: per event, the number of found tracks and the set of found tracks
(VELO index, hits, q/p, chi2, x, tx, nhits) are the oracle's, whatever
their order; every row of the event names a different VELO track.  On
compass_find, the persistent kernel and the group search."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth.grouped import generate_grouped

pytestmark = pytest.mark.gpu

P1 = synth.CompassParams(output_order=1)


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    assert torch.cuda.is_available()
    return g


def rows_of(tracks, trk_off):
    """(event -> sorted list of row tuples) of an atomic-order output."""
    velo = tracks.velo.cpu().numpy()
    nf = tracks.n_found.cpu().numpy()
    hit = tracks.hit.cpu().numpy()
    cols = [getattr(tracks, k).cpu().numpy().view(np.uint32) for k in ("qop", "chi2", "x", "tx")]
    nh = tracks.nhits.cpu().numpy()
    out = []
    for e in range(len(trk_off) - 1):
        t0 = int(trk_off[e])
        n = int(nf[e])
        assert 0 <= n <= int(trk_off[e + 1]) - t0
        rows = [(int(velo[r]), tuple(hit[r]), *(int(c[r]) for c in cols), int(nh[r])) for r in range(t0, t0 + n)]
        assert len({r[0] for r in rows}) == n                           # distinct VELO tracks
        assert all(t0 <= r[0] < int(trk_off[e + 1]) for r in rows)      # of this event
        out.append(sorted(rows))
    return out


def oracle_rows(ot, trk_off):
    out = []
    cols = [getattr(ot, k).view(np.uint32) for k in ("qop", "chi2", "x", "tx")]
    for e in range(len(trk_off) - 1):
        rows = [(t, tuple(ot.hit[t]), *(int(c[t]) for c in cols), int(ot.nhits[t]))
                for t in range(int(trk_off[e]), int(trk_off[e + 1])) if ot.found[t]]
        out.append(sorted(rows))
    return out


@pytest.mark.parametrize("form", ["find", "batched"])
def test_atomic_order_matches_oracle_as_sets(g, form):
    b = synth.generate_config("plain", n_events=64)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P1)
    pipe.tracks = g.TrackBuffers.allocate(b.n_tracks, n_events=b.n_events)
    if form == "find":
        pipe.run_fused(tracks_per_warp=8, block=800)
    else:
        pipe.run_batched(g.LaunchConfig(tracks_per_warp=8, block=800))
    ctx.check(what="atomic order")
    _, ot = oracle.run_batch(b, P1)
    got = rows_of(pipe.tracks, b.trk_off)
    assert got == oracle_rows(ot, b.trk_off)
    assert sum(len(r) for r in got) == int(ot.found.sum()) > 10000
    ctx.close()


def test_atomic_order_group_search(g):
    b = generate_grouped(20, tracks=80, hits=2000, seed=61)
    ctx, gh = g.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    velo = g.upload_velo(b)
    out = g.TrackBuffers.allocate(b.n_tracks, n_events=b.n_events)
    g.compass_find_groups(ctx, gh, b.geom, velo, b.n_events, P1, out, 10.0)
    ctx.check(what="atomic order groups")
    ref_gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    ref = oracle.compass_groups(ref_gh, b, P1, tol_y=10.0)
    assert rows_of(out, b.trk_off) == oracle_rows(ref, b.trk_off)
    ctx.close()


def test_atomic_order_needs_its_arrays(g):
    b = synth.generate_config("tiny")
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P1)       # TrackBuffers without velo / n_found
    with pytest.raises(g.UtError) as err:
        pipe.run_fused()
    assert err.value.code == g.UT_ERR_ARG
    with pytest.raises(g.UtError):
        g.compass_find(ctx, pipe.hits_a, pipe.velo, b.n_events, P1.replace(output_order=2), pipe.tracks)
    ctx.close()
