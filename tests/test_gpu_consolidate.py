"""ut_consolidate (through the C ABI) against the oracle's definition:
the found tracks in (event, VELO track) order and every event's first row,
bit-exact; events without tracks; the capacity error; no events."""
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


def _run(g, b, capacity=None):
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched()
    ctx.check(what="tracks")
    n_found = int(pipe.tracks.found[: b.n_tracks].sum().item()) if b.n_tracks else 0
    cap = n_found if capacity is None else capacity
    out = g.CompactTracks.allocate(cap)
    off = torch.full((b.n_events + 1,), -7, dtype=torch.int32, device="cuda")
    g.ut_consolidate(ctx, pipe.velo.trk_off, b.n_events, pipe.tracks, out, off)
    code, a, bb = ctx.status()
    return ctx, pipe, out, off.cpu().numpy().view(np.uint32), code, n_found


def _same(gpu, ref, n):
    for k in ("hit", "nhits", "velo"):
        assert np.array_equal(gpu[k][:n], ref[k][:n]), k
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(gpu[k][:n].view(np.uint32), ref[k][:n].view(np.uint32)), k


def test_consolidation_matches_the_oracle(g):
    b = synth.generate_config("batched", n_events=300)
    ctx, pipe, out, off, code, n = _run(g, b)
    assert code == 0 and n > 0
    tracks = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    ref, ref_off = oracle.consolidate(tracks, b.trk_off)
    assert np.array_equal(off, ref_off)
    _same(g.compact_to_numpy(out, n), ref, n)
    # the tracks themselves are the oracle's
    _, orc = oracle.run_batch(b, P)
    assert np.array_equal(tracks["hit"], orc.hit)


def test_parts_of_many_events_with_empty_events(g):
    """2000 events (several events per block part), a third of them with
    their found flags cleared, some parts ending in such events."""
    b = synth.generate_config("batched", n_events=2000)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched()
    ctx.check(what="tracks")
    rng = np.random.default_rng(5)
    for e in np.flatnonzero(rng.random(b.n_events) < 0.33):
        pipe.tracks.found[int(b.trk_off[e]):int(b.trk_off[e + 1])] = 0
    pipe.tracks.found[int(b.trk_off[b.n_events - 40]):int(b.trk_off[b.n_events])] = 0
    tracks = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    n = int(tracks["found"].sum())
    out = g.CompactTracks.allocate(n)
    off = torch.full((b.n_events + 1,), -7, dtype=torch.int32, device="cuda")
    g.ut_consolidate(ctx, pipe.velo.trk_off, b.n_events, pipe.tracks, out, off)
    ctx.check(what="consolidation")
    ref, ref_off = oracle.consolidate(tracks, b.trk_off)
    assert np.array_equal(off.cpu().numpy().view(np.uint32), ref_off)
    _same(g.compact_to_numpy(out, n), ref, n)
    ctx.close()


def test_events_without_tracks(g):
    b = synth.generate(n_events=33, n_sectors=8, tracks=0, hits=3, seed=8)
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    out = g.CompactTracks.allocate(0)
    off = torch.full((b.n_events + 1,), -7, dtype=torch.int32, device="cuda")
    g.ut_consolidate(ctx, pipe.velo.trk_off, b.n_events, pipe.tracks, out, off)
    ctx.check(what="empty")
    assert np.all(off.cpu().numpy() == 0)


def test_capacity_error_keeps_offsets_and_first_rows(g):
    b = synth.generate_config("batched", n_events=40)
    ctx, pipe, out, off, code, n = _run(g, b, capacity=None)
    assert code == 0
    ctx2, pipe2, out2, off2, code2, n2 = _run(g, b, capacity=n - 5)
    assert code2 == g.UT_ERR_CAPACITY
    assert np.array_equal(off2, off)
    _same(g.compact_to_numpy(out2, n - 5), g.compact_to_numpy(out, n), n - 5)


def test_no_events_writes_a_zero_offset(g):
    b = synth.generate_config("tiny")
    ctx = g.Context(b.geom)
    off = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    pipe = g.Pipeline(ctx, b, P)
    g.ut_consolidate(ctx, pipe.velo.trk_off, 0, pipe.tracks, g.CompactTracks.allocate(1), off)
    ctx.check(what="no events")
    assert int(off[0].item()) == 0
