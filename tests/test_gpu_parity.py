"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Decoded hits, offsets and sorted orders: bit-exact.  Compass: the kernels
take the same float decisions in the same operation order as the oracle, so
selected hits, nhits, found and the float fit outputs are compared exactly;
the count of tracks with a decision within 1e-5 of a cut is reported, and
the float q/p is checked against the oracle's double fit to 1e-5 relative
(floor 1e-2 1/GeV).
"""
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


_CTX = {}


def ctx_for(g, geom):
    key = geom.n_sectors
    if key not in _CTX:
        _CTX[key] = g.Context(geom)
    c = _CTX[key]
    c.reset()
    return c


def run_decode(g, ctx, raw, ev_off, n_events, geom, sorted_, capacity=None, n_words=None):
    raw_d, ev_d = g.upload_raw(raw, ev_off)
    nw = int(ev_off[n_events]) if n_words is None else n_words
    cap = 2 * nw + 8 if capacity is None else capacity
    hb = g.HitBuffers.allocate(cap, n_events, geom.n_sectors)
    g.ut_decode(ctx, raw_d, nw, ev_d, n_events, hb, sorted_)
    code, a, b = ctx.status()
    return code, (a, b), hb


def assert_hits_equal(gpu, orc, n):
    assert np.array_equal(gpu["hit_off"], orc.hit_off)
    assert np.array_equal(gpu["x"].view(np.uint32), orc.x[:n].view(np.uint32))
    assert np.array_equal(gpu["z"].view(np.uint32), orc.z[:n].view(np.uint32))
    assert np.array_equal(gpu["sector"], orc.sector[:n])
    assert np.array_equal(gpu["layer"], orc.layer[:n])
    assert np.array_equal(gpu["id"], orc.id[:n])


BATCHES = {
    "tiny": lambda: synth.generate_config("tiny"),
    "plain64": lambda: synth.generate_config("plain", n_events=64),
    "lognormal200": lambda: synth.generate_config("batched", n_events=200),
    # dense banks: exercise the counting-sort path (> 64 hits per bank)
    "dense": lambda: synth.generate(n_events=5, n_sectors=4, tracks=20, hits=3000, seed=7),
    # empty events in between
    "sparse": lambda: synth.generate(n_events=33, n_sectors=8, tracks=0, hits=3, seed=8),
    # more than 1024 banks per event (the sorted maps hold the bank in 16 bits)
    "wide600": lambda: synth.generate(n_events=8, n_sectors=600, tracks=100, hits=6000, seed=17),
}


@pytest.mark.parametrize("name", list(BATCHES))
@pytest.mark.parametrize("sorted_", [False, True])
def test_decode_bit_exact(g, name, sorted_):
    b = BATCHES[name]()
    ctx = ctx_for(g, b.geom)
    code, where, hb = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, sorted_)
    assert code == 0, (code, where)
    rc, orc, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_)
    assert rc == 0
    assert_hits_equal(g.hits_to_numpy(hb), orc, orc.n)


def test_decode_huge_bank_and_duplicates(g):
    """One bank with 5000 hits (duplicates of few strips) and 1-hit banks."""
    S = 4
    B = 4 * S
    rng = np.random.default_rng(3)
    n = np.ones((2, B), np.int64)
    n[1, 5] = 5000
    h = rng.integers(0, 40, int(n.sum())) * 2
    fl = rng.integers(0, 32, int(n.sum()))
    raw, ev_off = synth.encode(n, h, fl, S)
    geom = synth.Geometry(n_sectors=S)
    ctx = ctx_for(g, geom)
    for sorted_ in (False, True):
        code, where, hb = run_decode(g, ctx, raw, ev_off, 2, geom, sorted_)
        assert code == 0
        rc, orc, _ = oracle.decode(raw, ev_off, 2, geom, sorted_)
        assert_hits_equal(g.hits_to_numpy(hb), orc, orc.n)


def test_decode_event_larger_than_stage(g):
    """An event bigger than the shared-memory stage is read from global memory."""
    b = synth.generate(n_events=3, n_sectors=256, tracks=100, hits=20000, seed=9)
    ctx = ctx_for(g, b.geom)
    for sorted_ in (False, True):
        code, _, hb = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, sorted_)
        assert code == 0
        rc, orc, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_)
        assert_hits_equal(g.hits_to_numpy(hb), orc, orc.n)


@pytest.mark.parametrize("hits", [3000, 4500, 9000, 13000])
def test_decode_event_sizes_around_the_map_and_stage_limits(g, hits):
    """Events below and above the bank map's capacity (bank order: a map up
    to 4096 hits, the map-free output-order path above it) and below and
    above the staged size, in both output orders."""
    b = synth.generate(n_events=5, n_sectors=256, tracks=100, hits=hits, seed=31 + hits)
    ctx = ctx_for(g, b.geom)
    for sorted_ in (False, True):
        code, _, hb = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, sorted_)
        assert code == 0
        rc, orc, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_)
        assert_hits_equal(g.hits_to_numpy(hb), orc, orc.n)


def test_decode_empty_batch(g):
    geom = synth.Geometry(n_sectors=4)
    ctx = ctx_for(g, geom)
    hb = g.HitBuffers.allocate(4, 0, 4)
    hb.hit_off.fill_(123)
    raw_d = torch.zeros(4, dtype=torch.int32, device="cuda")
    ev_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.ut_decode(ctx, raw_d, 0, ev_d, 0, hb, True)
    assert ctx.status()[0] == 0
    assert int(hb.hit_off[0]) == 0


def _corrupt(b, cases):
    bad = b.raw.copy()
    B = b.geom.n_banks
    for e, bank, kind in cases:
        base = int(b.ev_off[e])
        d = base + int(bad[base + bank])
        if kind == "header":
            bad[d] = (bad[d] & 0xFFFF) | (((bank + 1) % B) << 16)
        elif kind == "dir":
            bad[base + bank] = 0xFFFFFF
        elif kind == "strip":
            # first non-empty bank at or after `bank`
            while (bad[d] & 0xFFFF) == 0:
                bank += 1
                d = base + int(bad[base + bank])
            bad[d + 1] = (bad[d + 1] & 0xFFFF0000) | 0x200 | (bad[d + 1] & 0xFC00)
    return bad


@pytest.mark.parametrize("cases", [
    [(9, 5, "header"), (3, 200, "header"), (3, 201, "strip")],
    [(2, 17, "dir")],
    [(12, 40, "strip"), (14, 2, "dir")],
])
def test_decode_errors_match_oracle(g, cases):
    b = synth.generate_config("tiny")
    # make sure the banks used for strip errors are not empty
    bad = _corrupt(b, [c for c in cases])
    ctx = ctx_for(g, b.geom)
    code, where, _ = run_decode(g, ctx, bad, b.ev_off, b.n_events, b.geom, True)
    rc, _, owhere = oracle.decode(bad, b.ev_off, b.n_events, b.geom, raise_on_error=False)
    assert rc != 0
    assert (code, where) == (rc, owhere)


def test_decode_capacity_error(g):
    b = synth.generate_config("tiny")
    ctx = ctx_for(g, b.geom)
    code, where, _ = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, True, capacity=b.n_hits - 1)
    assert code == g.UT_ERR_CAPACITY
    ctx.reset()
    code, _, _ = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, True, capacity=b.n_hits)
    assert code == 0


def test_decode_event_outside_buffer(g):
    b = synth.generate_config("tiny")
    ctx = ctx_for(g, b.geom)
    nw = int(b.ev_off[-1]) - 10       # last event claims words past the buffer
    code, where, _ = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, True, n_words=nw)
    rc, _, owhere = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, raise_on_error=False, n_words=nw)
    assert rc == g.UT_ERR_DIR and (code, where) == (rc, owhere)


@pytest.mark.parametrize("name", ["tiny", "dense", "plain64"])
def test_sort_hits_bit_exact(g, name):
    b = BATCHES[name]()
    ctx = ctx_for(g, b.geom)
    code, _, hu = run_decode(g, ctx, b.raw, b.ev_off, b.n_events, b.geom, False)
    assert code == 0
    n = int(hu.hit_off[-1].item() & 0xFFFFFFFF)
    hs = g.HitBuffers.allocate(max(n, 1), b.n_events, b.geom.n_sectors)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    g.ut_sort_hits(ctx, hu, hs, b.n_events, perm=perm)
    hs.hit_off = hu.hit_off
    assert ctx.status()[0] == 0
    _, ou, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, False)
    osorted, operm = oracle.sort_hits(ou)
    assert_hits_equal(g.hits_to_numpy(hs, n), osorted, n)
    assert np.array_equal(perm[:n].cpu().numpy().view(np.uint32), operm)


def run_compass(g, b, params, tracks_per_warp=1, block=256, want_windows=False, form="fused"):
    ctx = ctx_for(g, b.geom)
    pipe = g.Pipeline(ctx, b, params)
    win = None
    if want_windows:
        win = torch.full((max(b.n_tracks, 1), 4, params.n_sectors, 2), 7, dtype=torch.int16, device="cuda")
    if form == "fused":
        g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, b.n_events, pipe.hits_a, True, pipe.workspace)
        g.compass_find(ctx, pipe.hits_a, pipe.velo, b.n_events, params, pipe.tracks, win=win,
                       tracks_per_warp=tracks_per_warp, block=block)
    else:
        pipe.run_plain(tracks_per_warp=tracks_per_warp, block=block)
    code, a, bb = ctx.status()
    assert code == 0, (code, a, bb)
    out = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    if want_windows:
        out["win"] = win[: b.n_tracks].cpu().numpy()
    return out


def assert_tracks_equal(gpu, orc, b, report=True):
    T = b.n_tracks
    same_sel = np.all(gpu["hit"] == orc.hit, axis=1) & (gpu["nhits"] == orc.nhits) & (gpu["found"] == orc.found)
    near = orc.near <= 1e-5
    if report:
        print(f"\ntracks {T}: found {int(orc.found.sum())}, near-cut {int(near.sum())}, "
              f"selection mismatches {int((~same_sel).sum())} "
              f"(near-cut {int((~same_sel & near).sum())})")
    assert np.all(same_sel[~near]), np.nonzero(~same_sel & ~near)[0][:10]
    assert np.all(same_sel), "near-cut tracks also match"
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(gpu[k].view(np.uint32), getattr(orc, k).view(np.uint32)), k
    m = orc.found.astype(bool)
    rel = np.abs(gpu["qop"][m].astype(np.float64) - orc.qop64[m]) / np.maximum(np.abs(orc.qop64[m]), 1e-2)
    if m.any():
        print(f"float q/p vs double oracle fit: max rel err {rel.max():.3e}")
        assert rel.max() <= 1e-5


@pytest.mark.parametrize("name", ["tiny", "plain64", "lognormal200", "dense"])
def test_compass_find_matches_oracle(g, name):
    b = BATCHES[name]()
    gpu = run_compass(g, b, P)
    _, orc = oracle.run_batch(b, P)
    assert_tracks_equal(gpu, orc, b)


@pytest.mark.parametrize("tpw,block", [(1, 128), (2, 256), (4, 256), (4, 64), (8, 256), (8, 128),
                                       (8, 288), (8, 544), (8, 800)])
def test_compass_launch_shapes(g, tpw, block):
    b = BATCHES["plain64"]()
    gpu = run_compass(g, b, P, tracks_per_warp=tpw, block=block)
    _, orc = oracle.run_batch(b, P)
    assert_tracks_equal(gpu, orc, b, report=False)


@pytest.mark.parametrize("name", ["lognormal200", "dense"])
def test_compass_large_block_on_uneven_events(g, name):
    """800-thread blocks on events of very different track counts (several
    rounds of warp calls, or warps without tracks)."""
    b = BATCHES[name]()
    gpu = run_compass(g, b, P, tracks_per_warp=8, block=800, want_windows=True)
    _, orc = oracle.run_batch(b, P, want_windows=True)
    assert_tracks_equal(gpu, orc, b, report=False)
    assert np.array_equal(gpu["win"], orc.win)


@pytest.mark.parametrize("tpw,block", [(4, 512), (1, 288), (8, 832), (8, 300), (8, 32)])
def test_compass_rejects_unsupported_shapes(g, tpw, block):
    """Blocks above 256 threads exist for 8 tracks per warp only, up to 800
    threads, multiples of 32: other shapes return UT_ERR_ARG before any
    launch."""
    b = BATCHES["tiny"]()
    ctx = ctx_for(g, b.geom)
    pipe = g.Pipeline(ctx, b, P)
    g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, b.n_events, pipe.hits_a, True, pipe.workspace)
    with pytest.raises(g.UtError) as err:
        g.compass_find(ctx, pipe.hits_a, pipe.velo, b.n_events, P, pipe.tracks, tracks_per_warp=tpw, block=block)
    assert err.value.code == g.UT_ERR_ARG
    assert ctx.status()[0] == 0


@pytest.mark.parametrize("n_sec,n_cand", [(1, 1), (3, 2), (3, 16), (5, 1), (5, 16)])
def test_compass_parameter_sweep(g, n_sec, n_cand):
    b = BATCHES["tiny"]()
    params = P.replace(n_sectors=n_sec, n_candidates=n_cand)
    gpu = run_compass(g, b, params)
    _, orc = oracle.run_batch(b, params)
    assert_tracks_equal(gpu, orc, b, report=False)


def test_compass_windows_int16(g):
    b = synth.generate(n_events=8, n_sectors=64, tracks=60, hits=1200, seed=12, backward_frac=0.1)
    gpu = run_compass(g, b, P, want_windows=True)
    _, orc = oracle.run_batch(b, P, want_windows=True)
    assert np.array_equal(gpu["win"], orc.win)


def test_compass_wide_windows_beyond_stage(g):
    """Very dense events: combined ranges exceed the shared-memory stage."""
    b = synth.generate(n_events=2, n_sectors=8, tracks=30, hits=9000, seed=13)
    params = P.replace(n_candidates=4)
    for tpw in (1, 4):
        gpu = run_compass(g, b, params, tracks_per_warp=tpw)
        _, orc = oracle.run_batch(b, params)
        assert_tracks_equal(gpu, orc, b, report=False)


def test_plain_form_equals_fused_form(g):
    b = BATCHES["plain64"]()
    fused = run_compass(g, b, P, form="fused")
    plain = run_compass(g, b, P, form="plain")
    for k in fused:
        assert np.array_equal(fused[k], plain[k]), k


def test_compass_fit_matches_oracle(g):
    b = BATCHES["plain64"]()
    ctx = ctx_for(g, b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_fused()
    # refit the selected hits, plus tracks with hits knocked out
    hit = pipe.tracks.hit.clone()
    hit[::7, 1] = -1
    hit[::11, 0] = -1
    hit[::13, 2] = -1
    pipe.tracks.hit.copy_(hit)
    g.compass_fit(ctx, pipe.hits_a, pipe.velo, P, pipe.tracks)
    assert ctx.status()[0] == 0
    out = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    _, hits = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, True)[:2]
    ref = oracle.fit_tracks(hits.x, b.geom, oracle.Velo(b), hit.cpu().numpy(), P)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(out[k].view(np.uint32), ref[k].view(np.uint32)), k
    m = ref["ok"].astype(bool)
    rel = np.abs(out["qop"][m] - ref["qop64"][m]) / np.maximum(np.abs(ref["qop64"][m]), 1e-2)
    assert rel.max() <= 1e-5


def test_full_plain_workload_matches_oracle(g):
    """The 1000-event, 256-sector workload in the benchmark's launch form."""
    b = synth.generate_config("plain")
    gpu = run_compass(g, b, P, form="plain")
    _, orc = oracle.run_batch(b, P)
    assert_tracks_equal(gpu, orc, b)


@pytest.mark.parametrize("tpw", [1, 8])
def test_global_event_cut_matches_oracle(g, tpw):
    """Events over the Global Event Cut are not searched, in compass_find
    and in the persistent kernel alike."""
    b = synth.generate_config("batched", n_events=120)
    B = b.geom.n_banks
    ev_hits = b.bank_n.reshape(b.n_events, B).sum(axis=1)
    params = P.replace(gec_max_hits=int(np.median(ev_hits)))
    gpu = run_compass(g, b, params, tracks_per_warp=tpw, want_windows=True)
    _, orc = oracle.run_batch(b, params, want_windows=True)
    assert_tracks_equal(gpu, orc, b, report=False)
    assert np.array_equal(gpu["win"], orc.win)
    ctx = ctx_for(g, b.geom)
    pipe = g.Pipeline(ctx, b, params)
    pipe.run_batched(g.LaunchConfig(tracks_per_warp=tpw, block=256))
    ctx.check(what="batched gec")
    assert_tracks_equal(g.tracks_to_numpy(pipe.tracks, b.n_tracks), orc, b, report=False)
    assert int(orc.found.sum()) > 0 and not orc.found[np.repeat(ev_hits > params.gec_max_hits,
                                                                 np.diff(b.trk_off.astype(np.int64)))].any()
