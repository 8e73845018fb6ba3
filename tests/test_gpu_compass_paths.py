"""The tracklet-resolution paths of the GPU search against the oracle, on
hand-built events (through the C ABI).

A track whose layers each carry a cluster of hits around its straight line
gets one valid tracklet per (first anchor, second anchor) pair: clusters of
2..7 hits give 4..49 valid tracklets, so the GPU takes each of its paths --
at most n_candidates valid (the warp search's record), up to 32 (the
selection among the listed keys), more (the sequential ordered path).  The
hits sit at -1, 0, +1 half-strips from the line, so the tracklets differ in
chi2 and "the best of the first n_candidates in order" differs from "the
best of all".  A second event puts more than 32767 hits in front of the
first anchors in combined order, past what the packed key holds (the
per-group fallback).  Selections, nhits, found and the float fit outputs
must be identical to the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth.generator import Batch

pytestmark = pytest.mark.gpu

P = synth.CompassParams()


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    assert torch.cuda.is_available()
    return g


def _u(geom, x, y, tx, ty, l):
    dz = np.float64(geom.z[l]) - np.float64(geom.z_velo)
    return (np.float64(x) + np.float64(tx) * dz) - (np.float64(y) + np.float64(ty) * dz) * np.float64(geom.tan_stereo[l])


def _sector_h(geom, u):
    s = int(np.floor((u - geom.x_min) / geom.sector_pitch))
    h = int(np.floor((u - (geom.x_min + s * geom.sector_pitch)) / (geom.strip_pitch / 2)))
    return s, h


def build_event(geom, tracks, extra=()):
    """One event.  tracks: (x, y, tx, ty, offsets per layer) with hit
    offsets in half-strips from the track's line; extra: (layer, sector,
    list of h) added as they are.  Returns a Batch."""
    S, B = geom.n_sectors, geom.n_banks
    banks = [[] for _ in range(B)]
    vx, vy, vtx, vty = [], [], [], []
    for (x, y, tx, ty, offs) in tracks:
        vx.append(x), vy.append(y), vtx.append(tx), vty.append(ty)
        for l in range(4):
            s, h = _sector_h(geom, _u(geom, x, y, tx, ty, l))
            banks[l * S + s] += [h + o for o in offs[l] if 0 <= h + o < 2 * geom.strips]
    for (l, s, hs) in extra:
        banks[l * S + s] += list(hs)
    rng = np.random.default_rng(3)
    for b in banks:  # word order inside a bank: shuffled, like the generator
        rng.shuffle(b)
    bank_n = np.array([[len(b) for b in banks]], np.int64)
    h = np.array([v for b in banks for v in b], np.int64)
    flags = np.zeros(h.size, np.int64)
    raw, ev_off = synth.encode(bank_n, h, flags, S)
    T = len(tracks)
    f32 = lambda a: np.asarray(a, np.float32)
    nh = int(h.size)
    return Batch(geom=geom, n_events=1, raw=raw, ev_off=ev_off, velo_x=f32(vx), velo_y=f32(vy),
                 velo_tx=f32(vtx), velo_ty=f32(vty), velo_flags=np.zeros(T, np.uint8),
                 trk_off=np.array([0, T], np.uint32), qop_true=np.zeros(T, np.float32),
                 bank_n=bank_n.ravel().astype(np.uint32), truth_event=np.zeros(nh, np.int32),
                 truth_layer=np.zeros(nh, np.int32), truth_sector=np.zeros(nh, np.int32),
                 truth_h=h.astype(np.int32), truth_flags=np.zeros(nh, np.int32),
                 truth_track=np.full(nh, -1, np.int32))


def run(g, b, params, tpw):
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, params)
    g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, b.n_events, pipe.hits_a, True, pipe.workspace)
    g.compass_find(ctx, pipe.hits_a, pipe.velo, b.n_events, params, pipe.tracks, tracks_per_warp=tpw)
    code, a, bb = ctx.status()
    assert code == 0, (code, a, bb)
    gpu = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    cfg = g.LaunchConfig(tracks_per_warp=tpw, block=256)
    pipe.run_batched(cfg=cfg)
    ctx.check(what="batched")
    gpu_b = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
    return gpu, gpu_b


def same(gpu, orc):
    assert np.array_equal(gpu["hit"], orc.hit)
    assert np.array_equal(gpu["nhits"], orc.nhits) and np.array_equal(gpu["found"], orc.found)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(gpu[k].view(np.uint32), getattr(orc, k).view(np.uint32)), k


def cluster(n):
    return [(-1, 0, 1)[i % 3] for i in range(n)]


@pytest.mark.parametrize("n_cand", [8, 3])
@pytest.mark.parametrize("tpw", [1, 4, 8])
def test_record_list_and_ordered_paths(g, tpw, n_cand):
    geom = synth.Geometry(n_sectors=16)
    tracks = []
    # cluster sizes 1..7 in the anchor layers, 1..3 in the collection layers;
    # tracks 200 mm apart so that their windows do not meet
    for i, n in enumerate([2, 3, 4, 5, 6, 7, 1, 2, 6]):
        x = -700.0 + 170.0 * i
        offs = [cluster(n), cluster(1 + i % 3), cluster(n), cluster(1 + (i + 1) % 3)]
        tracks.append((x, 0.0, 0.0, 0.0, offs))
    b = build_event(geom, tracks)
    params = P.replace(n_candidates=n_cand)
    _, orc = oracle.run_batch(b, params)
    assert orc.found.all()
    gpu, gpu_b = run(g, b, params, tpw)
    same(gpu, orc)
    same(gpu_b, orc)


def test_combined_index_beyond_the_key(g):
    """More than 32767 hits precede the valid first anchors in combined
    order.  The track is predicted 0.05 mm below the lower edge of sector c,
    so its central sector is c - 1 (slot order c-1, c-2, c, ...); its hits
    lie just above that edge, in sector c, behind the 36000 hits that fill
    sector c - 1."""
    geom = synth.Geometry(n_sectors=8)
    c = 4
    x0 = float(np.float32(geom.x_min + c * geom.sector_pitch)) - 0.05
    s0, _ = _sector_h(geom, _u(geom, x0, 0.0, 0.0, 0.0, 0))
    assert s0 == c - 1
    dense = [k % 1024 for k in range(36000)]
    b = build_event(geom, [(x0, 0.0, 0.0, 0.0, [[], [], [], []])],
                    extra=[(0, c, [0, 1]), (1, c, [0]), (2, c, [0]), (3, c, [0]), (0, c - 1, dense)])
    assert b.bank_n.max() < 65536
    _, orc = oracle.run_batch(b, P)
    assert orc.found.all()
    gpu, gpu_b = run(g, b, P, 4)
    same(gpu, orc)
    same(gpu_b, orc)
