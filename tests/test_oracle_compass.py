"""Pins of the oracle's Compass search (Sec. V-A, V-B).

The oracle takes every decision in float (the paper's GPU precision); the
pins below re-derive the same results independently in double precision
(brute force over all hits of an event, library least squares) and must
agree on every track whose decisions are not within 1e-5 of a cut.
"""
import math

import numpy as np
import pytest

import brute
import oracle
import synth

P = synth.CompassParams()


def _event_hits(hits, e, B):
    a, b = int(hits.hit_off[e * B]), int(hits.hit_off[(e + 1) * B])
    return a, hits.x[a:b], hits.layer[a:b], hits.sector[a:b]


def _compare_with_brute(batch, params, mode, max_tracks=None):
    _, hits, _ = oracle.decode(batch.raw, batch.ev_off, batch.n_events, batch.geom)
    tr = oracle.compass(hits.x, hits.hit_off, batch.n_events, batch.geom, oracle.Velo(batch), params)
    B = batch.geom.n_banks
    checked = near = mismatched = 0
    for e in range(batch.n_events):
        base, x, lay, sec = _event_hits(hits, e, B)
        for t in range(int(batch.trk_off[e]), int(batch.trk_off[e + 1])):
            sel, q, chi2, nh = brute.track_search(
                x, lay, sec, batch.geom, batch.velo_x[t], batch.velo_y[t], batch.velo_tx[t],
                batch.velo_ty[t], batch.velo_flags[t] & 1, params, mode=mode)
            sel_g = [s + base if s >= 0 else -1 for s in sel]
            same = (list(tr.hit[t]) == sel_g) and int(tr.nhits[t]) == nh
            if tr.near[t] <= 1e-5:
                near += 1
                continue
            checked += 1
            if not same:
                mismatched += 1
                continue
            if nh:
                assert abs(tr.qop64[t] - q) <= 1e-9 * max(abs(q), 1e-2)
                assert abs(float(tr.qop[t]) - q) <= 1e-5 * max(abs(q), 1e-2)
    return checked, near, mismatched, tr


@pytest.mark.parametrize("n_sec,n_cand", [(5, 8), (3, 2), (1, 1), (5, 16)])
def test_sequential_rule_matches_double_brute_force(n_sec, n_cand):
    b = synth.generate(n_events=12, n_sectors=16, tracks=4, hits=60, seed=21 + n_sec * 7 + n_cand,
                       backward_frac=0.1)
    params = P.replace(n_sectors=n_sec, n_candidates=n_cand)
    checked, near, bad, tr = _compare_with_brute(b, params, "sequential")
    assert bad == 0
    assert checked >= 0.8 * b.n_tracks
    assert tr.found.sum() > 0


@pytest.mark.parametrize("n_cand", [1, 4, 16])
def test_sequential_rule_dense_events(n_cand):
    """Dense events (about 12 hits per bank): the candidate cut-off and the
    nearest-hit rule both act."""
    b = synth.generate(n_events=4, n_sectors=8, tracks=10, hits=400, seed=91 + n_cand)
    params = P.replace(n_candidates=n_cand)
    checked, near, bad, tr = _compare_with_brute(b, params, "sequential")
    assert bad == 0 and checked >= 0.7 * b.n_tracks


def test_global_argmin_when_unbounded_and_sparse():
    b = synth.generate(n_events=20, n_sectors=16, tracks=3, hits=20, seed=33)
    params = P.replace(n_candidates=100000)
    checked, near, bad, tr = _compare_with_brute(b, params, "argmin")
    assert bad == 0 and checked >= 0.8 * b.n_tracks


def test_isolated_noise_free_track_recovers_its_hits():
    b = synth.generate(n_events=200, n_sectors=64, tracks=1, hits=None, noise_frac=0.0,
                       seed=41, smear=False, efficiency=1.0)
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom)
    tr = oracle.compass(hits.x, hits.hit_off, b.n_events, b.geom, oracle.Velo(b), P)
    B = b.geom.n_banks
    n_full = 0
    for e in range(b.n_events):
        a, z = int(hits.hit_off[e * B]), int(hits.hit_off[(e + 1) * B])
        lay = hits.layer[a:z]
        if len(lay) != 4 or sorted(lay.tolist()) != [0, 1, 2, 3]:
            continue   # a hit fell in a sector gap or outside the plane
        n_full += 1
        expect = [a + int(np.nonzero(lay == l)[0][0]) for l in range(4)]
        assert tr.found[e] == 1 and tr.nhits[e] == 4
        assert list(tr.hit[e]) == expect
        assert abs(tr.qop64[e] - b.qop_true[e]) < 0.05 * abs(b.qop_true[e]) + 2e-3
    assert n_full > 150


def test_windows_hold_exactly_the_hits_in_tolerance():
    b = synth.generate(n_events=6, n_sectors=64, tracks=40, hits=600, seed=51)
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom)
    tr = oracle.compass(hits.x, hits.hit_off, b.n_events, b.geom, oracle.Velo(b), P,
                        want_windows=True)
    g = b.geom
    S, B = g.n_sectors, g.n_banks
    kq = P.kick_k * P.qop_max
    for e in range(b.n_events):
        for t in range(int(b.trk_off[e]), int(b.trk_off[e + 1])):
            if tr.near[t] <= 1e-5:
                continue
            u = [(float(b.velo_x[t]) + float(b.velo_tx[t]) * (float(g.z[l]) - 770.0))
                 - (float(b.velo_y[t]) + float(b.velo_ty[t]) * (float(g.z[l]) - 770.0)) * float(g.tan_stereo[l])
                 for l in range(4)]
            in_acc = g.x_min <= u[0] <= g.x_min + S * 96.0
            for l in range(4):
                c = min(max(int(math.floor((u[l] - g.x_min) / 96.0)), 0), S - 1)
                hw = kq * abs(float(g.z[l]) - P.z_kink) + P.tol_win
                start = int(hits.hit_off[e * B + l * S])
                for k, off in enumerate([0, -1, 1, -2, 2]):
                    s = c + off
                    w = tr.win[t, l, k]
                    if not in_acc or not 0 <= s < S:
                        assert tuple(w) == (-1, -1)
                        continue
                    a, z = int(hits.hit_off[e * B + l * S + s]), int(hits.hit_off[e * B + l * S + s + 1])
                    inside = [j for j in range(a, z) if abs(float(hits.x[j]) - u[l]) <= hw]
                    if not inside:
                        assert tuple(w) == (-1, -1)
                    else:
                        assert inside == list(range(inside[0], inside[-1] + 1))
                        assert tuple(w) == (inside[0] - start, len(inside))


def test_backward_and_out_of_acceptance_tracks_are_skipped():
    b = synth.generate(n_events=5, n_sectors=8, tracks=50, hits=400, seed=61, backward_frac=0.3)
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom)
    tr = oracle.compass(hits.x, hits.hit_off, b.n_events, b.geom, oracle.Velo(b), P,
                        want_windows=True)
    g = b.geom
    u0 = b.velo_x + b.velo_tx * (g.z[0] - 770.0) - (b.velo_y + b.velo_ty * (g.z[0] - 770.0)) * g.tan_stereo[0]
    skip = (b.velo_flags & 1).astype(bool) | (u0 < g.x_min - 1e-3) | (u0 > -g.x_min + 1e-3)
    assert skip.sum() > 10
    assert np.all(tr.found[skip] == 0)
    assert np.all(tr.win[skip] == -1)
    assert np.all(tr.hit[skip] == -1)


def test_zero_field_tracks_have_qop_near_zero():
    b = synth.generate(n_events=20, n_sectors=64, tracks=100, hits=600, seed=71, field=0.0)
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom)
    tr = oracle.compass(hits.x, hits.hit_off, b.n_events, b.geom, oracle.Velo(b), P)
    m = tr.found.astype(bool) & (tr.nhits == 4)
    assert m.sum() > 1000
    z = np.asarray(synth.Z_LAYERS)
    G = np.stack([np.ones(4), z - 770.0, 1.2 * (z - 2500.0)], 1)
    w = 1.0 / P.sigma_hit ** 2
    info = w * G.T @ G + np.diag([1 / P.sigma_x_prior ** 2, 1 / P.sigma_tx_prior ** 2, 0])
    # smearing (pitch/sqrt 12) plus half-strip binning (pitch/2/sqrt 12)
    sig_q = math.sqrt(np.linalg.inv(info)[2, 2]) * math.sqrt(1.25)
    assert np.max(np.abs(tr.qop64[m])) < 6 * sig_q
    assert abs(np.mean(tr.qop64[m])) < 5 * sig_q / math.sqrt(m.sum())


def test_reconstruction_of_generated_tracks_is_reported():
    """Efficiency on synthetic truth (reported, not pinned: the paper's
    figures are on LHCb samples, Table 2)."""
    b = synth.generate_config("tiny")
    hits, tr = oracle.run_batch(b, P)
    assert tr.found.mean() > 0.9
    m = tr.found.astype(bool)
    rel = np.abs(tr.qop64[m] - b.qop_true[m]) / np.abs(b.qop_true[m])
    assert np.median(rel) < 0.05


def test_global_event_cut_skips_busy_events_only():
    """Events with more hits than gec_max_hits are not searched (no found
    tracks, windows -1); every other event's tracks are those of a run
    without the cut."""
    b = synth.generate_config("batched", n_events=30)
    P = synth.CompassParams()
    hits, full = oracle.run_batch(b, P, want_windows=True)
    B = b.geom.n_banks
    ev_hits = np.diff(hits.hit_off[::B].astype(np.int64))
    cut = int(np.median(ev_hits))
    _, gec = oracle.run_batch(b, P.replace(gec_max_hits=cut), want_windows=True)
    busy = np.repeat(ev_hits > cut, np.diff(b.trk_off.astype(np.int64)))
    assert busy.any() and (~busy).any()
    assert not gec.found[busy].any() and np.all(gec.hit[busy] == -1) and np.all(gec.win[busy] == -1)
    assert np.array_equal(gec.x[busy], b.velo_x[busy]) and np.array_equal(gec.tx[busy], b.velo_tx[busy])
    for k in ("hit", "found", "nhits", "win"):
        assert np.array_equal(getattr(gec, k)[~busy], getattr(full, k)[~busy]), k
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(getattr(gec, k)[~busy].view(np.uint32), getattr(full, k)[~busy].view(np.uint32)), k


def test_consolidation_keeps_found_tracks_in_order_with_event_offsets():
    b = synth.generate_config("batched", n_events=25)
    P = synth.CompassParams()
    _, tr = oracle.run_batch(b, P)
    out, off = oracle.consolidate(tr, b.trk_off)
    found = tr.found.astype(bool)
    T = b.n_tracks
    assert off[0] == 0 and off[-1] == found.sum() == out["velo"].size
    assert np.all(np.diff(out["velo"].astype(np.int64)) > 0) and np.all(found[out["velo"]])
    for e in range(b.n_events):  # event e's rows hold exactly its found tracks
        rows = out["velo"][off[e]:off[e + 1]]
        t0, t1 = int(b.trk_off[e]), int(b.trk_off[e + 1])
        assert np.array_equal(rows, np.arange(t0, t1)[found[t0:t1]])
    assert np.array_equal(out["hit"], tr.hit[out["velo"]]) and np.array_equal(out["nhits"], tr.nhits[out["velo"]])
    assert 0 < found.sum() < T
