"""Pins of the oracle's decoding, offsets and sort (Sec. IV, Table I).

Each pin checks the oracle against something other than itself: the
generator's pre-encoding hit list (round trip), the physical hit position
the generator started from (closed form of x), numpy's stable sort, and
hand-built banks with known errors.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _bank_index(b):
    B = b.geom.n_banks
    return (b.truth_event.astype(np.int64) * B + b.truth_layer.astype(np.int64) * b.geom.n_sectors
            + b.truth_sector.astype(np.int64))


@pytest.mark.parametrize("cfg", ["tiny"])
def test_round_trip_unsorted_is_generator_order(cfg):
    b = synth.generate_config(cfg)
    rc, h, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=False)
    assert rc == 0
    assert h.n == b.n_hits
    # bank order, word order inside a bank == the generator's list order
    assert np.array_equal(h.layer, b.truth_layer.astype(np.uint8))
    assert np.array_equal(h.sector, b.truth_sector.astype(np.uint16))
    w = h.id & 0xFFFF
    hh = 2 * (w & 0x3FF) + ((w >> 10) & 1)
    assert np.array_equal(hh, b.truth_h.astype(np.uint32))
    assert np.array_equal(w >> 11, b.truth_flags.astype(np.uint32))
    assert np.array_equal(h.id >> 24, h.layer.astype(np.uint32))
    assert np.array_equal((h.id >> 16) & 0xFF, h.sector.astype(np.uint32) & 0xFF)
    assert np.array_equal(h.z, np.asarray(b.geom.z, np.float32)[h.layer])


def test_offsets_are_exclusive_scan_of_bank_counts():
    b = synth.generate_config("tiny")
    _, h, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=True)
    expect = np.zeros(b.bank_n.size + 1, np.uint64)
    expect[1:] = np.cumsum(b.bank_n.astype(np.uint64))
    assert np.array_equal(h.hit_off.astype(np.uint64), expect)


def test_sorted_is_numpy_stable_sort_per_bank():
    b = synth.generate_config("tiny")
    _, hu, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=False)
    _, hs, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=True)
    key = b.truth_h.astype(np.int64)
    bank = _bank_index(b)
    order = np.lexsort((np.arange(key.size), key, bank))   # stable by (bank, h)
    assert np.array_equal(hs.id, hu.id[order])
    assert np.array_equal(hs.x, hu.x[order])
    # x is non-decreasing inside every bank
    off = hs.hit_off.astype(np.int64)
    dx = np.diff(hs.x)
    same_bank = np.ones(dx.size, bool)
    same_bank[off[1:-1][(off[1:-1] > 0) & (off[1:-1] < hs.n)] - 1] = False
    assert np.all(dx[same_bank] >= 0)


def test_sort_hits_matches_sorted_decode_and_perm_is_bijection():
    b = synth.generate_config("tiny")
    _, hu, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=False)
    _, hs, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=True)
    out, perm = oracle.sort_hits(hu)
    assert np.array_equal(out.id, hs.id) and np.array_equal(out.x, hs.x)
    assert np.array_equal(np.sort(perm), np.arange(hu.n, dtype=np.uint32))
    assert np.array_equal(hu.id[perm], out.id)


def test_x_is_bin_centre_of_the_true_position():
    """Closed form: with smearing off, the generator's true u lies in the
    half-strip bin [x0 + h*hp, x0 + (h+1)*hp) and x is that bin's centre."""
    b = synth.generate(n_events=4, n_sectors=64, tracks=50, hits=None, noise_frac=0.0,
                       seed=11, smear=False, efficiency=1.0)
    _, h, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=False)
    g = b.geom
    tr = b.truth_track
    assert np.all(tr >= 0)
    l = b.truth_layer.astype(np.int64)
    z = np.asarray(synth.Z_LAYERS)[l]
    tan_a = synth.tan_stereo_f32().astype(np.float64)[l]
    vx, vy = b.velo_x[tr].astype(np.float64), b.velo_y[tr].astype(np.float64)
    vtx, vty = b.velo_tx[tr].astype(np.float64), b.velo_ty[tr].astype(np.float64)
    q = b.qop_true[tr].astype(np.float64)
    u = vx + vtx * (z - 770.0) + 1.2 * q * (z - 2500.0) - (vy + vty * (z - 770.0)) * tan_a
    hp = 0.187 / 2
    assert np.max(np.abs(h.x.astype(np.float64) - u)) <= hp / 2 + 2e-4
    # h = 0 sits at x0 + hp/2 and consecutive half-strips are hp apart
    s = h.sector.astype(np.float64)
    x0 = g.x_min + 96.0 * s
    hh = (2 * (h.id & 0x3FF) + ((h.id >> 10) & 1)).astype(np.float64)
    assert np.max(np.abs(h.x - (x0 + (hh + 0.5) * hp))) < 1e-3


def test_x_closed_form_float32_first_half_strip():
    """x(h=0) = x0_s + 0.04675 in float32, for every sector of a 64-sector plane."""
    S = 64
    B = 4 * S
    n = np.zeros((1, B), np.int64)
    n[0, :] = 1
    h = np.zeros(B, np.int64)
    raw, ev_off = synth.encode(n, h, np.zeros(B, np.int64), S)
    geom = synth.Geometry(n_sectors=S)
    _, hits, _ = oracle.decode(raw, ev_off, 1, geom)
    s = np.arange(B) % S
    x0 = np.float32(s).astype(np.float32) * np.float32(96.0) + np.float32(geom.x_min)
    expect = (x0 + np.float32(0.04675)).astype(np.float32)
    assert np.max(np.abs(hits.x - expect)) <= 1e-3
    assert np.all(np.abs(hits.x - x0 - 0.04675) < 1e-3)


def _hand_event(S, counts, words_by_bank):
    B = 4 * S
    n = np.zeros((1, B), np.int64)
    hs, fs = [], []
    for bnk in range(B):
        ws = words_by_bank.get(bnk, [])
        n[0, bnk] = len(ws)
        for w in ws:
            hs.append(2 * (w & 0x3FF) + ((w >> 10) & 1))
            fs.append(w >> 11)
    raw, ev_off = synth.encode(n, np.asarray(hs, np.int64), np.asarray(fs, np.int64), S)
    return raw, ev_off


def test_hand_banks_empty_odd_and_max_strip():
    S = 2
    geom = synth.Geometry(n_sectors=S)
    words = {0: [], 1: [511 | (1 << 10) | (31 << 11)], 2: [5, 3, 5 | (1 << 10)], 7: [0, 0]}
    raw, ev_off = _hand_event(S, None, words)
    rc, h, _ = oracle.decode(raw, ev_off, 1, geom, sorted_=True)
    assert rc == 0
    assert list(h.hit_off) == [0, 0, 1, 4, 4, 4, 4, 4, 6]
    # bank 1: strip 511, frac 1 -> h = 1023, last half-strip of sector 1
    assert h.sector[0] == 1 and h.layer[0] == 0
    assert h.id[0] == (0 << 24) | (1 << 16) | (511 | (1 << 10) | (31 << 11))
    # bank 2 (layer 1, sector 0) sorted by h: 3 (h=6), 5 (h=10), 5|frac (h=11)
    assert [int(v) & 0xFFFF for v in h.id[1:4]] == [3, 5, 5 | (1 << 10)]
    assert np.all(np.diff(h.x[1:4]) > 0)
    # bank 7: two identical words, stable
    assert h.layer[4] == 3 and h.sector[4] == 1 and h.x[4] == h.x[5]


def test_error_strip_512():
    S = 2
    geom = synth.Geometry(n_sectors=S)
    raw, ev_off = _hand_event(S, None, {3: [10, 512, 7]})
    rc, _, where = oracle.decode(raw, ev_off, 1, geom, raise_on_error=False)
    assert rc == -4 and where == (0, 3)


def test_error_source_id_and_directory():
    S = 2
    geom = synth.Geometry(n_sectors=S)
    raw, ev_off = _hand_event(S, None, {1: [1, 2], 4: [3]})
    bad = raw.copy()
    d = bad[4]
    bad[d] = (bad[d] & 0xFFFF) | (5 << 16)     # bank 4 claims to be bank 5
    rc, _, where = oracle.decode(bad, ev_off, 1, geom, raise_on_error=False)
    assert rc == -3 and where == (0, 4)
    bad = raw.copy()
    bad[6] = 10_000                             # bank 6 header outside the event
    rc, _, where = oracle.decode(bad, ev_off, 1, geom, raise_on_error=False)
    assert rc == -2 and where == (0, 6)
    bad = raw.copy()
    d = bad[1]
    bad[d] = (bad[d] & 0xFFFF0000) | 60000      # bank 1 hit words run past the event
    rc, _, where = oracle.decode(bad, ev_off, 1, geom, raise_on_error=False)
    assert rc == -2 and where == (0, 1)


def test_error_lowest_event_bank_wins_and_capacity():
    b = synth.generate_config("tiny")
    bad = b.raw.copy()
    B = b.geom.n_banks
    for e, bank in ((9, 5), (3, 200), (3, 201)):
        base = int(b.ev_off[e])
        d = base + int(bad[base + bank])
        bad[d] = (bad[d] & 0xFFFF) | (((bank + 1) % B) << 16)
    rc, _, where = oracle.decode(bad, b.ev_off, b.n_events, b.geom, raise_on_error=False)
    assert rc == -3 and where == (3, 200)
    rc, _, where = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, capacity=b.n_hits - 1,
                                 raise_on_error=False)
    assert rc == -5
    rc, h, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, capacity=b.n_hits)
    assert rc == 0 and h.n == b.n_hits


def test_empty_batch_and_empty_events():
    geom = synth.Geometry(n_sectors=4)
    n = np.zeros((3, 16), np.int64)
    raw, ev_off = synth.encode(n, np.zeros(0, np.int64), np.zeros(0, np.int64), 4)
    rc, h, _ = oracle.decode(raw, ev_off, 3, geom)
    assert rc == 0 and h.n == 0 and np.all(h.hit_off == 0)
    rc, h, _ = oracle.decode(raw, ev_off[:1], 0, geom)
    assert rc == 0 and h.n == 0
