"""Pins of the oracle's sector-group decoding (Sec. IV, Table I): hits
against the generator's truth, the group and row geometry, the order inside
a group, the offsets."""
import numpy as np

import oracle
from synth.grouped import generate_grouped


def _batch(**kw):
    return generate_grouped(6, seed=5, **kw)


def test_every_generated_hit_once_with_its_sensor_and_strip():
    b = _batch()
    gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    n = int(b.bank_n.sum())
    assert gh.x.size == n and gh.group_off[-1] == n
    assert np.array_equal(np.sort(gh.src), np.arange(n))
    ids = gh.id.astype(np.int64)
    R = b.geom.rows
    assert np.array_equal(ids >> 24, b.truth_layer[gh.src])
    assert np.array_equal((ids >> 16) & 0xFF, b.truth_column[gh.src].astype(np.int64) * R + b.truth_row[gh.src])
    half = 2 * (ids & 0x3FF) + ((ids >> 10) & 1)
    assert np.array_equal(half, b.truth_h[gh.src])


def test_positions_rows_and_weights():
    b = _batch()
    g = b.geom
    gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, g)
    col = b.truth_column[gh.src].astype(np.float64)
    lo = g.x_min + col * 96.0
    assert np.all(gh.x >= lo) and np.all(gh.x < lo + 512 * 0.187 + 1e-3)
    assert np.array_equal(gh.z, np.asarray(g.base.z, np.float32)[b.truth_layer[gh.src]])
    r = b.truth_row[gh.src].astype(np.float64)
    assert np.array_equal(gh.y_begin.astype(np.float64), g.y_min + r * g.sensor_height)
    assert np.array_equal(gh.y_end - gh.y_begin, np.full(gh.x.size, np.float32(g.sensor_height)))
    # the track's true y at the plane lies in its hit's strip range
    y = b.truth_y[gh.src]
    sig = ~np.isnan(y)
    assert sig.sum() > 100
    assert np.all((y[sig] >= gh.y_begin[sig]) & (y[sig] < gh.y_end[sig]))
    # weight = 1 / sigma^2 with sigma = pitch / sqrt(12)
    np.testing.assert_allclose(gh.weight, 12.0 / 0.187 ** 2, rtol=1e-6)


def test_groups_hold_their_x_region_and_are_narrow_in_the_centre():
    b = _batch()
    g = b.geom
    e = g.group_edges().astype(np.float64)
    w = np.diff(e)
    half = g.n_groups // 2
    assert np.all(np.diff(w[half:]) > 0) and np.all(np.diff(w[:half]) < 0)   # widening outwards
    assert e[0] == g.x_min and np.isclose(e[-1], -g.x_min)
    gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, g)
    NG = g.n_groups
    for cell in range(b.n_events * 4 * NG):
        a, z = int(gh.group_off[cell]), int(gh.group_off[cell + 1])
        if a == z:
            continue
        k = cell % NG
        l = (cell // NG) % 4
        x = gh.x[a:z].astype(np.float64)
        assert np.all((x >= e[k]) & (x < e[k + 1]) | ((k == NG - 1) & (x >= e[k])))
        assert np.all((gh.id[a:z].astype(np.int64) >> 24) == l)
        yb = gh.y_begin[a:z]
        assert np.all(np.diff(yb) >= 0)
        ties = np.diff(yb) == 0
        assert np.all(np.diff(gh.src[a:z])[ties] > 0)   # stable: raw order among equal yBegin


def test_event_offsets_match_the_banks():
    b = _batch(rows=3, n_groups=10)
    g = b.geom
    gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, g)
    per_event = b.bank_n.reshape(b.n_events, g.n_banks).sum(axis=1)
    assert np.array_equal(np.diff(gh.group_off[np.arange(0, b.n_events * 4 * g.n_groups + 1, 4 * g.n_groups)]),
                          per_event)


def _column_edges(S):
    x_min = -S * 96.0 / 2.0
    return (x_min + 96.0 * np.arange(S + 1)).astype(np.float32)


def test_group_search_reduces_to_the_sector_search():
    """One row of sensors taller than the tracks' y range, one group per
    column, no y cut and no candidate limit: the group search is the sector
    search of orc_compass on the same raw banks (the candidate order inside
    a window differs, which without a candidate limit only matters for exact
    ties: compared by hit position)."""
    import synth
    S = 16
    kw = dict(n_events=10, tracks=60, hits=900, seed=31)
    gb = generate_grouped(n_columns=S, rows=1, sensor_height=10000.0, n_groups=S, edges=_column_edges(S), **kw)
    b0 = synth.generate(n_sectors=S, **kw)
    assert np.array_equal(gb.raw, b0.raw)
    P = synth.CompassParams().replace(n_candidates=100000)
    hits, base = oracle.run_batch(b0, P)
    gh = oracle.decode_groups(gb.raw, gb.ev_off, gb.n_events, gb.geom)
    grp = oracle.compass_groups(gh, gb, P, tol_y=1e6)
    assert np.array_equal(grp.found, base.found) and np.array_equal(grp.nhits, base.nhits)
    assert int(base.found.sum()) > 300
    m = base.hit >= 0
    assert np.array_equal(grp.hit >= 0, m)
    assert np.array_equal(gh.x[grp.hit[m]].view(np.uint32), hits.x[base.hit[m]].view(np.uint32))
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(getattr(grp, k).view(np.uint32), getattr(base, k).view(np.uint32)), k


def test_y_windows_reject_the_other_rows():
    """With sensor rows, hits of the other rows in the searched groups are
    outside a track's y window (the track's y at the plane lies in its own
    strips' range): against the same search without a y cut, more found
    tracks carry their own particle's hits and far fewer are fakes; a y
    window that admits nothing finds nothing."""
    import synth
    gb = generate_grouped(12, rows=4, n_groups=16, tracks=80, hits=2000, seed=33)
    gh = oracle.decode_groups(gb.raw, gb.ev_off, gb.n_events, gb.geom)
    P = synth.CompassParams()
    owner = gb.truth_track[gh.src]

    def score(t):
        m = np.nonzero(t.found)[0]
        good = sum(np.mean(owner[t.hit[tr][t.hit[tr] >= 0]] == tr) >= 0.7 for tr in m)
        return good, len(m) - good

    good_y, fake_y = score(oracle.compass_groups(gh, gb, P, tol_y=5.0))
    good_n, fake_n = score(oracle.compass_groups(gh, gb, P, tol_y=1e6))
    assert good_y > good_n and fake_y < 0.2 * fake_n
    assert not oracle.compass_groups(gh, gb, P, tol_y=-1e6).found.any()


def test_group_search_event_cut_and_constant_kick_map():
    """The Global Event Cut and the kick map act on the group search as on
    the sector search: events above the cut find nothing, and a constant
    map equal to kick_k changes nothing, bit for bit."""
    import synth
    gb = generate_grouped(10, rows=4, n_groups=16, tracks=60, hits=1500, seed=35)
    gh = oracle.decode_groups(gb.raw, gb.ev_off, gb.n_events, gb.geom)
    P = synth.CompassParams()
    base = oracle.compass_groups(gh, gb, P, tol_y=5.0)
    per_event = np.diff(gh.group_off[:: 4 * gb.geom.n_groups].astype(np.int64))
    cutp = P.replace(gec_max_hits=int(np.median(per_event)))
    cut = oracle.compass_groups(gh, gb, cutp, tol_y=5.0)
    over = np.repeat(per_event > cutp.gec_max_hits, np.diff(gb.trk_off.astype(np.int64)))
    assert over.any() and (~over).any()
    assert not cut.found[over].any()
    assert np.array_equal(cut.hit[~over], base.hit[~over])
    km = synth.KickMap(2, 2, 0.3, 0.25, np.full((2, 2), P.kick_k, np.float32))
    same = oracle.compass_groups(gh, gb, P, tol_y=5.0, kick_map=km)
    assert np.array_equal(same.hit, base.hit)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(getattr(same, k).view(np.uint32), getattr(base, k).view(np.uint32)), k
