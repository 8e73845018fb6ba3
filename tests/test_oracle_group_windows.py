"""Exact pins of the group search's candidate windows (Sec. V-A with the
sector groups of Sec. IV): the oracle finds a track's candidates in a group
by two binary searches over the y-sorted hits, then refines them by the x
window.  Here every hit of the searched groups is scanned instead and kept
when yEnd >= y - tol_y, yBegin <= y + tol_y and |d| <= hw, each comparison
in float as the search states it.  The two lists must be equal, entry for
entry, at several tol_y, and when y - tol_y or y + tol_y falls exactly on a
row boundary (a strict comparison, or yBegin read for yEnd, fails there)."""
import numpy as np
import pytest

import oracle
import synth
from synth.grouped import generate_grouped

f32, f64 = np.float32, np.float64
SLOTS = (0, -1, 1, -2, 2)


def scan_candidates(gh, batch, params, tol_y, vy, vty):
    """Candidates of every track by a scan of every hit of the searched
    groups (float comparisons; the prediction in double)."""
    gg = batch.geom
    base = gg.base
    NG = gg.n_groups
    edges = np.asarray(gg.group_edges(), f32)
    S = gg.n_columns
    x_min = f64(f32(gg.x_min))
    x_max = x_min + f64(S) * f64(f32(base.sector_pitch))
    z = np.asarray(base.z, f32)
    kq = f32(params.kick_k) * f32(params.qop_max)
    hw = [kq * f32(abs(f32(z[l]) - f32(params.z_kink))) + f32(params.tol_win) for l in range(4)]
    out = []
    for e in range(batch.n_events):
        for tr in range(int(batch.trk_off[e]), int(batch.trk_off[e + 1])):
            lists = [[] for _ in range(4)]
            if batch.velo_flags[tr] & 1:
                out.append(lists)
                continue
            y0, ty = f64(f32(vy[tr])), f64(f32(vty[tr]))
            # the prediction (pinned on its own in test_oracle_extrapolate.py)
            hi, lo = oracle.extrapolate(base, batch.velo_x[tr], vy[tr], batch.velo_tx[tr], vty[tr])
            u = [f64(hi[l]) + f64(lo[l]) for l in range(4)]
            if not (x_min <= u[0] <= x_max):
                out.append(lists)
                continue
            for l in range(4):
                dz = f64(z[l]) - f64(f32(base.z_velo))
                y = f32(y0 + ty * dz)
                ylo, yhi = f32(y - f32(tol_y)), f32(y + f32(tol_y))
                c = sum(1 for k in range(1, NG) if f64(edges[k]) <= u[l])
                for k in range(params.n_sectors):
                    grp = c + SLOTS[k]
                    if grp < 0 or grp >= NG:
                        continue
                    cell = (e * 4 + l) * NG + grp
                    for j in range(int(gh.group_off[cell]), int(gh.group_off[cell + 1])):
                        if not (gh.y_end[j] >= ylo and gh.y_begin[j] <= yhi):
                            continue
                        d = f32(f32(gh.x[j] - hi[l]) - lo[l])
                        if d >= -hw[l] and d <= hw[l]:
                            lists[l].append(j)
            out.append(lists)
    return out


def _compare(gh, batch, params, tol_y, vy=None, vty=None):
    vy = batch.velo_y if vy is None else vy
    vty = batch.velo_ty if vty is None else vty
    cand, n = oracle.group_candidates(gh, batch, params, tol_y=tol_y, vy=vy, vty=vty)
    ref = scan_candidates(gh, batch, params, tol_y, vy, vty)
    assert len(ref) == n.shape[0]
    total = 0
    for tr, lists in enumerate(ref):
        for l in range(4):
            got = cand[tr, l, : n[tr, l]].tolist()
            assert got == lists[l], (tr, l, tol_y)
            total += len(got)
    return total


@pytest.fixture(scope="module")
def grouped():
    b = generate_grouped(6, rows=4, n_groups=16, tracks=40, hits=900, seed=41)
    gh = oracle.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    return b, gh


@pytest.mark.parametrize("tol_y", [0.0, 2.5, 40.0, 250.0, 1e6, -1.0, -300.0])
def test_candidates_equal_a_scan_of_the_searched_groups(grouped, tol_y):
    b, gh = grouped
    total = _compare(gh, b, synth.CompassParams(), tol_y)
    if tol_y > -250.0:
        assert total > 100    # (tol_y = -1: rows that reach 1 mm beyond y on both sides)
    else:
        assert total == 0     # no row of 250 mm is 300 mm beyond y on both sides


@pytest.mark.parametrize("n_sectors", [1, 3])
def test_candidates_with_fewer_groups(grouped, n_sectors):
    b, gh = grouped
    _compare(gh, b, synth.CompassParams(n_sectors=n_sectors), 30.0)


def test_y_cuts_inclusive_on_row_boundaries(grouped):
    """Tracks flat in y (ty = 0) at y = 130 mm: with tol_y = 130, y - tol_y
    is exactly 0, the yEnd of the row [-250, 0) and the yBegin of [0, 250);
    at y = 120, y + tol_y is exactly 250, the yBegin of the row [250, 500).
    Both boundary rows are in the window (yEnd >= ylo, yBegin <= yhi)."""
    b, gh = grouped
    T = b.n_tracks
    vty = np.zeros(T, f32)
    P = synth.CompassParams()
    for y, edge in ((130.0, 0.0), (120.0, 250.0)):
        vy = np.full(T, y, f32)
        _compare(gh, b, P, 130.0, vy, vty)
        cand, n = oracle.group_candidates(gh, b, P, tol_y=130.0, vy=vy, vty=vty)
        sel = np.concatenate([cand[tr, l, : n[tr, l]] for tr in range(T) for l in range(4)])
        # the boundary row is among the candidates: a hit whose yEnd (y = 130)
        # or yBegin (y = 120) lies exactly on the cut
        if y == 130.0:
            assert np.any(gh.y_end[sel] == f32(0.0))
        else:
            assert np.any(gh.y_begin[sel] == f32(250.0))


def test_search_selects_among_its_candidates(grouped):
    """The selected hits of the group search are candidates of their track
    and layer; tracks without candidates find nothing."""
    b, gh = grouped
    P = synth.CompassParams()
    res = oracle.compass_groups(gh, b, P, tol_y=10.0)
    cand, n = oracle.group_candidates(gh, b, P, tol_y=10.0)
    assert res.found.sum() > 50
    for tr in range(b.n_tracks):
        if not res.found[tr]:
            continue
        for l in range(4):
            h = res.hit[tr, l]
            if h >= 0:
                assert h in cand[tr, l, : n[tr, l]]
    assert not res.found[n.sum(axis=1) == 0].any()


def test_unsorted_group_is_refused(grouped):
    """A group whose yEnd decreases (sensors of different heights) breaks
    the binary search's precondition: the oracle refuses it."""
    b, gh = grouped
    import dataclasses
    ye = gh.y_end.copy()
    cells = np.nonzero(np.diff(gh.group_off.astype(np.int64)) >= 2)[0]
    a = int(gh.group_off[cells[0]])
    ye[a] = ye[a + 1] + f32(1.0)
    bad = dataclasses.replace(gh, y_end=ye)
    with pytest.raises(oracle.OracleError):
        oracle.group_candidates(bad, b, synth.CompassParams(), tol_y=10.0)
    with pytest.raises(oracle.OracleError):
        oracle.compass_groups(bad, b, synth.CompassParams(), tol_y=10.0)


def test_near_cut_margin_sees_the_y_cut(grouped):
    """The y decisions enter a track's smallest decision margin: a track
    whose y window ends exactly on a row boundary has margin 0."""
    b, gh = grouped
    T = b.n_tracks
    vy = np.full(T, 130.0, f32)
    vty = np.zeros(T, f32)
    P = synth.CompassParams()
    res = oracle.compass_groups(gh, b, P, tol_y=130.0, vy=vy, vty=vty)
    cand, n = oracle.group_candidates(gh, b, P, tol_y=130.0, vy=vy, vty=vty)
    searched = n.sum(axis=1) > 0
    on_cut = np.array([any(np.any(gh.y_end[cand[tr, l, : n[tr, l]]] == f32(0.0)) for l in range(4))
                       for tr in range(T)])
    assert on_cut.sum() > 0.5 * searched.sum()
    assert np.all(res.near[on_cut] == 0.0)
    far = oracle.compass_groups(gh, b, P, tol_y=10.0, vy=np.full(T, 125.0, f32), vty=vty)
    assert np.all(far.near[searched] > 0.0)


@pytest.mark.parametrize("n_sectors", [1, 3])
def test_group_choice_on_an_edge(grouped, n_sectors):
    """Straight tracks along z (tx = ty = 0, y = 0) at x exactly on a group
    edge: in the unrotated layers 0 and 3 the prediction u equals the edge,
    which belongs to the group on its right (edges[k] <= u).  Tracks at
    x_min and at x_max exactly are inside the plane."""
    b, gh = grouped
    T = b.n_tracks
    gg = b.geom
    edges = np.asarray(gg.group_edges(), f32)
    xs = np.concatenate([edges[1:-1], [f32(gg.x_min), f32(gg.x_min + gg.n_columns * 96.0)]]).astype(f32)
    vx = xs[np.arange(T) % xs.size]
    z = np.zeros(T, f32)
    import dataclasses
    flat = dataclasses.replace(b, velo_x=vx, velo_tx=z, velo_flags=np.zeros(T, np.uint8))
    P = synth.CompassParams(n_sectors=n_sectors)
    assert _compare(gh, flat, P, 1e6, z, z) > 100
    cand, n = oracle.group_candidates(gh, flat, P, tol_y=1e6, vy=z, vty=z)
    # the tracks at x_min are accepted: their layer-0 group 0 holds hits
    # within hw of the plane's edge
    at_min = vx == f32(gg.x_min)
    assert at_min.any() and np.all(n[at_min].sum(axis=1) > 0)
