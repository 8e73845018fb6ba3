"""Pins of the oracle's kick map (Sec. III-C: look-up tables give the
deflection a track is expected to get): the interpolation against closed
forms, the constant map against the constant kick, and q/p and efficiency
against the generator's direction-dependent field."""
import numpy as np

import oracle
import synth
from paper_2002_11529_gb300 import physics

P = synth.CompassParams()


def _affine_map(nx=9, ny=7, tx_max=0.3, ty_max=0.25):
    # bilinear in (tx, ty): interpolation on any grid reproduces it exactly
    # up to float rounding
    fn = lambda tx, ty: 1.1 + 0.5 * tx - 0.8 * ty + 2.0 * tx * ty + 0.0 * tx * ty
    return synth.kick_map(nx, ny, tx_max, ty_max, fn=fn), fn


def test_interpolation_reproduces_a_bilinear_field():
    km, fn = _affine_map()
    rng = np.random.default_rng(3)
    tx = rng.uniform(-0.3, 0.3, 500).astype(np.float32)
    ty = rng.uniform(-0.25, 0.25, 500).astype(np.float32)
    got = oracle.kick_at(P, km, tx, ty).astype(np.float64)
    want = fn(tx.astype(np.float64), ty.astype(np.float64))
    assert np.max(np.abs(got - want) / np.abs(want)) < 2e-6


def test_corner_and_clamping():
    km = synth.kick_map(5, 4)
    assert oracle.kick_at(P, km, [-0.3], [-0.25])[0] == km.values[0, 0]
    # outside the grid the coordinates are clamped: same value as on the edge
    for tx, ty, ex, ey in ((0.9, 0.1, 0.3, 0.1), (-2.0, -0.1, -0.3, -0.1), (0.1, 3.0, 0.1, 0.25)):
        assert oracle.kick_at(P, km, [tx], [ty])[0] == oracle.kick_at(P, km, [ex], [ey])[0]


def test_interpolation_is_between_the_cell_corners():
    km = synth.kick_map(17, 17)
    rng = np.random.default_rng(4)
    tx = rng.uniform(-0.3, 0.3, 300).astype(np.float32)
    ty = rng.uniform(-0.25, 0.25, 300).astype(np.float32)
    k = oracle.kick_at(P, km, tx, ty)
    assert k.min() >= km.values.min() * (1 - 1e-6) and k.max() <= km.values.max() * (1 + 1e-6)
    # the sampled field is close to the field itself (smooth on a 17 x 17 grid)
    true = synth.field_kick(tx, ty)
    assert np.max(np.abs(k - true) / true) < 2e-3


def test_constant_map_equals_the_constant_kick():
    b = synth.generate_config("tiny", seed=11)
    km = synth.KickMap(3, 3, 0.3, 0.25, np.full((3, 3), P.kick_k, np.float32))
    _, a = oracle.run_batch(b, P, want_windows=True)
    _, c = oracle.run_batch(b, P, want_windows=True, kick_map=km)
    assert np.array_equal(a.hit, c.hit) and np.array_equal(a.win, c.win)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(getattr(a, k).view(np.uint32), getattr(c, k).view(np.uint32)), k
    assert np.array_equal(a.qop64, c.qop64)


def _fieldmap_batch(n=40):
    return synth.generate_config("fieldmap", n_events=n)


def test_map_recovers_qop_in_a_direction_dependent_field():
    b = _fieldmap_batch()
    km = synth.kick_map()
    _, with_map = oracle.run_batch(b, P, kick_map=km)
    _, no_map = oracle.run_batch(b, P)
    truth = b.qop_true.astype(np.float64)
    kratio = synth.field_kick(b.velo_tx, b.velo_ty) / P.kick_k
    sel = (with_map.nhits == 4) & (no_map.nhits == 4) & (np.abs(truth) > 0.2)
    assert sel.sum() > 200
    r_map = with_map.qop[sel] / truth[sel]
    r_none = no_map.qop[sel] / truth[sel]
    assert abs(np.median(r_map) - 1.0) < 0.02
    # the constant kick is off by the field's ratio, track by track
    assert abs(np.median(r_none / kratio[sel]) - 1.0) < 0.02
    assert np.median(np.abs(r_map - 1.0)) < 0.5 * np.median(np.abs(r_none - 1.0))
    # the double fit is converted the same way
    rel = np.abs(with_map.qop[sel] - with_map.qop64[sel]) / np.abs(with_map.qop64[sel])
    assert rel.max() < 1e-5


def test_map_widens_windows_where_the_field_is_stronger():
    b = _fieldmap_batch()
    km = synth.kick_map()
    _, with_map = oracle.run_batch(b, P, kick_map=km)
    _, no_map = oracle.run_batch(b, P)
    e_map = physics.evaluate(b, {"hit": with_map.hit, "found": with_map.found})["efficiency"]
    e_none = physics.evaluate(b, {"hit": no_map.hit, "found": no_map.found})["efficiency"]
    assert e_map > e_none + 0.005


def test_fit_tracks_converts_qop_with_the_map():
    b = _fieldmap_batch(10)
    km = synth.kick_map()
    hits, tr = oracle.run_batch(b, P, kick_map=km)
    ref = oracle.fit_tracks(hits.x, b.geom, oracle.Velo(b), tr.hit, P, kick_map=km)
    m = tr.found.astype(bool)
    for k in ("qop", "chi2", "x", "tx"):
        assert np.array_equal(ref[k][m].view(np.uint32), getattr(tr, k)[m].view(np.uint32)), k
    plain = oracle.fit_tracks(hits.x, b.geom, oracle.Velo(b), tr.hit, P)
    k = oracle.kick_at(P, km, b.velo_tx, b.velo_ty)
    np.testing.assert_array_equal(ref["qop"][m], plain["qop"][m] * (np.float32(P.kick_k) / k[m]))
