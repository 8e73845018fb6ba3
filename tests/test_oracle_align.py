"""Pins of the oracle's alignment chi2, gradient and refit (the p-kick fit of
Sec. III-C with the selected hits held fixed, in a detector with per-sector
offsets dx, dz and in-plane rotations gamma)."""
import math

import numpy as np
import pytest

import oracle
import synth
from align_ref import reduced_hessian as _reduced_hessian

P = synth.CompassParams()


class _Velo:
    def __init__(self, a, sl=slice(None)):
        self.x, self.y, self.tx, self.ty = a.x[sl], a.y[sl], a.tx[sl], a.ty[sl]


@pytest.fixture(scope="module")
def small():
    a = synth.generate_alignment(2000, 16, seed=5)
    b = a.batch
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=False)
    return a, hits


def test_gradient_matches_central_differences(small):
    a, hits = small
    g = a.batch.geom
    v = _Velo(a)
    rng = np.random.default_rng(1)
    al = a.align_true() + rng.normal(0, [0.01, 0.05, 2e-5], a.align_true().shape)
    th = oracle.align_refit(hits, a.track_hits, g, v, P, al) + rng.normal(0, [1e-3, 1e-6, 1e-3], (a.n_tracks, 3))
    c2, gt, ga, _ = oracle.align_chi2(hits, a.track_hits, g, v, P, al, th)

    def f(al_, th_):
        return oracle.align_chi2(hits, a.track_hits, g, v, P, al_, th_, grads=False)

    steps = np.array([1e-5, 1e-5, 1e-8])
    for gi in rng.choice(al.shape[0], 12, replace=False):
        for k in range(3):
            ap, am = al.copy(), al.copy()
            ap[gi, k] += steps[k]
            am[gi, k] -= steps[k]
            fd = (f(ap, th) - f(am, th)) / (2 * steps[k])
            assert abs(fd - ga[gi, k]) <= 1e-7 * max(abs(ga[gi, k]), 1e-3 * np.abs(ga[:, k]).max()), (gi, k)
    tsteps = np.array([1e-3, 1e-4, 1e-3])   # chi2 is quadratic in theta: large steps, less rounding
    for t in rng.choice(a.n_tracks, 12, replace=False):
        for k in range(3):
            tp, tm = th.copy(), th.copy()
            tp[t, k] += tsteps[k]
            tm[t, k] -= tsteps[k]
            fd = (f(al, tp) - f(al, tm)) / (2 * tsteps[k])
            assert abs(fd - gt[t, k]) <= 1e-7 * max(abs(gt[t, k]), 1e-3 * np.abs(gt[:, k]).max()), (t, k)


def test_refit_is_the_minimiser(small):
    a, hits = small
    g = a.batch.geom
    v = _Velo(a)
    al = a.align_true()
    th = oracle.align_refit(hits, a.track_hits, g, v, P, al)
    _, gt, _, _ = oracle.align_chi2(hits, a.track_hits, g, v, P, al, th)
    # gradients of ~1e5 scale vanish to rounding at the minimum
    assert np.abs(gt[:, 0]).max() < 1e-5 and np.abs(gt[:, 2]).max() < 1e-3
    c_true = oracle.align_chi2(hits, a.track_hits, g, v, P, al, th, grads=False)
    assert abs(c_true / a.n_tracks - 3.0) < 0.3       # ~ndof per track
    th0 = oracle.align_refit(hits, a.track_hits, g, v, P, 0 * al)
    c_nom = oracle.align_chi2(hits, a.track_hits, g, v, P, 0 * al, th0, grads=False)
    assert c_nom > 2 * c_true


def test_nominal_geometry_equals_the_track_fit(small):
    """With no misalignment the aligned chi2 at the refit is the chi2 of the
    double p-kick fit of the same hits (an independently pinned function)."""
    a, hits = small
    g = a.batch.geom
    v = _Velo(a)
    al = np.zeros((4 * g.n_sectors, 3))
    th = oracle.align_refit(hits, a.track_hits, g, v, P, al)
    per_track = np.array([oracle.align_chi2(hits, a.track_hits[t:t + 1], g, _Velo(a, slice(t, t + 1)), P, al,
                                            th[t:t + 1], grads=False) for t in range(200)])
    ref = oracle.fit_tracks(hits.x, g, _Velo(a), a.track_hits[:200], P)
    assert np.allclose(per_track, ref["chi2_64"], rtol=1e-9, atol=1e-9)
    assert np.allclose(th[:200, 2], ref["qop64"], rtol=1e-9, atol=1e-12)


def test_sectors_without_hits_have_exactly_zero_gradient():
    a = synth.generate_alignment(3000, 64, seed=6, plane_covering=False)
    b = a.batch
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=False)
    v = _Velo(a)
    al = a.align_true()
    th = oracle.align_refit(hits, a.track_hits, b.geom, v, P, al)
    _, _, ga, ha = oracle.align_chi2(hits, a.track_hits, b.geom, v, P, al, th)
    used = np.zeros(4 * b.geom.n_sectors, bool)
    h = a.track_hits[a.track_hits >= 0]
    used[hits.layer[h].astype(int) * b.geom.n_sectors + hits.sector[h].astype(int)] = True
    assert (~used).sum() > 20
    assert np.all(ga[~used] == 0.0) and np.all(ha[~used] == 0.0)
    assert np.all(np.abs(ga[used]).sum(axis=1) > 0)


def test_preconditioned_cg_recovers_the_offsets(small):
    """Twenty block-preconditioned CG steps on the reduced Gauss-Newton
    system (re-linearised after ten) recover the injected offsets: the
    observable part (range of the reduced Hessian; three global modes are
    unobservable) within 3 sigma for >= 95% of parameters, sigma from the
    reduced Hessian, and a chi2 below the true alignment's."""
    a, hits = small
    g = a.batch.geom
    v = _Velo(a)
    truth = a.align_true()
    al = np.zeros_like(truth)
    for _ in range(2):
        th = oracle.align_refit(hits, a.track_hits, g, v, P, al)
        _, _, ga, ha = oracle.align_chi2(hits, a.track_hits, g, v, P, al, th)
        H = _reduced_hessian(a, hits, al, th)
        Minv = np.zeros((al.shape[0], 3, 3))
        for s in range(al.shape[0]):
            B = np.array([[ha[s, 0], ha[s, 1], ha[s, 2]], [ha[s, 1], ha[s, 3], ha[s, 4]],
                          [ha[s, 2], ha[s, 4], ha[s, 5]]])
            if B[0, 0] > 0:
                Minv[s] = np.linalg.inv(B)
        M = lambda r: np.einsum("sij,sj->si", Minv, r.reshape(-1, 3)).ravel()
        x = np.zeros(al.size)
        r = -ga.ravel()
        z = M(r)
        p = z.copy()
        rz = r @ z
        for _ in range(10):
            Ap = H @ p
            alpha = rz / (p @ Ap)
            x += alpha * p
            r -= alpha * Ap
            z = M(r)
            rzn = r @ z
            p = z + rzn / rz * p
            rz = rzn
        al = al + x.reshape(-1, 3)
    th = oracle.align_refit(hits, a.track_hits, g, v, P, al)
    c_est = oracle.align_chi2(hits, a.track_hits, g, v, P, al, th, grads=False)
    th_t = oracle.align_refit(hits, a.track_hits, g, v, P, truth)
    c_true = oracle.align_chi2(hits, a.track_hits, g, v, P, truth, th_t, grads=False)
    assert c_est < c_true
    H = _reduced_hessian(a, hits, al, th)
    d = np.sqrt(np.diag(H))
    Hs = H / np.outer(d, d)
    Hp = np.linalg.pinv(Hs, rcond=1e-7, hermitian=True)
    sig = np.sqrt(np.diag(2 * Hp / np.outer(d, d)))
    err = (al - truth).ravel()
    err_obs = (Hp @ (Hs @ (d * err))) / d
    assert np.mean(np.abs(err_obs) / sig <= 3.0) >= 0.95
    # exactly three unobservable global modes
    ev = np.linalg.eigvalsh(Hs)
    assert np.sum(ev < 1e-7 * ev[-1]) == 3
