"""Brute-force Compass search in double precision (pins the C oracle).

Independent of the oracle's code: windows are re-derived by scanning every
hit of the event (no bank offsets or window structure), residuals and pair
lines are computed in float64, and the fit is a library least-squares solve
(numpy.linalg.lstsq) of the model with the VELO prior written as two
pseudo-measurements.  Used on tiny events only.

mode "sequential": the first-candidates rule of Sec. V-B (forward pairs in
combined-range order, backward only if forward found nothing, nearest hit in
each collect layer, stop after n_candidates valid tracklets, best = most
hits then lowest chi2 then earliest).
mode "argmin": the global best over every one-hit-per-layer combination that
passes the same cuts (equal to "sequential" when n_candidates is unbounded
and each collect tolerance holds at most one hit).
"""
from __future__ import annotations

import math

import numpy as np


def _fit(d, present, t, f, w, px, ptx):
    rows, rhs = [], []
    sw = math.sqrt(w)
    for l in range(4):
        if present[l]:
            rows.append([sw, sw * t[l], sw * f[l]])
            rhs.append(sw * d[l])
    rows.append([math.sqrt(px), 0.0, 0.0])
    rhs.append(0.0)
    rows.append([0.0, math.sqrt(ptx), 0.0])
    rhs.append(0.0)
    A = np.asarray(rows)
    b = np.asarray(rhs)
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    r = A @ sol - b
    return sol, float(r @ r)


def track_search(x_hits, hit_layer, hit_sector, geom, vx, vy, vtx, vty, backward, p,
                 mode="sequential"):
    """x_hits etc.: all hits of ONE event in stored (sorted) order.

    Returns (hits[4] as positions into x_hits or -1, qop, chi2, nhits).
    """
    # the method receives its constants as float32 values
    p = p.replace(**{k: float(np.float32(getattr(p, k))) for k in (
        "qop_max", "tol_win", "tol_kink", "tol_col", "tol_slope", "chi2ndof_max", "sigma_hit",
        "sigma_x_prior", "sigma_tx_prior", "z_kink", "kick_k")})
    S = geom.n_sectors
    z = [float(v) for v in geom.z]
    tan_a = [float(v) for v in geom.tan_stereo]
    zv = float(geom.z_velo)
    x_min = float(geom.x_min)
    pitch = float(geom.sector_pitch)
    none = ([-1] * 4, 0.0, 0.0, 0)
    if backward:
        return none
    u = []
    for l in range(4):
        dz = z[l] - zv
        u.append((float(vx) + float(vtx) * dz) - (float(vy) + float(vty) * dz) * tan_a[l])
    if u[0] < x_min or u[0] > x_min + S * pitch:
        return none
    kq = p.kick_k * p.qop_max
    hw = [kq * abs(z[l] - p.z_kink) + p.tol_win for l in range(4)]
    slots = [0, -1, 1, -2, 2][: p.n_sectors]
    lists = []
    for l in range(4):
        c = min(max(int(math.floor((u[l] - x_min) / pitch)), 0), S - 1)
        lst = []
        for off in slots:
            s = c + off
            if not 0 <= s < S:
                continue
            for j in range(len(x_hits)):
                if hit_layer[j] == l and hit_sector[j] == s and abs(float(x_hits[j]) - u[l]) <= hw[l]:
                    lst.append(j)
        lists.append(lst)
    if not any(lists):
        return none
    w = 1.0 / p.sigma_hit ** 2
    px = 1.0 / p.sigma_x_prior ** 2
    ptx = 1.0 / p.sigma_tx_prior ** 2
    t = [z[l] - zv for l in range(4)]
    f = [p.kick_k * (z[l] - p.z_kink) for l in range(4)]
    slope_tol = kq + p.tol_slope

    def d_of(l, j):
        return float(x_hits[j]) - u[l]

    best = None   # (key, hits, q, chi2, nh)
    for la, lb, c1, c2 in ((0, 2, 1, 3), (3, 1, 2, 0)):
        count = 0
        cands = []
        for ja in lists[la]:
            for jb in lists[lb]:
                if mode == "sequential" and count >= p.n_candidates:
                    break
                da, db = d_of(la, ja), d_of(lb, jb)
                sr = (db - da) / (z[lb] - z[la])
                if abs(sr) > slope_tol:
                    continue
                if abs(da + sr * (p.z_kink - z[la])) > p.tol_kink:
                    continue
                opts = []
                for lc in (c1, c2):
                    pred = da + sr * (z[lc] - z[la])
                    near = [(abs(d_of(lc, j) - pred), k, j) for k, j in enumerate(lists[lc])
                            if abs(d_of(lc, j) - pred) <= p.tol_col]
                    if mode == "sequential":
                        opts.append([min(near)[2]] if near else [-1])
                    else:
                        opts.append([-1] + [j for _, _, j in near])
                for jc1 in opts[0]:
                    for jc2 in opts[1]:
                        sel = [-1] * 4
                        sel[la], sel[lb], sel[c1], sel[c2] = ja, jb, jc1, jc2
                        nh = sum(1 for v in sel if v >= 0)
                        if nh < 3:
                            continue
                        present = [v >= 0 for v in sel]
                        d = [d_of(l, sel[l]) if sel[l] >= 0 else 0.0 for l in range(4)]
                        sol, chi2 = _fit(d, present, t, f, w, px, ptx)
                        if chi2 / (nh - 1) > p.chi2ndof_max:
                            continue
                        count += 1
                        cands.append(((-nh, chi2, len(cands)), sel, sol[2], chi2, nh))
            if mode == "sequential" and count >= p.n_candidates:
                break
        if cands:
            best = min(cands, key=lambda c: c[0])
            break
    if best is None:
        return none
    return best[1], float(best[2]), best[3], best[4]
