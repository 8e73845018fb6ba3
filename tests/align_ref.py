"""Dense reduced Gauss-Newton Hessian of the alignment chi2 (test helper).

Built from the model's per-hit derivatives (the same model as the oracle's
alignment chi2) with each track's states profiled out:
H = sum_t [2w JA^T JA - Hta^T Htt^-1 Hta].  Small problems only."""
import math

import numpy as np

import synth

P = synth.CompassParams()


def reduced_hessian(a, hits, al, th):
    """Reduced Gauss-Newton Hessian (track states profiled out), assembled
    densely from per-hit derivatives of the model (small problems only)."""
    g = a.batch.geom
    S = g.n_sectors
    NA = 12 * S
    w = 1 / np.float32(P.sigma_hit) ** 2
    k = float(np.float32(P.kick_k))
    px = 1 / np.float32(P.sigma_x_prior) ** 2
    ptx = 1 / np.float32(P.sigma_tx_prior) ** 2
    H = np.zeros((NA, NA))
    for t in range(a.n_tracks):
        Jt, JA = [], []
        for l in range(4):
            h = a.track_hits[t, l]
            if h < 0:
                continue
            gi = int(hits.layer[h]) * S + int(hits.sector[h])
            z = float(g.z[l]) + al[gi, 1]
            y = a.y[t] + a.ty[t] * (z - g.z_velo)
            ta, tg = float(g.tan_stereo[l]), math.tan(al[gi, 2])
            T = (ta + tg) / (1 - ta * tg)
            Jt.append([-1.0, -(z - g.z_velo), -k * (z - P.z_kink)])
            row = np.zeros(NA)
            row[3 * gi:3 * gi + 3] = [1.0, a.ty[t] * T - th[t, 1] - k * th[t, 2], y * (1 + T * T)]
            JA.append(row)
        Jt, JA = np.asarray(Jt), np.asarray(JA)
        Htt = 2 * w * Jt.T @ Jt + np.diag([2 * px, 2 * ptx, 0.0])
        Hta = 2 * w * Jt.T @ JA
        H += 2 * w * JA.T @ JA - Hta.T @ np.linalg.solve(Htt, Hta)
    return H
