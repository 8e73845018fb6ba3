"""Pins of the oracle's p-kick fit (Sec. III-C, Sec. V-B).

The model: residual d_l = a + b*t_l + q*f_l against the VELO line, with a
Gaussian prior on (a, b).  Pins: noise-free data on the model (linear and
parabolic kick shapes) return the generating q/p to double rounding with
chi2 = 0; a vanishing prior reduces to the one-parameter closed form
q = sum w f d / sum w f^2; zero field gives q/p = 0; pulls on smeared data
have mean 0 and unit width; the float fit agrees with the double one.
"""
import math

import numpy as np
import pytest

import oracle
import synth

Z = np.asarray(synth.Z_LAYERS)
T = Z - 770.0
K = 1.2
F_LIN = K * (Z - 2500.0)
F_PAR = 1e-3 * np.where(Z > 2500.0, (Z - 2500.0) ** 2, 0.0) - 1e-3 * np.where(Z < 2500.0, (Z - 2500.0) ** 2, 0.0)
P = synth.CompassParams()
W = 1.0 / P.sigma_hit ** 2
PX = 1.0 / P.sigma_x_prior ** 2
PTX = 1.0 / P.sigma_tx_prior ** 2


@pytest.mark.parametrize("basis", [F_LIN, F_PAR], ids=["linear", "parabolic"])
@pytest.mark.parametrize("present", [(1, 1, 1, 1), (1, 0, 1, 1), (1, 1, 1, 0), (0, 1, 1, 1)])
def test_noise_free_recovers_qop_exactly(basis, present):
    for qop in (0.5, -0.2, 0.013, -0.6667):
        d = qop * basis
        ok, delta, chi2 = oracle.fit64_d(d, present, T, basis, W, PX, PTX)
        assert ok
        assert abs(delta[2] - qop) <= 1e-12 * abs(qop)
        assert abs(delta[0]) < 1e-12 and abs(delta[1]) < 1e-15
        assert chi2 < 1e-20


def test_vanishing_prior_is_one_parameter_form():
    """With the (a, b) prior infinitely tight, q = sum w f d / sum w f^2."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        d = rng.normal(0, 2.0, 4)
        ok, delta, _ = oracle.fit64_d(d, (1, 1, 1, 1), T, F_LIN, W, 1e24, 1e30)
        q1 = float(np.sum(W * F_LIN * d) / np.sum(W * F_LIN ** 2))
        assert ok
        assert abs(delta[2] - q1) <= 1e-9 * max(abs(q1), 1e-3)


def test_kick_shape_is_affine_in_t():
    """f = k*(z - z_kink) is affine in t = z - z_velo, so without the VELO
    prior the three columns (1, t, f) are dependent: the prior is needed."""
    G = np.stack([np.ones(4), T, F_LIN], 1)
    assert np.linalg.matrix_rank(G) == 2
    ok, delta, _ = oracle.fit64_d(np.asarray([0.1, 0.2, -0.3, 0.4]), (1, 1, 1, 1), T, F_LIN,
                                  W, PX, PTX)
    assert ok and np.all(np.isfinite(delta))


def test_zero_field_gives_zero_qop():
    ok, delta, chi2 = oracle.fit64_d(np.zeros(4), (1, 1, 1, 1), T, F_LIN, W, PX, PTX)
    assert ok and delta[2] == 0.0 and chi2 == 0.0
    ok, out = oracle.fit32_d(np.zeros(4), (1, 1, 1, 1), T, F_LIN, W, PX, PTX)
    assert ok and out[2] == 0.0 and out[3] == 0.0


def test_pulls_unit_width():
    """1e5 smeared tracks: (q_hat - q)/sigma_q has mean ~0 and RMS ~1, with
    sigma_q the Cramer-Rao width from the model's information matrix."""
    rng = np.random.default_rng(7)
    n = 100_000
    qs = rng.uniform(-0.66, 0.66, n)
    a_true = rng.normal(0, P.sigma_x_prior, n)
    b_true = rng.normal(0, P.sigma_tx_prior, n)
    noise = rng.normal(0, P.sigma_hit, (n, 4))
    G = np.stack([np.ones(4), T, F_LIN], 1)
    info = W * G.T @ G + np.diag([PX, PTX, 0.0])
    sig_q = math.sqrt(np.linalg.inv(info)[2, 2])
    pulls = np.empty(n)
    chi2s = np.empty(n)
    for i in range(n):
        d = a_true[i] + b_true[i] * T + qs[i] * F_LIN + noise[i]
        ok, delta, c2 = oracle.fit64_d(d, (1, 1, 1, 1), T, F_LIN, W, PX, PTX)
        pulls[i] = (delta[2] - qs[i]) / sig_q
        chi2s[i] = c2
    assert abs(pulls.mean()) < 0.02
    assert abs(pulls.std() - 1.0) < 0.02
    # chi2 of a correct linear model has mean = number of data rows - parameters = 4+2-3
    assert abs(chi2s.mean() - 3.0) < 0.05


def test_float_fit_agrees_with_double():
    rng = np.random.default_rng(9)
    worst = 0.0
    for i in range(20_000):
        q = rng.uniform(-0.67, 0.67)
        pres = [(1, 1, 1, 1), (1, 0, 1, 1), (1, 1, 1, 0), (0, 1, 1, 1), (1, 1, 0, 1)][i % 5]
        d = q * F_LIN + rng.normal(0, P.sigma_hit, 4)
        d = np.where(np.asarray(pres) > 0, d, 0.0)
        d32 = d.astype(np.float32)
        ok, ref, c64 = oracle.fit64_d(d32.astype(np.float64), pres, T, F_LIN, W, PX, PTX)
        ok2, out = oracle.fit32_d(d32, pres, T.astype(np.float32), F_LIN.astype(np.float32),
                                  np.float32(W), np.float32(PX), np.float32(PTX))
        assert ok and ok2
        err = abs(float(out[2]) - ref[2]) / max(abs(ref[2]), 1e-2)
        worst = max(worst, err)
        assert abs(float(out[3]) - c64) <= 1e-3 * max(c64, 1.0)
    assert worst < 1e-5, worst
