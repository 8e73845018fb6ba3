"""Pin of the oracle's extrapolation (Sec. V-A): the float pair (hi, lo)
that carries the straight VELO line's measured coordinate
u_l = x + tx dz - (y + ty dz) tan(a_l), dz = z_l - z_velo, is within a few
units of 2^-48 of the exact value (rational arithmetic on the float
inputs), and lo is below hi's last place: the pair is as good as a double
prediction for every float decision."""
from fractions import Fraction

import numpy as np

import oracle
import synth


def test_pair_is_the_exact_prediction_to_2_pow_minus_45():
    g = synth.Geometry(n_sectors=256)
    rng = np.random.default_rng(11)
    f32 = np.float32
    worst = 0.0
    for _ in range(400):
        x, y = f32(rng.normal(0, 200)), f32(rng.normal(0, 200))
        tx, ty = f32(rng.uniform(-0.3, 0.3)), f32(rng.uniform(-0.25, 0.25))
        hi, lo = oracle.extrapolate(g, x, y, tx, ty)
        for l in range(4):
            dz = f32(f32(g.z[l]) - f32(g.z_velo))
            t = f32(g.tan_stereo[l])
            xv = Fraction(float(x)) + Fraction(float(tx)) * Fraction(float(dz))
            yv = Fraction(float(y)) + Fraction(float(ty)) * Fraction(float(dz))
            u = xv - yv * Fraction(float(t))
            err = abs(Fraction(float(hi[l])) + Fraction(float(lo[l])) - u)
            scale = abs(xv) + abs(yv * Fraction(float(t))) + 1
            worst = max(worst, float(err / scale))
            assert abs(float(lo[l])) <= float(np.spacing(np.abs(hi[l])))
    assert worst <= 2.0 ** -45, worst


def test_zero_direction_and_zero_position():
    """A track along z through the origin lies on u = 0 exactly; a track
    with tx = ty = 0 at (x, y) predicts u = x - y tan exactly in the
    unrotated layers."""
    g = synth.Geometry(n_sectors=64)
    hi, lo = oracle.extrapolate(g, 0.0, 0.0, 0.0, 0.0)
    assert np.all(hi == 0) and np.all(lo == 0)
    hi, lo = oracle.extrapolate(g, 123.25, 40.0, 0.0, 0.0)
    assert hi[0] == np.float32(123.25) and lo[0] == 0 and hi[3] == np.float32(123.25) and lo[3] == 0
