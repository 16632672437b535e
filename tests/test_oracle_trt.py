"""Pins of the oracle's two-relaxation-time collision: with equal rates it is
BGK; it conserves mass and adds exactly rho g of momentum; and with the magic
parameter Lam = 3/16 the bounce-back walls of plane Poiseuille flow sit
exactly half-way, so the steady profile is the parabola
u(y_j) = g/(2 nu) ((H/2)^2 - y_j^2) with no slip term, for any viscosity."""
import numpy as np
import pytest


def test_equal_rates_is_bgk(ora):
    _, w = ora.lattice()
    rng = np.random.default_rng(3)
    f = w * (1 + 0.1 * rng.random(19))
    g = (1e-3, -2e-3, 5e-4)
    for om in (0.7, 1.0, 1.6):
        assert np.allclose(ora.collide_trt(f, om, om, g), ora.collide(f, om, g), rtol=0, atol=1e-16)


def test_trt_conservation(ora):
    c, w = ora.lattice()
    rng = np.random.default_rng(4)
    f = w * (1 + 0.2 * rng.random(19))
    g = np.array([2e-3, 1e-3, -1e-3])
    for lp, lm in ((1.0, 1.7), (0.6, 1.2), (1.9, 0.8)):
        fs = ora.collide_trt(f, lp, lm, g)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert np.allclose(c.T @ fs - c.T @ f, f.sum() * g, atol=1e-16, rtol=1e-12)


@pytest.mark.parametrize("omega", [0.8, 1.0, 1.7])
def test_trt_poiseuille_exact_walls(ora, omega):
    H = 12
    dims, per = (2, H, 2), (1, 0, 1)
    gx = 1e-6
    lm = ora.trt_lambda_minus(omega, 3.0 / 16.0)
    nu = (1.0 / omega - 0.5) / 3.0
    steps = int(40 * H * H / nu / np.pi ** 2) + 2000
    f = ora.run_push_trt(dims, per, None, ora.rest_state(2 * H * 2), steps, omega, lm, (gx, 0, 0), 1)
    _, u = ora.macroscopics(f, (gx, 0, 0))
    prof = u[:, 0].reshape(2, H, 2, order="F")[0, :, 0]
    y = np.arange(H) - (H - 1) / 2.0
    exact = gx / (2 * nu) * ((H / 2.0) ** 2 - y ** 2)
    assert np.max(np.abs(prof - exact)) / np.max(exact) < 1e-9
