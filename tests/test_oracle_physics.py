"""Pins of the oracle's step against closed forms and conservation laws:
plane Poiseuille flow with half-way bounce-back (exact LB solution of BGK,
including its viscosity-dependent slip), mass and momentum balance, exact
fixed points, and the decay rate of a shear wave."""
import numpy as np
import pytest


def _nu(omega):
    return (1.0 / omega - 0.5) / 3.0


@pytest.mark.parametrize("omega", [1.0, 1.7, 0.8])
def test_poiseuille_closed_form(ora, omega):
    """Body-force driven flow between walls at y = -1/2 and y = H - 1/2.  The
    BGK solution with half-way bounce-back is the parabola
    u(y_j) = g/(2 nu) ((H/2)^2 - y_j^2) + g (16 Lam - 3) / (24 nu),
    y_j = j - (H-1)/2, Lam = (1/omega - 1/2)^2."""
    H = 16
    dims, per = (2, H, 2), (1, 0, 1)
    gx = 1e-6
    nu = _nu(omega)
    steps = int(40 * H * H / nu / np.pi ** 2) + 2000
    f = ora.run_push(dims, per, None, ora.rest_state(2 * H * 2), steps, omega, (gx, 0, 0), 1)
    rho, u = ora.macroscopics(f, (gx, 0, 0))
    prof = u[:, 0].reshape(2, H, 2, order="F")[0, :, 0]
    lam = (1.0 / omega - 0.5) ** 2
    y = np.arange(H) - (H - 1) / 2.0
    exact = gx / (2 * nu) * ((H / 2.0) ** 2 - y ** 2) + gx * (16 * lam - 3) / (24 * nu)
    assert np.max(np.abs(prof - exact)) / np.max(exact) < 1e-9
    assert np.max(np.abs(u[:, 1:])) < 1e-10 * np.max(exact)  # round-off only
    # permeability of the slit: k = nu <u_x> / g = (H^2 + 8 Lam - 1) / 12
    mass, jx = ora.flux(f, (gx, 0, 0))
    k = ora.permeability(jx, 2 * H * 2, omega, gx)
    assert abs(k - (H * H + 8 * lam - 1) / 12.0) / k < 1e-9


def test_mass_conservation_closed_box(ora):
    dims = (5, 6, 7)
    n = int(np.prod(dims))
    rng = np.random.default_rng(6)
    solid = (rng.random(n) < 0.25).astype(np.uint8)
    f = ora.rest_state(n) * (1 + 0.1 * rng.random((19, n)))
    fl = solid == 0
    m0 = f[:, fl].sum()
    f = ora.run_push(dims, (0, 0, 0), solid, f, 20, 1.4, (1e-4, 0, 0))
    assert abs(f[:, fl].sum() - m0) / m0 < 1e-14


def test_momentum_balance_periodic(ora):
    """On a periodic box without solids the total momentum sum_x sum_i c_i f_i
    grows by g * sum(rho) per step (zero without force)."""
    c, _ = ora.lattice()
    dims = (6, 5, 4)
    n = int(np.prod(dims))
    rng = np.random.default_rng(7)
    f = ora.rest_state(n) * (1 + 0.1 * rng.random((19, n)))
    g = np.array([2e-4, -1e-4, 5e-5])
    for gg in (np.zeros(3), g):
        j0 = (c.T @ f).sum(1)
        m = f.sum()
        f2 = ora.push_full(dims, (1, 1, 1), None, f, 1.3, gg)
        j1 = (c.T @ f2).sum(1)
        assert np.allclose(j1 - j0, gg * m, atol=1e-13)


@pytest.mark.parametrize("u0", [(0, 0, 0), (0.05, -0.03, 0.02)])
def test_uniform_states_are_fixed_points(ora, u0):
    dims = (4, 5, 3)
    n = int(np.prod(dims))
    feq = ora.equilibrium(1.0, u0)
    f = np.repeat(feq[:, None], n, 1)
    out = ora.run_push(dims, (1, 1, 1), None, f, 3, 1.6)
    assert np.max(np.abs(out - f)) < 4e-16  # a few ulps of 1/3


def test_shear_wave_decay(ora):
    """u_x = U sin(2 pi y / L) decays as exp(-nu k^2 t); LB's error is O(k^2)."""
    L = 32
    dims = (2, L, 2)
    n = int(np.prod(dims))
    omega = 1.2
    nu = _nu(omega)
    U = 1e-4
    y = (np.arange(n) // 2) % L
    k = 2 * np.pi / L
    ux = U * np.sin(k * y)
    f = np.stack([ora.equilibrium(1.0, (ux[j], 0, 0)) for j in range(n)], 1)
    t1, t2 = 200, 600
    f1 = ora.run_push(dims, (1, 1, 1), None, f, t1, omega)
    f2 = ora.run_push(dims, (1, 1, 1), None, f1, t2 - t1, omega)
    a1 = ora.macroscopics(f1)[1][:, 0] @ np.sin(k * y)
    a2 = ora.macroscopics(f2)[1][:, 0] @ np.sin(k * y)
    nu_fit = np.log(a1 / a2) / (k * k * (t2 - t1))
    assert abs(nu_fit - nu) / nu < 2 * k * k
