"""Pins of the oracle's velocity set, weights, equilibrium and collision
against identities fixed by the mathematics of D3Q19 (not by the oracle's own
code): lattice moment isotropy, equilibrium moments, and the exact momentum
change of BGK with the Guo force term."""
import numpy as np
import pytest


def test_velocity_set_isotropy(ora):
    c, w = ora.lattice()
    assert c.shape == (19, 3)
    # every velocity has at most two nonzero unit components; all 19 distinct
    assert len({tuple(v) for v in c}) == 19
    assert np.all(np.abs(c) <= 1) and np.all(np.sum(np.abs(c), 1) <= 2)
    assert tuple(c[0]) == (0, 0, 0)
    # opposite pairs: c_{i+1} = -c_i for odd i
    for i in range(1, 19, 2):
        assert np.array_equal(c[i + 1], -c[i])
    # moments of the weights (D3Q19, c_s^2 = 1/3)
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(3):
        assert abs(np.dot(w, c[:, a])) < 1e-16
        for b in range(3):
            m2 = np.dot(w, c[:, a] * c[:, b])
            assert abs(m2 - (1.0 / 3.0 if a == b else 0.0)) < 1e-15
            for d in range(3):
                assert abs(np.dot(w, c[:, a] * c[:, b] * c[:, d])) < 1e-16
    # fourth moment: sum w c_a^2 c_b^2 = 1/9 (a != b), sum w c_a^4 = 1/3
    for a in range(3):
        assert abs(np.dot(w, c[:, a] ** 4) - 1.0 / 3.0) < 1e-15
        for b in range(3):
            if a != b:
                assert abs(np.dot(w, c[:, a] ** 2 * c[:, b] ** 2) - 1.0 / 9.0) < 1e-15
    # the stated order: rest, +x -x +y -y +z -z, then the diagonals
    assert [tuple(v) for v in c[1:7]] == [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                          (0, 0, 1), (0, 0, -1)]
    assert np.all(np.sum(np.abs(c[7:]), 1) == 2)


@pytest.mark.parametrize("rho,u", [(1.0, (0, 0, 0)), (1.03, (0.05, -0.02, 0.01)),
                                   (0.97, (-0.1, 0.07, 0.03))])
def test_equilibrium_moments(ora, rho, u):
    c, _ = ora.lattice()
    u = np.array(u, float)
    feq = ora.equilibrium(rho, u)
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
    # second moment of the second-order equilibrium: rho (u u + I/3)
    pi = np.einsum("i,ia,ib->ab", feq, c, c)
    assert np.allclose(pi, rho * (np.outer(u, u) + np.eye(3) / 3.0), atol=1e-14)


def test_collision_conserves_mass_and_adds_force(ora):
    c, w = ora.lattice()
    rng = np.random.default_rng(1)
    for omega in (0.6, 1.0, 1.7):
        f = w * (1.0 + 0.2 * rng.random(19))
        g = np.array([1e-3, -2e-3, 5e-4])
        fs = ora.collide(f, omega, g)
        rho = f.sum()
        # sum c_i F_i = (1 - omega/2) rho g and the BGK part moves j to rho u,
        # u = (j + rho g / 2)/rho: together the momentum grows by exactly rho g
        assert abs(fs.sum() - rho) < 1e-15
        assert np.allclose(c.T @ fs - c.T @ f, rho * g, atol=1e-16, rtol=1e-12)


def test_collision_relaxes_nonequilibrium(ora):
    """Without force the post-collision state is feq + (1 - omega)(f - feq)."""
    c, w = ora.lattice()
    rng = np.random.default_rng(2)
    f = w * (1.0 + 0.1 * rng.random(19))
    rho = f.sum()
    u = (c.T @ f) / rho
    feq = ora.equilibrium(rho, u)
    for omega in (0.5, 1.0, 1.9):
        fs = ora.collide(f, omega)
        assert np.allclose(fs, feq + (1 - omega) * (f - feq), atol=1e-16, rtol=1e-13)


def test_identity_collision(ora):
    _, w = ora.lattice()
    f = w * np.linspace(0.9, 1.1, 19)
    assert np.array_equal(ora.collide(f, 0.0), f)
