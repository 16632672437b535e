"""Pins of the oracle's propagation: with the identity collision (omega = 0,
no force) a step is a pure permutation of the (node, direction) slots.  It
must move a marked PDF one cell along its own velocity, bounce it back at
walls, be a bijection, and return to the start after lcm of the periods."""
import math

import numpy as np
import pytest


def _marked(ora, dims, i, cell, value=0.5):
    n = int(np.prod(dims))
    f = ora.rest_state(n)
    f[i, cell] += value
    return f


def _cell(dims, x, y, z):
    return x + dims[0] * (y + dims[1] * z)


def test_one_hot_moves_along_velocity(ora):
    c, w = ora.lattice()
    dims = (5, 6, 7)
    per = (1, 1, 1)
    x0 = (2, 3, 4)
    for i in range(19):
        f = _marked(ora, dims, i, _cell(dims, *x0))
        out = ora.push_full(dims, per, None, f, 0.0)
        delta = out - ora.rest_state(out.shape[1])
        nz = np.argwhere(np.abs(delta) > 0)
        assert nz.shape == (1, 2)
        j, cell = nz[0]
        target = tuple((np.array(x0) + c[i]) % np.array(dims))
        assert j == i and cell == _cell(dims, *target)


def test_wall_bounce_back(ora):
    c, _ = ora.lattice()
    dims = (4, 5, 3)
    per = (1, 0, 1)  # walls beyond y = 0 and y = ny-1
    for i in range(1, 19):
        if c[i, 1] != -1:
            continue
        cell = _cell(dims, 1, 0, 1)
        f = _marked(ora, dims, i, cell)
        out = ora.push_full(dims, per, None, f, 0.0)
        delta = out - ora.rest_state(out.shape[1])
        nz = np.argwhere(np.abs(delta) > 0)
        j = next(k for k in range(19) if np.array_equal(c[k], -c[i]))
        assert [tuple(v) for v in nz] == [(j, cell)]


def test_solid_bounce_back_sparse_and_full(ora):
    c, _ = ora.lattice()
    dims = (5, 5, 5)
    per = (1, 1, 1)
    solid = np.zeros(125, np.uint8)
    solid[_cell(dims, 3, 2, 2)] = 1
    cell = _cell(dims, 2, 2, 2)
    cells, node_of = ora.build_nodes(dims, per, solid)
    idx = ora.build_idx(dims, per, solid, cells, node_of)
    for i in (1, 7, 9, 11, 13):  # all have c_x = +1
        f = _marked(ora, dims, i, cell)
        out = ora.push_full(dims, per, solid, f, 0.0)
        j = next(k for k in range(19) if np.array_equal(c[k], -c[i]))
        if i == 1:
            assert out[j, cell] == f[i, cell]
        fs = ora.push_sparse(idx, f[:, cells], 0.0)
        assert np.array_equal(fs, out[:, cells])


@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 1), (0, 0, 0)])
def test_streaming_is_a_bijection(ora, per):
    dims = (4, 6, 3)
    n = int(np.prod(dims))
    rng = np.random.default_rng(3)
    solid = (rng.random(n) < 0.2).astype(np.uint8)
    f = ora.rest_state(n) * (1 + 0.3 * rng.random((19, n)))
    out = ora.push_full(dims, per, solid, f, 0.0)
    fl = solid == 0
    assert np.array_equal(np.sort(out[:, fl].ravel()), np.sort(f[:, fl].ravel()))


def test_returns_after_lcm_steps(ora):
    dims = (4, 6, 3)
    per = (1, 1, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(4)
    f0 = ora.rest_state(n) * (1 + 0.3 * rng.random((19, n)))
    L = math.lcm(*dims)
    f = ora.run_push(dims, per, None, f0, L, 0.0)
    assert np.array_equal(f, f0)
    f1 = ora.run_push(dims, per, None, f0, L - 1, 0.0)
    assert not np.array_equal(f1, f0)


def test_returns_with_walls(ora):
    """With walls on y (extent 6) every trajectory has period 2*6 = 12, and
    lcm(4, 12, 3) = 12."""
    dims = (4, 6, 3)
    per = (1, 0, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(5)
    f0 = ora.rest_state(n) * (1 + 0.3 * rng.random((19, n)))
    assert np.array_equal(ora.run_push(dims, per, None, f0, 12, 0.0), f0)
