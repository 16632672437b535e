"""Pins of the oracle's geometry and node-list builders against brute force
in plain Python on small boxes, the Boolean-model porosity law on a large
box, and the equality of the sparse (IDX) step with the full-grid step."""
import itertools

import numpy as np
import pytest

from paper_1111_0922_gb300 import inputs


def _brute_mask(dims, per, centres, r, unit):
    out = np.zeros(int(np.prod(dims)), np.uint8)
    for z, y, x in itertools.product(range(dims[2]), range(dims[1]), range(dims[0])):
        p = (x * unit, y * unit, z * unit)
        for c in centres:
            d2 = 0
            for a in range(3):
                d = p[a] - int(c[a])
                if per[a]:
                    L = dims[a] * unit
                    d = min(abs(d - k * L) for k in (-1, 0, 1))
                d2 += d * d
            if d2 <= r * r:
                out[x + dims[0] * (y + dims[1] * z)] = 1
                break
    return out


@pytest.mark.parametrize("per", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
def test_sphere_mask_brute_force(ora, per):
    dims = (9, 7, 8)
    rng = np.random.default_rng(12)
    unit = 16
    centres = np.stack([rng.integers(0, d * unit, 6) for d in dims], 1)
    r = int(2.5 * unit)
    got = ora.sphere_mask(dims, per, centres, r, unit)
    assert np.array_equal(got, _brute_mask(dims, per, centres, r, unit))


def test_sphere_mask_exact_boundary(ora):
    """A cell exactly at distance r is solid; one unit farther is not."""
    unit = 4
    dims = (10, 10, 10)
    c = np.array([[5 * unit, 5 * unit, 5 * unit]])
    m = ora.sphere_mask(dims, (0, 0, 0), c, 3 * unit, unit).reshape(10, 10, 10)
    assert m[5, 5, 8] == 1 and m[5, 5, 9] == 0  # [z, y, x]
    m = ora.sphere_mask(dims, (0, 0, 0), c, 3 * unit - 1, unit).reshape(10, 10, 10)
    assert m[5, 5, 8] == 0


def test_sphere_mask_periodic_wrap(ora):
    unit = 8
    dims = (12, 12, 12)
    c = np.array([[0, 0, 0]])
    m = ora.sphere_mask(dims, (1, 1, 1), c, 2 * unit, unit).reshape(12, 12, 12)
    assert m[0, 0, 11] == 1 and m[11, 11, 11] == 1 and m[0, 0, 10] == 1 and m[0, 0, 9] == 0


def test_porosity_law(ora):
    """Overlapping spheres at uniform centres: porosity = exp(-n v / V) within
    the sampling error and the discretisation of small spheres."""
    dims = (96, 96, 96)
    pack = inputs.sphere_pack(dims, 0.6, radius=8.0, seed=3)
    m = ora.sphere_mask(dims, pack.periodic, pack.centres, pack.radius, pack.unit)
    por = 1.0 - m.mean()
    assert abs(por - 0.6) < 0.02


def test_node_list_and_idx_brute_force(ora):
    c, _ = ora.lattice()
    dims = (5, 4, 6)
    per = (1, 0, 1)
    rng = np.random.default_rng(13)
    n = int(np.prod(dims))
    solid = (rng.random(n) < 0.3).astype(np.uint8)
    cells, node_of = ora.build_nodes(dims, per, solid)
    assert np.array_equal(cells, np.flatnonzero(solid == 0))
    idx = ora.build_idx(dims, per, solid, cells, node_of)
    lookup = {int(cell): k for k, cell in enumerate(cells)}
    for k, cell in enumerate(cells):
        x, y, z = cell % 5, (cell // 5) % 4, cell // 20
        for i in range(1, 19):
            p = [x + c[i, 0], y + c[i, 1], z + c[i, 2]]
            ok = True
            for a in range(3):
                if 0 <= p[a] < dims[a]:
                    continue
                if per[a]:
                    p[a] %= dims[a]
                else:
                    ok = False
            want = -1
            if ok:
                d = p[0] + 5 * (p[1] + 4 * p[2])
                want = lookup.get(d, -1)
            assert idx[i - 1, k] == want


def test_sparse_step_equals_full_step(ora):
    dims = (8, 6, 7)
    per = (1, 0, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(14)
    solid = (rng.random(n) < 0.3).astype(np.uint8)
    f = ora.rest_state(n) * (1 + 0.05 * rng.random((19, n)))
    cells, node_of = ora.build_nodes(dims, per, solid)
    idx = ora.build_idx(dims, per, solid, cells, node_of)
    full = ora.run_push(dims, per, solid, f, 5, 1.1, (1e-4, 0, 0))
    sparse = ora.run_sparse(idx, f[:, cells], 5, 1.1, (1e-4, 0, 0))
    assert np.array_equal(full[:, cells], sparse)


def test_splitmix64_published_vector():
    """SplitMix64 seeded with state 0: first output 0xE220A8397B1DCDAF."""
    assert int(inputs.mix64(np.uint64(0x9E3779B97F4A7C15))) == 0xE220A8397B1DCDAF


def test_uniform_range_and_determinism():
    a = inputs.uniform(7, 1, 100000)
    assert a.min() >= 0.0 and a.max() < 1.0 and abs(a.mean() - 0.5) < 0.005
    assert np.array_equal(a[500:600], inputs.uniform(7, 1, 100, start=500))
    assert not np.array_equal(a[:100], inputs.uniform(7, 2, 100))
