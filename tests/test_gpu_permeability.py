"""Permeability of a sphere pack run to a steady flux: CUDA path against the
oracle, same geometry, same convergence rule (rounds of 100 steps, relative
flux change < 1e-6).  Tolerances on k: FP64 1e-10, FP32 1e-5, FP16 storage
1e-3."""
import numpy as np
import pytest

import oracle
from paper_1111_0922_gb300 import inputs, permeability

pytestmark = pytest.mark.gpu

DIMS, PER = (32, 32, 32), (1, 1, 1)
OMEGA, GX = 1.0, 1e-6
TOL_K = {"f64": 1e-10, "f32": 1e-5, "f16s": 1e-3}


@pytest.fixture(scope="module")
def pack_and_oracle():
    pack = inputs.sphere_pack(DIMS, 0.6, radius=4.0, seed=11)
    mask = oracle.sphere_mask(DIMS, PER, pack.centres, pack.radius, pack.unit)
    cells, node_of = oracle.build_nodes(DIMS, PER, mask)
    idx = oracle.build_idx(DIMS, PER, mask, cells, node_of)
    f = oracle.rest_state(cells.size)
    prev, steps = None, 0
    while steps < 200000:
        _, phi = oracle.flux(f, (GX, 0, 0))  # state at the start of the round
        f = oracle.run_sparse(idx, f, 100, OMEGA, (GX, 0, 0))
        steps += 100
        if prev is not None and abs(phi - prev) < 1e-6 * abs(phi):
            break
        prev = phi
    k = oracle.permeability(phi, int(np.prod(DIMS)), OMEGA, GX)
    return pack, k, steps


@pytest.mark.parametrize("variant,precision", [("aa", "f64"), ("aa", "f32"), ("et", "f32"),
                                               ("aa", "f16s"), ("et", "f16s"), ("os_pull", "f32")])
def test_permeability_matches_oracle(pack_and_oracle, variant, precision):
    from paper_1111_0922_gb300 import build, lbm

    build.build()
    pack, k_ora, steps_ora = pack_and_oracle
    lat = lbm.Lattice(DIMS, PER, variant=variant, addressing="indirect", precision=precision,
                      omega=OMEGA, force=(GX, 0, 0))
    lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
    lat.init()
    res = permeability.solve(lat)
    lat.close()
    assert res.converged
    assert abs(res.k - k_ora) <= TOL_K[precision] * k_ora, (res.k, k_ora)
    if precision != "f16s":
        assert abs(res.steps - steps_ora) <= 100
