"""Full-size parity of the sparse workload: the periodic 512^3 box of
overlapping spheres (r = 8, porosity 0.6, seed 3; 80.5 M fluid nodes), node
list, AA pattern and esoteric twist, FP32 and FP16 storage, in the launch
shape the benchmark times.  The state starts from rho = 1 + 1e-3 U[-1,1) on
every fluid node (seed 2) with g = 1e-6 along x and omega 1.0; after four
steps, sampled nodes are compared with the oracle run on the 9^3
neighbourhood of each (four steps cannot reach the wrap of a 9^3 patch)."""
import numpy as np
import pytest

import oracle
from paper_1111_0922_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS = (512, 512, 512)
STEPS = 4
G = (1e-6, 0.0, 0.0)
TOL_U = {"f32": 1e-5, "f16s": 2e-3}


@pytest.fixture(scope="module")
def setup():
    import torch

    from paper_1111_0922_gb300 import build
    from paper_1111_0922_gb300 import lbm as L

    assert torch.cuda.is_available()
    build.build()
    L.load()
    pack = inputs.sphere_pack(DIMS, 0.6, radius=8.0, seed=3)
    mask = oracle.sphere_mask(DIMS, (1, 1, 1), pack.centres, pack.radius, pack.unit)
    cells = np.flatnonzero(mask == 0)
    rho_cell = inputs.density_noise(DIMS, seed=2)
    return L, pack, mask, cells, rho_cell


def _patch_oracle(mask, rho_cell, cell):
    n = DIMS[0]
    x, y, z = cell % n, (cell // n) % n, cell // (n * n)
    r = np.arange(-4, 5)
    zz, yy, xx = np.meshgrid((z + r) % n, (y + r) % n, (x + r) % n, indexing="ij")
    idx = (xx + n * (yy + n * zz)).reshape(-1)
    pm = mask[idx]
    f = np.stack([oracle.equilibrium(rv, (0, 0, 0)) for rv in rho_cell[idx]], 1)
    f2 = oracle.run_push((9, 9, 9), (1, 1, 1), pm, f, STEPS, 1.0, G)
    return f2[:, 364]  # the patch centre


@pytest.mark.parametrize("precision", ["f32", "f16s"])
@pytest.mark.parametrize("variant", ["aa", "et"])
def test_pack512_sampled_nodes(setup, variant, precision):
    import torch

    L, pack, mask, cells, rho_cell = setup
    lat = L.Lattice(DIMS, (1, 1, 1), variant=variant, addressing="indirect", precision=precision, omega=1.0,
                    force=G)
    lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
    n = int(lat.info.nodes)
    assert n == cells.size
    rho_dev = torch.from_numpy(rho_cell[cells]).cuda()
    lat.init(rho_dev, on_device=True)
    del rho_dev
    lat.step(STEPS)
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(n, 200, replace=False))
    out = torch.empty((19, n), dtype=torch.float64, device="cuda")
    L.lbm_get_pdfs(lat.h, n, out=out, on_device=True)
    got = out[:, torch.from_numpy(sample).cuda()].cpu().numpy()
    del out
    lat.close()
    torch.cuda.empty_cache()
    ref = np.stack([_patch_oracle(mask, rho_cell, cells[k]) for k in sample], 1)
    _, ug = oracle.macroscopics(got, G)
    _, uo = oracle.macroscopics(ref, G)
    assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= TOL_U[precision]
    rg, _ = oracle.macroscopics(got, G)
    ro, _ = oracle.macroscopics(ref, G)
    assert np.max(np.abs(rg - ro)) <= (1e-6 if precision == "f32" else 1e-4)
