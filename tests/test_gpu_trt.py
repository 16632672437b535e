"""Two-relaxation-time collision on the GPU against the oracle's TRT, and
the Poiseuille profile with Lam = 3/16 (walls exactly half-way)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

MAGIC = 3.0 / 16.0


@pytest.fixture(scope="module")
def L():
    from paper_1111_0922_gb300 import build, lbm

    build.build()
    lbm.load()
    return lbm


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("addressing", ["direct", "indirect"])
@pytest.mark.parametrize("variant", ["ts", "os_push", "os_pull", "cg", "swap", "aa", "et"])
def test_trt_matches_oracle(L, variant, addressing, precision):
    dims, per = (12, 9, 10), (1, 0, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(5)
    solid = (rng.random(n) < 0.1).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    omega, g = 1.4, (2e-5, 0.0, -1e-5)
    lm = oracle.trt_lambda_minus(omega, MAGIC)
    ref = oracle.run_push_trt(dims, per, solid, f0, 4, omega, lm, g)
    lat = L.Lattice(dims, per, variant=variant, addressing=addressing, precision=precision, omega=omega,
                    force=g, trt_magic=MAGIC)
    lat.set_geometry(solid)
    fl = solid == 0
    if addressing == "direct":
        lat.set_pdfs(f0)
        lat.step(4)
        out = lat.pdfs()[:, fl]
    else:
        cells = lat.nodes()
        lat.set_pdfs(f0[:, cells])
        lat.step(4)
        out = lat.pdfs()
    want = ref[:, fl]
    if precision == "f64":
        assert np.max(np.abs(out - want) / want) <= 1e-12
    else:
        _, ug = oracle.macroscopics(out, g)
        _, uo = oracle.macroscopics(want, g)
        assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= 1e-5
    lat.close()


@pytest.mark.parametrize("omega", [0.8, 1.6])
def test_trt_poiseuille_exact_walls_gpu(L, omega):
    H = 12
    dims, per = (2, H, 2), (1, 0, 1)
    gx = 1e-6
    nu = (1.0 / omega - 0.5) / 3.0
    steps = int(40 * H * H / nu / np.pi ** 2) + 2000
    steps += steps % 2
    lat = L.Lattice(dims, per, variant="aa", precision="f64", omega=omega, force=(gx, 0, 0), trt_magic=MAGIC)
    lat.set_geometry(None)
    lat.init()
    lat.step(steps)
    _, u = lat.macroscopics()
    prof = u[:, 0].reshape(2, H, 2, order="F")[0, :, 0]
    y = np.arange(H) - (H - 1) / 2.0
    exact = gx / (2 * nu) * ((H / 2.0) ** 2 - y ** 2)
    assert np.max(np.abs(prof - exact)) / np.max(exact) < 1e-9
    lat.close()
