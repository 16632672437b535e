"""Swap on a full grid with the tiles staged by tensor copies (TMA) against
the plain-load pass and the FP64 oracle, and the bounded wait those copies
use.  Boxes are chosen so that rows are a multiple of 16 bytes (the tensor
copies' rule) with ragged last tiles on every axis and an odd periodic tile
count (a third colour)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL_U = {"f32": 1e-5, "f16s": 2e-3}


@pytest.fixture(scope="module")
def L():
    import torch

    from paper_1111_0922_gb300 import build
    from paper_1111_0922_gb300 import lbm as lbm_mod

    assert torch.cuda.is_available()
    build.build()
    lbm_mod.load()
    return lbm_mod


def _run(L, dims, per, precision, staging, solid, f0, steps, omega, g):
    lat = L.Lattice(dims, per, variant="swap", precision=precision, omega=omega, force=g, swap_schedule=staging)
    lat.set_geometry(solid)
    lat.set_pdfs(f0)
    lat.step(steps)
    out = lat.pdfs()
    staged = lat.info.tile_staged
    lat.close()
    return out, staged


@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 1), (0, 0, 0)])
@pytest.mark.parametrize("precision,dims", [("f32", (72, 9, 5)), ("f16s", (72, 9, 5)), ("f64", (70, 9, 5)),
                                            ("f32", (8, 3, 2)), ("f64", (2, 3, 2))])
def test_staged_swap_equals_plain_and_oracle(L, precision, dims, per):
    n = int(np.prod(dims))
    rng = np.random.default_rng(sum(dims) + 7 * per[1])
    solid = (rng.random(n) < 0.1).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, 1e-5, -5e-6)
    a, sa = _run(L, dims, per, precision, 2, solid, f0, 6, 1.2, g)
    b, sb = _run(L, dims, per, precision, 1, solid, f0, 6, 1.2, g)
    assert sa == 1 and sb == 0
    assert np.array_equal(a, b)
    ref = oracle.run_push(dims, per, solid, f0, 6, 1.2, g)
    fl = solid == 0
    if precision == "f64":
        assert np.max(np.abs(a[:, fl] - ref[:, fl]) / np.abs(ref[:, fl])) <= 1e-12
    else:
        _, ug = oracle.macroscopics(a[:, fl], g)
        _, uo = oracle.macroscopics(ref[:, fl], g)
        assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= TOL_U[precision]


def test_rows_off_the_16_byte_grid_use_plain_loads(L):
    # FP32 rows of 70 cells are 280 bytes: no tensor copies
    lat = L.Lattice((70, 8, 4), (1, 1, 1), variant="swap", precision="f32", swap_schedule=2)
    lat.set_geometry(None)
    assert lat.info.tile_staged == 0
    lat.close()


def test_bounded_wait_gives_up_and_context_survives(L):
    import torch

    st = L.lbm_selftest_bounded_wait(2_000_000)
    assert st == L.LBM_ERR_TIMEOUT
    assert L.lbm_selftest_bounded_wait(10) == L.LBM_ERR_INVALID_ARG
    # the context is still usable
    lat = L.Lattice((16, 8, 4), (1, 1, 1), variant="swap", precision="f32")
    lat.set_geometry(None)
    lat.init()
    lat.step(2)
    rho, _ = lat.macroscopics()
    assert np.allclose(rho, 1.0)
    lat.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("staging", [0, 1, 2])
@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 1), (0, 0, 0), (0, 1, 1)])
@pytest.mark.parametrize("dims", [(64, 8, 6), (96, 12, 8), (72, 9, 5), (192, 4, 6), (200, 6, 6)])
def test_swap_without_solids_matches_oracle(L, dims, per, staging):
    """No solid cells: full tiles away from the walls take the warp-uniform
    path with the x faces completed afterwards; tiles on a wall or cut by the
    box take the general path.  FP64 against the oracle."""
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + staging)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (1e-5, -2e-5, 3e-6)
    ref = oracle.run_push(dims, per, None, f0, 5, 1.3, g)
    lat = L.Lattice(dims, per, variant="swap", precision="f64", omega=1.3, force=g, swap_schedule=staging)
    lat.set_geometry(None)
    lat.set_pdfs(f0)
    lat.step(5)
    out = lat.pdfs()
    lat.close()
    assert np.max(np.abs(out - ref) / np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("precision", ["f32", "f16s"])
@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 1)])
@pytest.mark.parametrize("dims", [(192, 4, 6), (200, 6, 6)])
def test_swap_full_tiles_4byte_arithmetic(L, dims, per, precision):
    """Full tiles with FP32 arithmetic (three and four tiles along x, an odd
    periodic count giving a third x colour): plain and staged passes agree
    bit for bit and match the oracle."""
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + per[1])
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, 0.0, -1e-5)
    a, _ = _run(L, dims, per, precision, 1, None, f0, 6, 1.3, g)
    b, _ = _run(L, dims, per, precision, 2, None, f0, 6, 1.3, g)
    assert np.array_equal(a, b)
    ref = oracle.run_push(dims, per, None, f0, 6, 1.3, g)
    _, ug = oracle.macroscopics(a, g)
    _, uo = oracle.macroscopics(ref, g)
    assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= TOL_U[precision]
