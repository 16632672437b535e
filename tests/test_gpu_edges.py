"""Degenerate geometries through every scheme: no fluid node at all, a single
node whose every link bounces back, one plane, a channel one cell wide."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

VARIANTS = ["ts", "os_push", "os_pull", "cg", "swap", "aa", "et"]


@pytest.fixture(scope="module")
def L():
    from paper_1111_0922_gb300 import build, lbm

    build.build()
    lbm.load()
    return lbm


@pytest.mark.parametrize("variant", VARIANTS)
def test_no_fluid_node(L, variant):
    dims = (4, 3, 2)
    lat = L.Lattice(dims, (1, 1, 1), variant=variant, addressing="indirect", precision="f64", omega=1.0)
    lat.set_geometry(np.ones(24, np.uint8))
    assert lat.info.nodes == 0
    lat.step(4)
    assert lat.flux() == (0.0, 0.0)
    assert lat.pdfs().shape == (19, 0)
    lat.close()


@pytest.mark.parametrize("addressing", ["direct", "indirect"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_single_node_closed_box(L, variant, addressing):
    """One cell with walls on every face: pure bounce-back; mass and the
    force-free rest state are kept exactly, a body force makes the node's
    momentum oscillate but never drift (all links reflect)."""
    dims, per = (1, 1, 1), (0, 0, 0)
    f0 = oracle.rest_state(1) * (1 + 0.01 * np.linspace(-1, 1, 19)[:, None])
    g = (1e-4, 0, 0)
    ref = oracle.run_push(dims, per, None, f0, 6, 1.2, g)
    lat = L.Lattice(dims, per, variant=variant, addressing=addressing, precision="f64", omega=1.2, force=g)
    lat.set_geometry(None)
    lat.set_pdfs(f0)
    lat.step(6)
    out = lat.pdfs()
    assert np.max(np.abs(out - ref) / ref) <= 1e-12
    lat.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dims,per", [((7, 5, 1), (1, 1, 0)), ((1, 6, 5), (0, 1, 1)), ((9, 1, 1), (1, 0, 0))])
def test_thin_boxes(L, variant, dims, per):
    n = int(np.prod(dims))
    rng = np.random.default_rng(n)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (1e-5, 2e-5, 0)
    ref = oracle.run_push(dims, per, None, f0, 4, 0.9, g)
    for addressing in ("direct", "indirect"):
        lat = L.Lattice(dims, per, variant=variant, addressing=addressing, precision="f64", omega=0.9, force=g)
        lat.set_geometry(None)
        lat.set_pdfs(f0)
        lat.step(4)
        assert np.max(np.abs(lat.pdfs() - ref) / ref) <= 1e-12
        lat.close()


def test_rejects_bad_requests(L):
    with pytest.raises(L.LBMError) as e:
        L.Lattice((4, 4, 4), (1, 1, 1), variant="aa", block_size=100)
    assert e.value.status == L.LBM_ERR_INVALID_ARG
    lat = L.Lattice((4, 4, 4), (1, 1, 1), variant="aa", precision="f32")
    with pytest.raises(L.LBMError) as e:
        lat.step(1)  # no geometry yet
    assert e.value.status == L.LBM_ERR_STATE
    lat.set_geometry(None)
    lat.step(1)
    with pytest.raises(L.LBMError) as e:
        lat.pdfs()  # AA pattern after an odd step count
    assert e.value.status == L.LBM_ERR_STATE
    lat.close()
