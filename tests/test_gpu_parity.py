"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (per precision of the stored PDFs):
  f64   max_i,x |f_gpu - f_ora| / |f_ora| <= 1e-12
  f32   max |u_gpu - u_ora| / max |u_ora| <= 1e-5  (velocity, u incl. g/2)
  f16s  max |u_gpu - u_ora| / max |u_ora| <= 2e-3  over a few steps: FP16
        keeps 11 significant bits of (f - w) * S, a relative rounding of
        2^-11 = 4.9e-4 per store, and a velocity sums 10 such values
Streaming and index work are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1111_0922_gb300 import inputs

pytestmark = pytest.mark.gpu

VARIANTS = ["ts", "os_push", "os_pull", "cg", "swap", "aa", "et"]
DIRECT_ONLY = set()
TOL_U = {"f32": 1e-5, "f16s": 2e-3}


@pytest.fixture(scope="module")
def lbm():
    import torch

    from paper_1111_0922_gb300 import build
    from paper_1111_0922_gb300 import lbm as L

    assert torch.cuda.is_available()
    build.build()
    L.load()
    return L


def _lattice(L, dims, per, variant, addressing="direct", layout="soa", precision="f64", omega=1.0,
             force=(0.0, 0.0, 0.0), **kw):
    return L.Lattice(dims, per, variant=variant, addressing=addressing, layout=layout,
                     precision=precision, omega=omega, force=force, **kw)


def _case(dims, frac, seed, amp=0.02):
    n = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    solid = (rng.random(n) < frac).astype(np.uint8) if frac > 0 else None
    f = oracle.rest_state(n) * (1 + amp * (rng.random((19, n)) - 0.5))
    return solid, f


def _compare(prec, f_gpu, f_ora, g, sel):
    if prec == "f64":
        rel = np.max(np.abs(f_gpu[:, sel] - f_ora[:, sel]) / np.abs(f_ora[:, sel]))
        assert rel <= 1e-12, rel
    else:
        _, ug = oracle.macroscopics(f_gpu[:, sel], g)
        _, uo = oracle.macroscopics(f_ora[:, sel], g)
        rel = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
        assert rel <= TOL_U[prec], rel


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("layout", ["soa", "aos"])
@pytest.mark.parametrize("addressing", ["direct", "indirect"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_matches_oracle(lbm, variant, addressing, layout, precision):
    """19x13x11 box (2717 cells: several blocks and a ragged last block),
    periodic x and z, walls on y, 12 % solid cells, a body force, 6 steps."""
    if addressing == "indirect" and variant in DIRECT_ONLY:
        pytest.skip("direct addressing only")
    dims, per = (19, 13, 11), (1, 0, 1)
    solid, f0 = _case(dims, 0.12, seed=31)
    g = (2e-5, -1e-5, 5e-6)
    omega = 1.25
    ref = oracle.run_push(dims, per, solid, f0, 6, omega, g)
    lat = _lattice(lbm, dims, per, variant, addressing, layout, precision, omega, g)
    lat.set_geometry(solid)
    fl = np.ones(f0.shape[1], bool) if solid is None else solid == 0
    if addressing == "direct":
        lat.set_pdfs(f0)
        lat.step(6)
        out = lat.pdfs()
        _compare(precision, out, ref, g, fl)
    else:
        cells = lat.nodes()
        assert np.array_equal(cells, np.flatnonzero(fl))
        lat.set_pdfs(f0[:, cells])
        lat.step(6)
        out = lat.pdfs()
        _compare(precision, out, ref[:, cells], g, slice(None))
    lat.close()


@pytest.mark.parametrize("variant", ["ts", "os_pull"])
def test_duct_32_two_step_and_pull_fp64(lbm, variant):
    """32^3 duct, periodic in x, bounce-back walls in y and z, omega 1,
    g = 1e-6 along x, 100 steps from rest, FP64 SoA direct."""
    dims, per = inputs.duct(32)
    g = (1e-6, 0.0, 0.0)
    f0 = oracle.rest_state(32 ** 3)
    ref = oracle.run_push(dims, per, None, f0, 100, 1.0, g)
    lat = _lattice(lbm, dims, per, variant, omega=1.0, force=g)
    lat.set_geometry(None)
    lat.init()
    lat.step(100)
    out = lat.pdfs()
    rel = np.max(np.abs(out - ref) / np.abs(ref))
    assert rel <= 1e-12, rel
    _, u = lat.macroscopics()
    _, uo = oracle.macroscopics(ref, g)
    # u sums 19 PDFs of size <= 1/3: round-off of a few 1e-17 on each
    assert np.max(np.abs(u - uo)) <= 1e-15
    lat.close()


def _dyadic_state(n, scale, seed):
    """f = w + k / scale with integer k: exactly representable deviations in
    every storage precision (FP16 with this scale, FP32, FP64)."""
    rng = np.random.default_rng(seed)
    _, w = oracle.lattice()
    k = rng.integers(-1500, 1500, size=(19, n))
    return w[:, None] + k / scale


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("addressing", ["direct", "indirect"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_streaming_is_exact_permutation(lbm, variant, addressing, precision):
    """Identity collision (omega 0, no force): every scheme moves the PDFs
    exactly as the oracle's streaming does, bit for bit."""
    if addressing == "indirect" and variant in DIRECT_ONLY:
        pytest.skip("direct addressing only")
    dims, per = (8, 6, 5), (1, 0, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(7)
    solid = (rng.random(n) < 0.15).astype(np.uint8)
    scale = 2.0 ** 20
    f0 = _dyadic_state(n, scale, 8)
    ref = oracle.run_push(dims, per, solid, f0, 4, 0.0)
    lat = _lattice(lbm, dims, per, variant, addressing, "soa", precision, omega=0.0,
                   f16_scale=scale)
    lat.set_geometry(solid)
    fl = solid == 0
    if addressing == "direct":
        lat.set_pdfs(np.where(fl[None, :], f0, oracle.rest_state(n)))
        lat.step(4)
        out = lat.pdfs()
        assert np.array_equal(out[:, fl], ref[:, fl])
    else:
        cells = lat.nodes()
        lat.set_pdfs(f0[:, cells])
        lat.step(4)
        assert np.array_equal(lat.pdfs(), ref[:, cells])
    lat.close()


@pytest.mark.parametrize("per", [(1, 1, 1), (1, 0, 0), (0, 0, 0)])
def test_sphere_geometry_node_list_and_idx_bit_exact(lbm, per):
    dims = (37, 29, 23)
    pack = inputs.sphere_pack(dims, 0.6, radius=4.0, seed=5, periodic=per)
    mask_ora = oracle.sphere_mask(dims, per, pack.centres, pack.radius, pack.unit)
    cells_ora, node_of = oracle.build_nodes(dims, per, mask_ora)
    idx_ora = oracle.build_idx(dims, per, mask_ora, cells_ora, node_of)
    for variant in ("aa", "et"):
        lat = _lattice(lbm, dims, per, variant, "indirect", precision="f32")
        lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
        assert np.array_equal(lat.mask(), mask_ora)
        assert lat.info.nodes == cells_ora.size
        assert np.array_equal(lat.nodes(), cells_ora)
        assert np.array_equal(lat.idx(), idx_ora)
        lat.close()


def test_host_mask_geometry_matches(lbm):
    dims, per = (20, 17, 9), (1, 1, 0)
    rng = np.random.default_rng(3)
    mask = (rng.random(int(np.prod(dims))) < 0.35).astype(np.uint8)
    cells_ora, node_of = oracle.build_nodes(dims, per, mask)
    idx_ora = oracle.build_idx(dims, per, mask, cells_ora, node_of)
    lat = _lattice(lbm, dims, per, "os_pull", "indirect")
    lat.set_geometry(mask * 7)  # any nonzero byte is solid
    assert np.array_equal(lat.mask(), mask)
    assert np.array_equal(lat.nodes(), cells_ora)
    assert np.array_equal(lat.idx(), idx_ora)
    lat.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("addressing", ["direct", "indirect"])
def test_flux_reductions(lbm, variant, addressing):
    """lbm_flux and the reduction fused into lbm_step_flux give the mass and
    flux of the state the call starts from (FP64 state: 1e-12 relative)."""
    if addressing == "indirect" and variant in DIRECT_ONLY:
        pytest.skip("direct addressing only")
    dims, per = (24, 10, 12), (1, 0, 1)
    solid, f0 = _case(dims, 0.1, seed=4)
    g = (1e-5, 0.0, 0.0)
    fl = solid == 0
    lat = _lattice(lbm, dims, per, variant, addressing, precision="f64", omega=1.1, force=g)
    lat.set_geometry(solid)
    lat.set_pdfs(f0 if addressing == "direct" else f0[:, fl])
    f2 = oracle.run_push(dims, per, solid, f0, 2, 1.1, g)
    m0, j0 = oracle.flux(f0[:, fl], g)
    m2, j2 = oracle.flux(f2[:, fl], g)
    m, j = lat.flux()
    assert abs(m - m0) <= 1e-12 * m0 and abs(j - j0) <= 1e-12 * abs(j0)
    m, j = lat.step_flux(2)
    assert abs(m - m0) <= 1e-12 * m0 and abs(j - j0) <= 1e-12 * abs(j0)
    m, j = lat.flux()
    assert abs(m - m2) <= 1e-12 * m2 and abs(j - j2) <= 1e-12 * abs(j2)
    lat.close()


@pytest.mark.parametrize("variant", ["aa", "et"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_init_density_noise_256_sampled(lbm, variant, precision):
    """Full-size 256^3 periodic box from rho = 1 + 1e-3 U[-1,1) (seed 2),
    omega 1.7, in the bench's launch shape: after 2 steps, sampled nodes
    against the oracle computed node by node from the initial state."""
    dims, per = (256, 256, 256), (1, 1, 1)
    n = 256 ** 3
    rho = inputs.density_noise(dims, seed=2)
    lat = _lattice(lbm, dims, per, variant, precision=precision, omega=1.7)
    lat.set_geometry(None)
    lat.init(rho)
    lat.step(2)
    out = lat.pdfs()
    rng = np.random.default_rng(0)
    sample = rng.choice(n, 400, replace=False)
    # oracle: the 5^3 neighbourhood of each sampled cell, two steps
    ref = np.empty((19, sample.size))
    for s_i, c in enumerate(sample):
        x, y, z = c % 256, (c // 256) % 256, c // 65536
        sub = [(x + dx) % 256 + 256 * (((y + dy) % 256) + 256 * ((z + dz) % 256))
               for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)]
        r = rho[sub]
        f = np.stack([oracle.equilibrium(rv, (0, 0, 0)) for rv in r], 1)
        f2 = oracle.run_push((5, 5, 5), (1, 1, 1), None, f, 2, 1.7)
        ref[:, s_i] = f2[:, 62]  # centre of the 5^3 patch; its wrap never reaches it in 2 steps
    got = out[:, sample]
    if precision == "f64":
        assert np.max(np.abs(got - ref) / ref) <= 1e-12
    else:
        _, ug = oracle.macroscopics(got)
        _, uo = oracle.macroscopics(ref)
        assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= 1e-5
    lat.close()


@pytest.mark.parametrize("per", [(1, 1, 1), (0, 0, 0), (1, 0, 1), (0, 1, 0)])
@pytest.mark.parametrize("dims", [(70, 9, 13), (33, 5, 7), (64, 8, 8), (2, 3, 2), (150, 4, 3)])
def test_swap_tiling_and_colouring(lbm, dims, per):
    """Blocked swap over tile counts that are odd, even, one per axis, with
    periodic wrap between tiles and inside a single tile."""
    if any(p and d < 2 for p, d in zip(per, dims)):
        pytest.skip("periodic extent < 2")
    n = int(np.prod(dims))
    rng = np.random.default_rng(sum(dims))
    solid = (rng.random(n) < 0.1).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    ref = oracle.run_push(dims, per, solid, f0, 3, 1.2, (1e-5, 0, 0))
    lat = _lattice(lbm, dims, per, "swap", omega=1.2, force=(1e-5, 0, 0))
    lat.set_geometry(solid)
    lat.set_pdfs(f0)
    lat.step(3)
    fl = solid == 0
    out = lat.pdfs()
    assert np.max(np.abs(out[:, fl] - ref[:, fl]) / ref[:, fl]) <= 1e-12
    lat.close()


@pytest.mark.parametrize("shift", [2, 3, 5, 0])
@pytest.mark.parametrize("per", [(1, 1, 1), (1, 1, 0)])
def test_compressed_grid_shifts(lbm, shift, per):
    """Compressed grid with shifts of 2 planes (slabs of one plane) up to the
    default, periodic and walled z."""
    dims = (11, 7, 13)
    n = int(np.prod(dims))
    rng = np.random.default_rng(shift + 3)
    solid = (rng.random(n) < 0.1).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    ref = oracle.run_push(dims, per, solid, f0, 5, 0.9, (0, 0, 2e-5))
    lat = _lattice(lbm, dims, per, "cg", omega=0.9, force=(0, 0, 2e-5), cg_shift=shift)
    lat.set_geometry(solid)
    lat.set_pdfs(f0)
    lat.step(5)
    fl = solid == 0
    out = lat.pdfs()
    assert np.max(np.abs(out[:, fl] - ref[:, fl]) / ref[:, fl]) <= 1e-12
    lat.close()


@pytest.mark.parametrize("slab", [1, 7, 100, 0])
@pytest.mark.parametrize("per", [(1, 1, 1), (1, 1, 0), (0, 1, 1)])
def test_compressed_grid_node_list_slabs(lbm, slab, per):
    """Compressed grid on a node list: slabs of 1 node up to the default,
    z-wrapped links through the ghost copies, walls on z or x."""
    dims = (9, 7, 8)
    n = int(np.prod(dims))
    rng = np.random.default_rng(slab + 11)
    solid = (rng.random(n) < 0.2).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (1e-5, 0, -2e-5)
    ref = oracle.run_push(dims, per, solid, f0, 5, 1.1, g)
    lat = _lattice(lbm, dims, per, "cg", "indirect", omega=1.1, force=g, cg_shift=slab)
    lat.set_geometry(solid)
    cells = lat.nodes()
    lat.set_pdfs(f0[:, cells])
    lat.step(5)
    out = lat.pdfs()
    assert np.max(np.abs(out - ref[:, cells]) / ref[:, cells]) <= 1e-12
    lat.close()


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("addressing", ["direct", "indirect"])
@pytest.mark.parametrize("variant", ["os_push", "os_pull"])
def test_streaming_stores_match(lbm, variant, addressing, precision):
    """OS push/pull with cache-streaming stores of the second lattice (the
    OS-NT analogue): the same arithmetic as ordinary stores, so the PDFs agree
    bit for bit, and with the oracle within the precision's tolerance."""
    dims, per = (19, 13, 11), (1, 0, 1)
    solid, f0 = _case(dims, 0.12, seed=37)
    g = (2e-5, -1e-5, 5e-6)
    ref = oracle.run_push(dims, per, solid, f0, 5, 1.3, g)
    fl = solid == 0
    outs = []
    for hint in (0, 1):
        lat = _lattice(lbm, dims, per, variant, addressing, "soa", precision, 1.3, g, store_hint=hint)
        lat.set_geometry(solid)
        cells = lat.nodes() if addressing == "indirect" else None
        lat.set_pdfs(f0 if cells is None else f0[:, cells])
        lat.step(5)
        outs.append(lat.pdfs())
        lat.close()
    assert np.array_equal(outs[0], outs[1])
    if addressing == "direct":
        _compare(precision, outs[1], ref, g, fl)
    else:
        _compare(precision, outs[1], ref[:, np.flatnonzero(fl)], g, slice(None))
