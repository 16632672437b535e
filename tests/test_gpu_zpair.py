"""FP16 and FP32 storage in z pairs (cells z and z + nz/2 in one 4- or 8-byte
word, one thread per pair) for the AA pattern (Sec. 6, Fig. 5), the two-step (Sec. 2),
the one-step push and pull (Sec. 3) schemes and, on periodic boxes, the
esoteric twist (Sec. 7) and the coloured swap (Sec. 5); the compressed
grid (Sec. 4) pairs cells y and y + ny/2 instead.

The per-node arithmetic is that of the one-node-per-thread kernels, so the
two layouts give the same PDFs bit for bit; the oracle comparison uses the
FP16 velocity tolerance of test_gpu_parity (2e-3 relative).
"""
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


VARIANTS = ["aa", "ts", "os_push", "os_pull"]


def _run(L, dims, per, f0, steps, pair_z, g=(0.0, 0.0, 0.0), omega=1.3, solid=None, variant="aa", precision="f16s"):
    lat = L.Lattice(dims, per, variant=variant, precision=precision, omega=omega, force=g, pair_z=pair_z)
    lat.set_geometry(solid)
    lat.set_pdfs(f0)
    lat.step(steps)
    out = lat.pdfs()
    paired = lat.info.pair_z
    lat.close()
    return out, paired


CASES = [
    ((24, 10, 12), (1, 1, 1)),
    ((24, 10, 12), (1, 0, 1)),
    ((24, 10, 12), (0, 1, 0)),
    ((20, 6, 8), (0, 0, 0)),
    ((33, 7, 10), (1, 1, 0)),
    ((16, 8, 2), (1, 1, 1)),
    ((16, 8, 4), (1, 1, 0)),
    ((130, 3, 6), (1, 1, 1)),
]


@pytest.mark.parametrize("precision", ["f16s", "f32"])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("dims,per", CASES)
def test_pairs_equal_single_nodes_bitwise(L, dims, per, force, variant, precision):
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + 3 * per[2] + force)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, -1e-5, 5e-6) if force else (0.0, 0.0, 0.0)
    for steps in (2, 6):
        a, pa = _run(L, dims, per, f0, steps, 0, g, variant=variant, precision=precision)
        b, pb = _run(L, dims, per, f0, steps, 2, g, variant=variant, precision=precision)
        assert pa == 1 and pb == 0
        assert np.array_equal(a, b), (dims, per, steps)


@pytest.mark.parametrize("precision", ["f16s", "f32"])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("dims", [(24, 10, 12), (16, 8, 2), (130, 3, 6), (8, 4, 6)])
def test_et_pairs_equal_single_nodes_bitwise(L, dims, force, precision):
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + force)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, -1e-5, 5e-6) if force else (0.0, 0.0, 0.0)
    for steps in (1, 2, 5):
        a, pa = _run(L, dims, (1, 1, 1), f0, steps, 0, g, variant="et", precision=precision)
        b, pb = _run(L, dims, (1, 1, 1), f0, steps, 2, g, variant="et", precision=precision)
        assert pa == 1 and pb == 0
        assert np.array_equal(a, b), (dims, steps)
    _, pw = _run(L, dims, (1, 0, 1), f0, 1, 0, g, variant="et", precision=precision)
    assert pw == 0  # walls: halo slots, one node per thread


CG_CASES = [
    ((24, 10, 12), (1, 1, 1)),
    ((24, 10, 12), (1, 0, 1)),
    ((20, 6, 9), (0, 0, 0)),
    ((33, 8, 7), (1, 1, 0)),
    ((16, 2, 6), (1, 1, 1)),
    ((130, 4, 5), (0, 1, 1)),
]


@pytest.mark.parametrize("precision", ["f16s", "f32"])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("dims,per", CG_CASES)
def test_cg_y_pairs_equal_single_nodes_bitwise(L, dims, per, force, precision):
    """Compressed grid: cells y and y + ny/2 paired (z pairs would not survive
    the plane shifts); several shifts per run and both sweep directions."""
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + force)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, -1e-5, 5e-6) if force else (0.0, 0.0, 0.0)
    for steps in (1, 2, 5):
        a, pa = _run(L, dims, per, f0, steps, 0, g, variant="cg", precision=precision)
        b, pb = _run(L, dims, per, f0, steps, 2, g, variant="cg", precision=precision)
        assert pa == 1 and pb == 0
        assert np.array_equal(a, b), (dims, per, steps)


SWAP_CASES = [
    ((130, 6, 8), (1, 1, 1)),
    ((64, 4, 12), (1, 0, 1)),
    ((70, 8, 16), (0, 1, 1)),
    ((128, 2, 8), (1, 1, 1)),
    ((64, 6, 8), (1, 1, 1)),
    ((40, 5, 8), (0, 0, 1)),
]


@pytest.mark.parametrize("precision", ["f16s", "f32"])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("dims,per", SWAP_CASES)
def test_swap_pairs_equal_single_nodes_bitwise(L, dims, per, force, precision):
    """Coloured swap on the grid of pair words (periodic z, nz a multiple of
    4): tile counts odd and even, one tile along x or y, walls along x or y,
    cut tiles; links across the seam exchange the halves."""
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + force)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, -1e-5, 5e-6) if force else (0.0, 0.0, 0.0)
    for steps in (1, 2, 5):
        a, pa = _run(L, dims, per, f0, steps, 0, g, variant="swap", precision=precision)
        b, pb = _run(L, dims, per, f0, steps, 2, g, variant="swap", precision=precision)
        assert pa == 1 and pb == 0
        assert np.array_equal(a, b), (dims, per, steps)


def test_swap_pairs_only_where_allowed(L):
    for dims, per, kw in (((64, 4, 6), (1, 1, 1), {}), ((64, 4, 8), (1, 1, 0), {}), ((64, 4, 4), (1, 1, 1), {}),
                          ((64, 4, 8), (1, 1, 1), {"swap_schedule": 2})):
        lat = L.Lattice(dims, per, variant="swap", precision="f32", **kw)
        lat.set_geometry(None)
        assert lat.info.pair_z == 0, (dims, per, kw)
        lat.close()


@pytest.mark.parametrize("precision", ["f16s", "f32"])
@pytest.mark.parametrize("variant", VARIANTS + ["cg"])
@pytest.mark.parametrize("dims,per", [((24, 10, 12), (1, 1, 1)), ((20, 6, 8), (0, 0, 0)), ((16, 8, 4), (1, 0, 0))])
def test_pairs_match_oracle(L, dims, per, variant, precision):
    n = int(np.prod(dims))
    rng = np.random.default_rng(n)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (1e-5, 0.0, -2e-5)
    out, paired = _run(L, dims, per, f0, 8, 0, g, variant=variant, precision=precision)
    assert paired == 1
    ref = oracle.run_push(dims, per, None, f0, 8, 1.3, g)
    _, ug = oracle.macroscopics(out, g)
    _, uo = oracle.macroscopics(ref, g)
    assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= TOL_U[precision]


@pytest.mark.parametrize("precision", ["f16s", "f32"])
@pytest.mark.parametrize("variant", VARIANTS + ["cg", "swap"])
def test_pairs_fused_reduction_and_readout(L, variant, precision):
    """Mass and flux from the fused reduction and the read-out kernel agree
    with the one-node-per-thread layout (FP64 sums, 1e-12 relative), and a
    state written and read back is unchanged."""
    dims, per = (32, 12, 16), (1, 0, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(7)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    res = []
    for pz in (0, 2):
        lat = L.Lattice(dims, per, variant=variant, precision=precision, omega=1.2, force=(1e-5, 0, 0), pair_z=pz)
        lat.set_geometry(None)
        lat.set_pdfs(f0)
        back = lat.pdfs()
        m0, j0 = lat.step_flux(4)
        m1, j1 = lat.flux()
        res.append((back, m0, j0, m1, j1))
        lat.close()
    (ba, *ra), (bb, *rb) = res
    assert np.array_equal(ba, bb)
    for x, y in zip(ra, rb):
        assert abs(x - y) <= 1e-12 * max(abs(x), abs(y), 1e-30)


def test_pairs_off_with_solids_or_odd_nz(L):
    n = 16 * 8 * 6
    solid = np.zeros(n, np.uint8)
    solid[5] = 1
    lat = L.Lattice((16, 8, 6), (1, 1, 1), variant="aa", precision="f16s")
    lat.set_geometry(solid)
    assert lat.info.pair_z == 0
    lat.close()
    lat = L.Lattice((16, 8, 5), (1, 1, 1), variant="aa", precision="f16s")
    lat.set_geometry(None)
    assert lat.info.pair_z == 0
    lat.close()
    lat = L.Lattice((16, 7, 6), (1, 1, 1), variant="cg", precision="f16s")  # odd ny
    lat.set_geometry(None)
    assert lat.info.pair_z == 0
    lat.close()
    for variant, kw in (("aa", {"precision": "f64"}), ("os_push", {"store_hint": 1}),
                        ("aa", {"layout": "aos"}), ("os_pull", {"addressing": "indirect"}), ("aa", {"pair_z": 2}),
                        ("aa", {"addressing": "indirect", "pair_z": 2}), ("et", {"addressing": "indirect", "pair_z": 2}),
                        ("et", {"addressing": "indirect", "precision": "f32"}),
                        ("aa", {"addressing": "indirect", "precision": "f32"}),
                        ("aa", {"addressing": "indirect", "precision": "f64"})):
        kw.setdefault("precision", "f16s")
        lat = L.Lattice((16, 8, 6), (1, 1, 1), variant=variant, **kw)
        lat.set_geometry(None)
        assert lat.info.pair_z == 0, variant
        lat.close()


NODE_CASES = [
    ((16, 8, 6), (1, 1, 1), 0.15),
    ((17, 9, 7), (1, 0, 1), 0.2),
    ((24, 10, 12), (0, 0, 0), 0.1),
    ((33, 7, 10), (1, 1, 0), 0.3),
    ((5, 3, 3), (1, 1, 1), 0.0),
]


@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("dims,per,solid_frac", NODE_CASES)
@pytest.mark.parametrize("variant", ["aa", "et"])
def test_node_pairs_equal_single_nodes_bitwise(L, variant, dims, per, solid_frac, force):
    """AA pattern and esoteric twist on a node list with FP16 storage:
    consecutive nodes 2t and 2t + 1 in one thread (one word per array for
    the own-slot loads and stores, one 8-byte index word and two gathers per
    direction for the neighbour slots) against one node per thread, with odd
    and even node counts (the last node of an odd count alone), solid links
    (folded into the AA pattern's IDX; ghost slots and split stores in the
    esoteric twist), walls and periodic axes, several pairs per thread."""
    precision = "f16s"
    n = int(np.prod(dims))
    rng = np.random.default_rng(n + 7 * force)
    solid = (rng.random(n) < solid_frac).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, -1e-5, 5e-6) if force else (0.0, 0.0, 0.0)
    fl = solid == 0
    for steps in (2, 4, 6):
        out = []
        for pz in (0, 2):
            lat = L.Lattice(dims, per, variant=variant, addressing="indirect", precision=precision, omega=1.3,
                            force=g, pair_z=pz)
            lat.set_geometry(solid)
            cells = lat.nodes()
            assert np.array_equal(cells, np.flatnonzero(fl))
            lat.set_pdfs(f0[:, cells])  # node order
            lat.step(steps)
            m, j = lat.step_flux(2)  # sums of the state after `steps`, fused into the next step
            out.append((lat.pdfs(), lat.info.pair_z, int(lat.info.nodes), m, j))
            lat.close()
        (a, pa, na, ma, ja), (b, pb, nb, mb, jb) = out
        assert pa == 1 and pb == 0 and na == nb == int(fl.sum())
        assert np.array_equal(a, b), (dims, per, steps)
        assert abs(ma - mb) <= 1e-12 * abs(mb) and abs(ja - jb) <= 1e-12 * max(abs(jb), 1e-30)


@pytest.mark.parametrize("variant", ["aa", "et"])
def test_node_pairs_match_oracle(L, variant):
    precision = "f16s"
    dims, per = (24, 10, 12), (1, 1, 0)
    n = int(np.prod(dims))
    rng = np.random.default_rng(11)
    solid = (rng.random(n) < 0.2).astype(np.uint8)
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (1e-5, 0.0, -2e-5)
    lat = L.Lattice(dims, per, variant=variant, addressing="indirect", precision=precision, omega=1.3, force=g)
    lat.set_geometry(solid)
    cells = lat.nodes()
    lat.set_pdfs(f0[:, cells])
    lat.step(8)
    out = lat.pdfs()
    assert lat.info.pair_z == 1
    lat.close()
    ref = oracle.run_push(dims, per, solid, f0, 8, 1.3, g)
    _, ug = oracle.macroscopics(out, g)
    _, uo = oracle.macroscopics(ref[:, cells], g)
    assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= TOL_U[precision]


@pytest.mark.parametrize("variant", ["aa", "et"])
@pytest.mark.parametrize("nfluid", [1, 2, 3, 64, 65])
def test_node_pairs_tiny_lists(L, variant, nfluid):
    """Node lists of one, two and three nodes (a lone last node, one pair, a
    pair and a lone node) and of 64 / 65 nodes, with FP16 node pairs against
    one node per thread; every other cell solid."""
    dims, per = (5, 4, 4), (1, 1, 1)
    n = int(np.prod(dims))
    rng = np.random.default_rng(nfluid)
    solid = np.ones(n, np.uint8)
    solid[np.sort(rng.choice(n, nfluid, replace=False))] = 0
    f0 = oracle.rest_state(n) * (1 + 0.02 * (rng.random((19, n)) - 0.5))
    g = (2e-5, 0.0, 1e-5)
    out = []
    for pz in (0, 2):
        lat = L.Lattice(dims, per, variant=variant, addressing="indirect", precision="f16s", omega=1.2, force=g,
                        pair_z=pz)
        lat.set_geometry(solid)
        cells = lat.nodes()
        assert cells.size == nfluid
        lat.set_pdfs(f0[:, cells])
        lat.step(4)
        out.append((lat.pdfs(), lat.info.pair_z))
        lat.close()
    (a, pa), (b, pb) = out
    assert pa == 1 and pb == 0
    assert np.array_equal(a, b)
    ref = oracle.run_push(dims, per, solid, f0, 4, 1.2, g)
    _, ug = oracle.macroscopics(a, g)
    _, uo = oracle.macroscopics(ref[:, cells], g)
    assert np.max(np.abs(ug - uo)) <= 2e-3 * max(np.max(np.abs(uo)), 1e-12) + 1e-9
