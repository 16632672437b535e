"""Batched geometries (continuous batching) against the oracle, and the
same geometry alone and in a mix: bit-identical states and fluxes."""
import numpy as np
import pytest

import oracle
from paper_1111_0922_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1111_0922_gb300 import build, lbm

    build.build()
    lbm.load()
    return lbm


def _packs():
    return [
        (inputs.sphere_pack((20, 20, 20), 0.6, radius=3.0, seed=21), 1.0, (1e-5, 0, 0)),
        (inputs.sphere_pack((24, 18, 16), 0.5, radius=4.0, seed=22, periodic=(1, 0, 1)), 1.3, (0, 2e-5, 0)),
        (inputs.sphere_pack((16, 16, 16), 0.7, radius=2.5, seed=23, periodic=(0, 1, 1)), 0.8, (3e-6, 0, 1e-5)),
    ]


def _oracle_steps(pack, omega, force, nsteps, f0=None):
    mask = oracle.sphere_mask(pack.dims, pack.periodic, pack.centres, pack.radius, pack.unit)
    cells, node_of = oracle.build_nodes(pack.dims, pack.periodic, mask)
    idx = oracle.build_idx(pack.dims, pack.periodic, mask, cells, node_of)
    f = oracle.rest_state(cells.size) if f0 is None else f0
    return oracle.run_sparse(idx, f, nsteps, omega, force), f


@pytest.mark.parametrize("variant", ["aa", "et"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_matches_oracle(L, variant, precision):
    b = L.Batch(3 * 16384, variant=variant, precision=precision, max_geometries=8)
    slots = [b.admit(p, om, g) for p, om, g in _packs()]
    b.round(6)
    for s, (p, om, g) in zip(slots, _packs()):
        got = b.pdfs(s)
        ref, f0 = _oracle_steps(p, om, g, 6)
        m0, j0 = oracle.flux(f0, g)
        m, j, steps = b.poll(s)
        assert steps == 6
        # the fused sums add per-node moments from the collision, computed in
        # the storage's arithmetic (FP32: ~6e-8 relative each), in FP64
        tol = 1e-12 if precision == "f64" else 1e-6
        assert abs(m - m0) <= tol * m0 and abs(j - j0) <= tol * abs(j0)
        if precision == "f64":
            assert np.max(np.abs(got - ref) / ref) <= 1e-12
        else:
            _, ug = oracle.macroscopics(got, g)
            _, uo = oracle.macroscopics(ref, g)
            assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= 1e-5
    b.close()


@pytest.mark.parametrize("variant", ["aa", "et"])
def test_alone_equals_mix_bitwise(L, variant):
    packs = _packs()
    target = packs[0]
    alone = L.Batch(16384, variant=variant, precision="f32", max_geometries=4)
    s_alone = alone.admit(*target)
    fl_alone = []
    for _ in range(3):
        alone.round(4)
        fl_alone.append(alone.poll(s_alone))
    mix = L.Batch(4 * 16384, variant=variant, precision="f32", max_geometries=8, block_size=128,
                  nodes_per_thread=2)
    other = mix.admit(*packs[1])
    mix.round(3)  # the other geometry is at an odd step count when the target arrives
    s_mix = mix.admit(*target)
    mix.admit(*packs[2])
    fl_mix = []
    for _ in range(3):
        mix.round(4)
        fl_mix.append(mix.poll(s_mix))
    assert mix.poll(other)[2] == 15
    assert fl_mix == fl_alone
    a = alone.pdfs(s_alone)
    m = mix.pdfs(s_mix)
    assert np.array_equal(a, m)
    alone.close()
    mix.close()


def test_release_reuse_and_capacity(L):
    packs = _packs()
    b = L.Batch(2 * 8192, variant="aa", precision="f32", max_geometries=2)
    s0 = b.admit(*packs[0])
    s1 = b.admit(*packs[2])
    with pytest.raises(L.LBMError) as e:
        b.admit(*packs[1])
    assert e.value.status == L.LBM_ERR_OOM
    b.release(s0)
    s2 = b.admit(*packs[1])
    assert s2 == s0
    b.round(2)
    assert b.info.active_geometries == 2
    small = L.Batch(8192, variant="aa", precision="f32", max_geometries=4)
    big = inputs.sphere_pack((30, 30, 30), 0.6, radius=3.0, seed=24)
    with pytest.raises(L.LBMError) as e:
        small.admit(big, 1.0, (1e-5, 0, 0))
    assert e.value.status == L.LBM_ERR_OOM and small.info.free_slots == 8192
    small.close()
    ref, _ = _oracle_steps(packs[1][0], packs[1][1], packs[1][2], 2)
    got = b.pdfs(s2)
    _, ug = oracle.macroscopics(got, packs[1][2])
    _, uo = oracle.macroscopics(ref, packs[1][2])
    assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= 1e-5
    b.close()


def test_tuner_picks_a_valid_shape(L):
    packs = _packs()
    b = L.Batch(3 * 16384, variant="aa", precision="f32", max_geometries=4)
    for p in packs:
        b.admit(*p)
    bs, npt, mflups = b.tune(rounds=1, k=4)
    assert bs in (64, 128, 256) and npt in (1, 2, 4) and mflups > 0
    assert (b.info.block_size, b.info.nodes_per_thread) == (bs, npt)
    b.round(2)
    b.close()


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
def test_folded_and_plain_idx_agree(L, precision):
    """The AA pattern's batch IDX with bounce-back slots folded in (the
    default below 2^30 slots) and with -1 kept for solid links give the same
    bits."""
    outs = []
    for keep in (0, 1):
        b = L.Batch(3 * 16384, variant="aa", precision=precision, max_geometries=8, keep_idx=keep,
                    f16_scale=2.0 ** 20 if precision == "f16s" else 0.0)
        slots = [b.admit(p, om, g) for p, om, g in _packs()]
        b.round(5)
        b.round(3)
        outs.append([b.pdfs(s) for s in slots] + [b.poll(s) for s in slots])
        b.close()
    for a, c in zip(outs[0], outs[1]):
        if isinstance(a, np.ndarray):
            assert np.array_equal(a, c)
        else:
            assert a == c
