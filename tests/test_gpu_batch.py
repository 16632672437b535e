"""Batched geometries (continuous batching) against the oracle, and the
same geometry alone and in a mix, with one launch per step or one persistent
launch per round: bit-identical states and fluxes.  Mask admission, the
library's steady-flux test and permeability against the oracle's; the
autotuner over variant, launch shape and round mode."""
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


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("variant", ["aa", "et"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_matches_oracle(L, variant, precision, mode):
    b = L.Batch(3 * 16384, variant=variant, precision=precision, max_geometries=8, round_mode=mode)
    slots = [b.admit(p, om, g) for p, om, g in _packs()]
    b.round(6)
    for s, (p, om, g) in zip(slots, _packs()):
        got = b.pdfs(s)
        ref, f0 = _oracle_steps(p, om, g, 6)
        m0, j0 = oracle.flux(f0, g)
        m, j, steps = b.flux(s)
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


@pytest.mark.parametrize("mix_npt", [2, 4])
@pytest.mark.parametrize("mix_mode", [0, 1])
@pytest.mark.parametrize("variant", ["aa", "et"])
@pytest.mark.parametrize("precision", ["f32", "f16s"])
def test_alone_equals_mix_bitwise(L, precision, variant, mix_mode, mix_npt):
    """One geometry alone and in a mix with other geometries admitted
    earlier and later, with the same launch shape (either round mode): the
    same PDF and flux bits.  Against a third run with another shape (256 x 1,
    per-step launches; with FP16 storage the AA pattern's mix runs node pairs
    and this one one node per thread): the same PDF bits, and flux sums that
    differ at most in the last bits (the threads group the nodes' FP64
    terms differently)."""
    packs = _packs()
    target = packs[0]
    kw = {"f16_scale": 2.0 ** 20} if precision == "f16s" else {}
    shape = dict(block_size=512 if mix_mode else 128, nodes_per_thread=mix_npt, round_mode=mix_mode)

    def run_alone(**sh):
        b = L.Batch(16384, variant=variant, precision=precision, max_geometries=4, **sh, **kw)
        s = b.admit(*target)
        fl = []
        for _ in range(3):
            b.round(4)
            fl.append(b.flux(s))
        out = b.pdfs(s)
        b.close()
        return fl, out

    fl_alone, a = run_alone(**shape)
    fl_ref, r = run_alone(block_size=256, nodes_per_thread=1)
    mix = L.Batch(4 * 16384, variant=variant, precision=precision, max_geometries=8, **shape, **kw)
    other = mix.admit(*packs[1])
    mix.round(3)  # the other geometry is at an odd step count when the target arrives
    s_mix = mix.admit(*target)
    mix.admit(*packs[2])
    fl_mix = []
    for _ in range(3):
        mix.round(4)
        fl_mix.append(mix.flux(s_mix))
    assert mix.flux(other)[2] == 15
    m = mix.pdfs(s_mix)
    mix.close()
    assert fl_mix == fl_alone
    assert np.array_equal(a, m) and np.array_equal(r, m)
    for (ma, ja, sa), (mb, jb, sb) in zip(fl_mix, fl_ref):
        assert sa == sb and abs(ma - mb) <= 1e-12 * mb and abs(ja - jb) <= 1e-12 * max(abs(jb), 1e-30)


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


@pytest.mark.parametrize("tune_variant", [0, 1])
def test_tuner_picks_a_valid_configuration(L, tune_variant):
    """The autotuner returns one of its candidates, leaves every geometry at
    rest in it, and the tuned batch then matches the oracle."""
    packs = _packs()
    b = L.Batch(4 * 16384, variant="aa", precision="f32", max_geometries=4, tune_variant=tune_variant)
    slots = [b.admit(*p) for p in packs]
    b.round(3)
    v, bs, npt, mode, mflups = b.tune(rounds=1, k=4)
    assert v in ((L.LBM_AA, L.LBM_ET) if tune_variant else (L.LBM_AA,))
    assert bs in (128, 256, 512) and npt in (1, 2, 4, 8) and mode in (0, 1) and mflups > 0
    i = b.info
    assert (i.variant, i.block_size, i.nodes_per_thread, i.round_mode) == (v, bs, npt, mode)
    assert all(b.slot_info(s)[2] == 0 for s in slots)
    b.round(6)
    for s, (p, om, g) in zip(slots, packs):
        ref, _ = _oracle_steps(p, om, g, 6)
        _, ug = oracle.macroscopics(b.pdfs(s), g)
        _, uo = oracle.macroscopics(ref, g)
        assert np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) <= 1e-5
    b.close()


@pytest.mark.parametrize("start", ["aa", "et"])
def test_tuned_variant_equals_fixed(L, start):
    """A batch whose variant may be tuned is relaid out for both variants
    while tuning and for the chosen one at the end; afterwards it gives the
    same bits as a batch built for that variant."""
    packs = _packs()
    tun = L.Batch(4 * 16384, variant=start, precision="f32", max_geometries=4, tune_variant=1)
    ts = [tun.admit(*p) for p in packs]
    tun.round(3)
    v, _, _, _, _ = tun.tune(rounds=1, k=2)
    tun.round(6)
    fixed = L.Batch(4 * 16384, variant="aa" if v == L.LBM_AA else "et", precision="f32", max_geometries=4)
    fs = [fixed.admit(*p) for p in packs]
    fixed.round(6)
    for a, c in zip(fs, ts):
        assert np.array_equal(fixed.pdfs(a), tun.pdfs(c))
    fixed.close()
    tun.close()


def _random_mask(dims, solid_frac, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(int(np.prod(dims))) < solid_frac).astype(np.uint8)


def _oracle_solve(mask, dims, per, omega, g, k_round=100, tol=1e-6, cap=200000):
    cells, node_of = oracle.build_nodes(dims, per, mask)
    idx = oracle.build_idx(dims, per, mask, cells, node_of)
    f = oracle.rest_state(cells.size)
    prev, steps = None, 0
    while steps < cap:
        _, phi = oracle.flux(f, g)  # state at the start of the round
        f = oracle.run_sparse(idx, f, k_round, omega, g)
        steps += k_round
        if prev is not None and abs(phi - prev) < tol * abs(phi):
            break
        prev = phi
    return oracle.permeability(phi, int(np.prod(dims)), omega, g[0]), steps


@pytest.mark.parametrize("variant,precision,tol_k", [("aa", "f64", 1e-10), ("et", "f32", 1e-5),
                                                     ("aa", "f16s", 1e-3)])
def test_mask_admission_steady_flux_and_permeability(L, variant, precision, tol_k):
    """A random (not sphere) solid mask admitted through lbm_batch_admit,
    beside a sphere pack: the library's steady-flux test stops it where the
    oracle's rule does, and its permeability matches the oracle's."""
    dims, per, omega, g = (18, 14, 12), (1, 1, 1), 1.0, (1e-5, 0.0, 0.0)
    mask = _random_mask(dims, 0.25, 41)
    k_ora, steps_ora = _oracle_solve(mask, dims, per, omega, g)
    b = L.Batch(4 * 16384, variant=variant, precision=precision, max_geometries=4,
                f16_scale=2.0 ** 20 if precision == "f16s" else 0.0)
    s = b.admit_mask(mask, dims, per, omega, g, tol=1e-6, max_steps=100000)
    other = b.admit(*_packs()[0], tol=1e-6)
    assert b.slot_info(s)[0] == int((mask == 0).sum())
    done = 0
    while not done:
        b.round(100)
        done, k, steps = b.poll(s)
    assert done == 1
    if precision != "f16s":
        assert steps == steps_ora
    assert abs(k - k_ora) <= tol_k * k_ora, (k, k_ora)
    assert b.poll(other)[2] == steps
    b.close()


def test_step_cap_and_release_from_poll(L):
    b = L.Batch(2 * 16384, variant="aa", precision="f32", max_geometries=4)
    p, om, g = _packs()[0]
    s = b.admit(p, om, g, tol=0.0, max_steps=300)  # tol 0: never steady
    states = []
    for _ in range(3):
        b.round(100)
        states.append(b.poll(s))
    assert [d for d, _, _ in states] == [0, 0, 2] and states[-1][2] == 300
    assert np.isfinite(states[-1][1]) and states[-1][1] > 0
    zero_g = b.admit(p, om, (0.0, 0.0, 0.0), tol=1e-6)
    b.round(2)
    assert np.isnan(b.poll(zero_g)[1])
    b.close()


@pytest.mark.parametrize("npt", [1, 2, 8])
@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
def test_folded_and_plain_idx_agree(L, precision, npt):
    """The AA pattern's batch IDX with bounce-back slots folded in (the
    default below 2^30 slots) and with -1 kept for solid links give the same
    bits (FP16 with two or eight nodes per thread: node pairs)."""
    outs = []
    for keep in (0, 1):
        b = L.Batch(3 * 16384, variant="aa", precision=precision, max_geometries=8, keep_idx=keep,
                    block_size=128, nodes_per_thread=npt, f16_scale=2.0 ** 20 if precision == "f16s" else 0.0)
        slots = [b.admit(p, om, g) for p, om, g in _packs()]
        b.round(5)
        b.round(3)
        outs.append([b.pdfs(s) for s in slots] + [b.flux(s) for s in slots])
        b.close()
    for a, c in zip(outs[0], outs[1]):
        if isinstance(a, np.ndarray):
            assert np.array_equal(a, c)
        else:
            assert a == c
