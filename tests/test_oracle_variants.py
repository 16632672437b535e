"""Pins of the paper's propagation schemes as written in the oracle (serial
forms of Sec. 2-7): each must reproduce the definition f -> S(C(f)) exactly
after an even number of steps, with walls, solids, periodic axes and a body
force, and with the identity collision each must return to its start."""
import numpy as np
import pytest

VARIANTS = ["ts", "os_push", "os_pull", "cg", "swap", "aa", "et"]


def _case(ora, dims, per, frac, seed):
    n = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    solid = (rng.random(n) < frac).astype(np.uint8)
    f = ora.rest_state(n) * (1 + 0.05 * (rng.random((19, n)) - 0.5))
    return solid, f


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dims,per,frac", [((6, 5, 4), (1, 0, 1), 0.1),
                                           ((5, 7, 3), (1, 1, 1), 0.0),
                                           ((4, 4, 5), (0, 0, 0), 0.2),
                                           ((7, 3, 6), (0, 1, 0), 0.15)])
def test_variant_equals_definition(ora, variant, dims, per, frac):
    solid, f0 = _case(ora, dims, per, frac, seed=sum(dims))
    g = (1e-4, -3e-5, 2e-5)
    ref = ora.run_push(dims, per, solid, f0, 6, 1.3, g)
    out = ora.run_variant(variant, dims, per, solid, f0, 6, 1.3, g)
    fl = solid == 0
    assert np.array_equal(out[:, fl], ref[:, fl])


@pytest.mark.parametrize("variant", [v for v in VARIANTS if v != "aa"])
def test_variant_odd_steps(ora, variant):
    dims, per = (5, 6, 4), (1, 0, 1)
    solid, f0 = _case(ora, dims, per, 0.1, seed=9)
    ref = ora.run_push(dims, per, solid, f0, 3, 0.9)
    out = ora.run_variant(variant, dims, per, solid, f0, 3, 0.9)
    fl = solid == 0
    assert np.array_equal(out[:, fl], ref[:, fl])


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_identity_returns(ora, variant):
    dims, per = (4, 6, 3), (1, 1, 1)
    _, f0 = _case(ora, dims, per, 0.0, seed=11)
    out = ora.run_variant(variant, dims, per, None, f0, 12, 0.0)
    assert np.array_equal(out, f0)
    out = ora.run_variant(variant, dims, per, None, f0, 2, 0.0)
    assert not np.array_equal(out, f0)


def test_aa_rejects_odd_count(ora):
    dims = (4, 4, 4)
    with pytest.raises(ValueError):
        ora.run_variant("aa", dims, (1, 1, 1), None, ora.rest_state(64), 3, 1.0)
