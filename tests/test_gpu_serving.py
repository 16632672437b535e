"""Continuous-batching service on the GPU: every request's permeability and
step count are the same when it is served among others as when it is served
alone, and agree with the oracle's solve (FP32 1e-5, FP16 storage 1e-3)."""
import numpy as np
import pytest

import oracle
from paper_1111_0922_gb300 import serving

pytestmark = pytest.mark.gpu

TOL_K = {"f32": 1e-5, "f16s": 1e-3}


def _requests():
    return serving.poisson_requests(4, 500.0, seed=17, side_range=(20, 28), porosity_range=(0.5, 0.8),
                                    radius=4.0, force=(1e-5, 0.0, 0.0))


def _oracle_k(req):
    p = req.pack
    mask = oracle.sphere_mask(p.dims, p.periodic, p.centres, p.radius, p.unit)
    cells, node_of = oracle.build_nodes(p.dims, p.periodic, mask)
    idx = oracle.build_idx(p.dims, p.periodic, mask, cells, node_of)
    f = oracle.rest_state(cells.size)
    prev = None
    for _ in range(2000):
        _, phi = oracle.flux(f, req.force)
        f = oracle.run_sparse(idx, f, 100, req.omega, req.force)
        if prev is not None and abs(phi - prev) < 1e-6 * abs(phi):
            break
        prev = phi
    return oracle.permeability(phi, int(np.prod(p.dims)), req.omega, req.force[0])


@pytest.mark.parametrize("precision", ["f32", "f16s"])
def test_served_results_equal_alone_and_match_oracle(precision):
    from paper_1111_0922_gb300 import build

    build.build()
    reqs = _requests()
    cap = 6 * 16384
    eng = serving.BatchEngine(cap, precision=precision, f16_scale=2.0 ** 20, max_geometries=8)
    mixed = serving.serve(reqs, eng, serving.RealClock(), k_round=100)
    eng.close()
    assert len(mixed.results) == len(reqs) and all(r.converged for r in mixed.results)
    for res in mixed.results:
        req = reqs[res.rid]
        eng1 = serving.BatchEngine(cap, precision=precision, f16_scale=2.0 ** 20, max_geometries=8)
        alone = serving.serve([serving.Request(req.rid, 0.0, req.pack, req.omega, req.force)], eng1,
                              serving.RealClock(), k_round=100)
        eng1.close()
        assert alone.results[0].k == res.k and alone.results[0].steps == res.steps
        k_ora = _oracle_k(req)
        assert abs(res.k - k_ora) <= TOL_K[precision] * k_ora, (res.k, k_ora)
    s = mixed.summary()
    assert s["completed"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"]
