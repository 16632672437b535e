"""The continuous-batching loop on the CPU: a stand-in engine built on the
oracle (tiny boxes), a simulated clock.  Checks admission under a capacity
limit, FIFO order, retirement, rejection, the step cap, latency accounting,
and that every result equals the same geometry solved alone."""
import math

import numpy as np

import oracle
from paper_1111_0922_gb300 import serving


class OracleEngine:
    """Same interface as serving.BatchEngine; capacity in fluid nodes;
    a round costs `nodes * k / rate` simulated seconds.  Like the library,
    it decides convergence itself (relative flux change between rounds) and
    reports the permeability from the oracle's flux."""

    def __init__(self, capacity, clock, rate=2e5):
        self.capacity, self.clock, self.rate = capacity, clock, rate
        self.used = 0
        self.slots = {}
        self.max_used = 0
        self.order = []

    def admit(self, req, tol, max_steps):
        p = req.pack
        mask = oracle.sphere_mask(p.dims, p.periodic, p.centres, p.radius, p.unit)
        cells, node_of = oracle.build_nodes(p.dims, p.periodic, mask)
        n = cells.size
        if self.used + n > self.capacity:
            raise serving.OutOfCapacity("full")
        idx = oracle.build_idx(p.dims, p.periodic, mask, cells, node_of)
        slot = min(set(range(len(self.slots) + 1)) - set(self.slots))
        self.slots[slot] = dict(req=req, idx=idx, f=oracle.rest_state(n), steps=0, flux=0.0, prev=None, done=0,
                                tol=tol, max_steps=max_steps, pending=False)
        self.used += n
        self.max_used = max(self.max_used, self.used)
        self.order.append(req.rid)
        return slot, n

    def release(self, slot):
        self.used -= self.slots[slot]["idx"].shape[1]
        del self.slots[slot]

    def round(self, k):
        total = 0
        for s in self.slots.values():
            r = s["req"]
            _, s["flux"] = oracle.flux(s["f"], r.force)
            s["f"] = oracle.run_sparse(s["idx"], s["f"], k, r.omega, r.force, nthreads=1)
            s["steps"] += k
            s["pending"] = True
            total += s["idx"].shape[1]
        self.clock.advance(total * k / self.rate)

    def poll(self, slot):
        s = self.slots[slot]
        if s["pending"] and not s["done"]:
            steady = s["prev"] is not None and abs(s["flux"] - s["prev"]) < s["tol"] * abs(s["flux"])
            s["prev"] = s["flux"]
            s["done"] = 1 if steady else (2 if s["steps"] >= s["max_steps"] else 0)
        s["pending"] = False
        r = s["req"]
        k = oracle.permeability(s["flux"], int(np.prod(r.pack.dims)), r.omega, r.force[0])
        return s["done"], k, s["steps"]


def _requests(n=5, rate=50.0):
    return serving.poisson_requests(n, rate, seed=7, side_range=(8, 12), porosity_range=(0.5, 0.8),
                                    radius=2.0, force=(1e-5, 0.0, 0.0))


def _alone(req, k_round=20, tol=1e-6):
    clock = serving.SimClock()
    eng = OracleEngine(10 ** 9, clock)
    st = serving.serve([serving.Request(req.rid, 0.0, req.pack, req.omega, req.force)], eng, clock,
                       k_round=k_round, tol=tol)
    return st.results[0]


def test_serving_results_equal_alone_and_capacity_respected():
    reqs = _requests()
    sizes = []
    for r in reqs:
        m = oracle.sphere_mask(r.pack.dims, r.pack.periodic, r.pack.centres, r.pack.radius, r.pack.unit)
        sizes.append(int((m == 0).sum()))
    cap = max(sizes) + min(sizes)  # at most two geometries at a time
    clock = serving.SimClock()
    eng = OracleEngine(cap, clock)
    seen = []
    st = serving.serve(reqs, eng, clock, k_round=20, tol=1e-6,
                       on_round=lambda c, k, act: seen.append(sum(a.nodes for a in act.values())))
    assert len(st.results) == len(reqs) and all(r.converged for r in st.results)
    assert max(seen) <= cap and eng.max_used <= cap
    assert eng.order == sorted(eng.order)  # FIFO admission
    for res in st.results:
        alone = _alone(reqs[res.rid])
        assert res.k == alone.k and res.steps == alone.steps
        assert res.finished >= res.admitted >= res.arrival
    s = st.summary()
    assert s["completed"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_rejects_geometry_larger_than_engine():
    reqs = _requests(2)
    clock = serving.SimClock()
    st = serving.serve(reqs, OracleEngine(10, clock), clock, k_round=20)
    assert st.rejected == 2 and all(math.isnan(r.k) for r in st.results)


def test_step_cap_reports_unconverged():
    reqs = _requests(1)
    clock = serving.SimClock()
    st = serving.serve(reqs, OracleEngine(10 ** 9, clock), clock, k_round=20, tol=1e-14, max_steps=60)
    assert len(st.results) == 1 and not st.results[0].converged and st.results[0].steps == 60


def test_poisson_trace_is_seeded():
    a = serving.poisson_requests(20, 20.0, seed=5, side_range=(64, 384))
    b = serving.poisson_requests(20, 20.0, seed=5, side_range=(64, 384))
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(64 <= r.pack.dims[0] <= 384 for r in a)
    gaps = np.diff([0.0] + [r.arrival for r in serving.poisson_requests(2000, 20.0, seed=6,
                                                                         side_range=(8, 8))])
    assert abs(gaps.mean() - 1 / 20.0) < 0.005
