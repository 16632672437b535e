"""Continuous-batching permeability service.

Requests (a sphere-pack geometry, omega, force) arrive over time.  They are
admitted into a shared batch of node-list segments as device memory frees up
(the batch's capacity is the HBM budget divided by the bytes per node slot),
advanced together in rounds of `k_round` steps, and retired when the library
reports their flux steady (relative change below `tol` between two rounds) or
their step cap reached; the permeability comes from the library too.  Each
round's first step also reduces every geometry's flux, so convergence checks
cost no extra pass.  Admission runs while a round is in flight: the geometry
is built on the library's second stream and joins the next round.  Reports
latency (arrival to result) and throughput.

The engine is anything with the small interface of `BatchEngine` (the GPU
batch); tests drive the same loop with a CPU stand-in and a simulated clock.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    pack: inputs.SpherePack
    omega: float = 1.0
    force: tuple = (1e-6, 0.0, 0.0)


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    k: float
    steps: int
    nodes: int
    converged: bool

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    slot: int
    admitted: float
    nodes: int


class RealClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def wait_until(self, t: float) -> None:
        dt = t - self.now()
        if dt > 0:
            time.sleep(dt)


class SimClock:
    """A clock that advances only when told (CPU tests)."""

    def __init__(self):
        self.t = 0.0

    def now(self) -> float:
        return self.t

    def wait_until(self, t: float) -> None:
        self.t = max(self.t, t)

    def advance(self, dt: float) -> None:
        self.t += dt


class OutOfCapacity(Exception):
    """The engine has no room for a geometry right now."""


class BatchEngine:
    """The GPU batch (lbm.Batch) behind the serving interface."""

    def __init__(self, capacity_slots, variant="aa", precision="f16s", f16_scale=2.0 ** 22,
                 max_geometries=4096, block_size=0, nodes_per_thread=0, round_mode=0):
        from . import lbm

        self.lbm = lbm
        self.batch = lbm.Batch(capacity_slots, variant=variant, precision=precision,
                               max_geometries=max_geometries, f16_scale=f16_scale,
                               block_size=block_size, nodes_per_thread=nodes_per_thread, round_mode=round_mode)

    def admit(self, req: Request, tol: float, max_steps: int) -> tuple[int, int]:
        try:
            slot = self.batch.admit(req.pack, req.omega, req.force, tol, max_steps)
        except self.lbm.LBMError as e:
            if e.status == self.lbm.LBM_ERR_OOM:
                raise OutOfCapacity(str(e)) from e
            raise
        nodes, _, _ = self.batch.slot_info(slot)
        return slot, nodes

    def release(self, slot: int) -> None:
        self.batch.release(slot)

    def round(self, k: int) -> None:
        """Enqueue k steps of every active geometry (returns at once)."""
        self.batch.round(k)

    def poll(self, slot: int):
        """(done, permeability, steps) after the last round: done 0 running,
        1 steady, 2 step cap."""
        return self.batch.poll(slot)

    def close(self):
        self.batch.close()


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    rounds: int = 0
    node_updates: int = 0
    rejected: int = 0
    wall: float = 0.0

    def summary(self) -> dict:
        served = [r for r in self.results if r.nodes > 0]
        lat = np.array([r.latency for r in served]) if served else np.zeros(1)
        done = [r for r in self.results if r.converged]
        span = (max(r.finished for r in self.results) - min(r.arrival for r in self.results)) \
            if self.results else 0.0
        return {
            "completed": len(served), "converged": len(done), "rejected": self.rejected,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()),
            "solves_per_s": len(self.results) / span if span > 0 else 0.0,
            "rounds": self.rounds, "node_updates": self.node_updates,
            "mflups": self.node_updates / self.wall / 1e6 if self.wall > 0 else 0.0,
            "wall_s": self.wall,
        }


def serve(requests, engine, clock=None, k_round: int = 100, tol: float = 1e-6, max_steps: int = 200000,
          on_round=None) -> ServeStats:
    """Run the requests (sorted by arrival) to completion through `engine`.

    Each loop iteration: enqueue one round on every active geometry; while it
    runs, admit every arrived request that fits (FIFO; a request that does
    not fit waits and blocks the ones behind it), so its geometry build
    overlaps the round; then read the round's results and retire the
    geometries the engine reports steady or at `max_steps` (the latter with
    converged = False).  The admitted requests join the next round."""
    clock = clock or RealClock()
    queue = sorted(requests, key=lambda r: r.arrival)
    qi = 0
    active: dict[int, _Active] = {}
    stats = ServeStats()
    t_start = clock.now()
    while qi < len(queue) or active:
        launched = bool(active)
        if launched:
            engine.round(k_round)
            stats.rounds += 1
            stats.node_updates += k_round * sum(a.nodes for a in active.values())
            if on_round:
                on_round(clock, k_round, active)
        newly: dict[int, _Active] = {}
        now = clock.now()
        while qi < len(queue) and queue[qi].arrival <= now:
            try:
                slot, nodes = engine.admit(queue[qi], tol, max_steps)
            except OutOfCapacity:
                if not active and not newly:  # does not fit even in an empty engine: reject it
                    r = queue[qi]
                    stats.results.append(Result(r.rid, r.arrival, clock.now(), clock.now(), float("nan"), 0, 0,
                                                False))
                    stats.rejected += 1
                    qi += 1
                    continue
                break
            newly[slot] = _Active(queue[qi], slot, clock.now(), nodes)
            qi += 1
        if launched:
            for slot in list(active):
                a = active[slot]
                done, k, steps = engine.poll(slot)
                if done:
                    stats.results.append(Result(a.req.rid, a.req.arrival, a.admitted, clock.now(), k, int(steps),
                                                a.nodes, done == 1))
                    engine.release(slot)
                    del active[slot]
        active.update(newly)
        if not active and qi < len(queue):
            clock.wait_until(queue[qi].arrival)
    stats.wall = clock.now() - t_start
    return stats


def poisson_requests(count: int, rate: float, seed: int = 5, side_range=(64, 384),
                     porosity_range=(0.3, 0.8), radius: float = 8.0, omega: float = 1.0,
                     force=(1e-6, 0.0, 0.0)):
    """Seeded request trace: Poisson arrivals, cube side ~ U{lo..hi},
    porosity ~ U[lo, hi), overlapping spheres of the given radius."""
    t = inputs.poisson_arrivals(count, rate, seed)
    u = inputs.uniform(seed, inputs.STREAM_STATE, 2 * count).reshape(count, 2)
    reqs = []
    for i in range(count):
        side = side_range[0] + int(u[i, 0] * (side_range[1] - side_range[0] + 1))
        por = porosity_range[0] + u[i, 1] * (porosity_range[1] - porosity_range[0])
        pack = inputs.sphere_pack((side, side, side), por, radius, seed=seed * 100000 + i)
        reqs.append(Request(i, float(t[i]), pack, omega, tuple(force)))
    return reqs
