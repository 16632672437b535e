"""Seeded synthetic inputs shared by the library's users, its tests and its
benchmark.  This module draws random numbers and lays out workload shapes; it
holds none of the lattice Boltzmann arithmetic (no collision, streaming,
geometry test or index building), so both the CUDA path and the CPU oracle may
consume what it produces.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value k of stream s under seed S is

    key   = mix64(mix64(S) ^ s)
    x_k   = mix64(key + (k + 1) * 0x9E3779B97F4A7C15)      (mod 2^64)

with mix64 the SplitMix64 output function.  A uniform double in [0, 1) is
(x_k >> 11) * 2^-53.

Workloads (shapes from the paper's porous-media benchmarks, Sec. 10, Fig. 7):
  * ``density_noise``  rho = 1 + amp * U[-1, 1) per cell;
  * ``sphere_pack``    overlapping spheres of radius r with uniform centres,
    count from the Boolean-model law porosity = exp(-n v_sphere / V), centres
    quantised to 1/unit lattice spacings (int64) so that the solid test can be
    done exactly in integers by both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids used by the workloads below.
STREAM_DENSITY = 1
STREAM_SPHERES = 2
STREAM_BATCH = 3
STREAM_ARRIVALS = 4
STREAM_STATE = 5


def mix64(z):
    """SplitMix64 output function on uint64 scalars or arrays (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Values start .. start+count-1 of the counter-based generator."""
    key = mix64(mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF)) ^ np.uint64(stream))
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + k * GOLDEN)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1)."""
    x = splitmix64(seed, stream, count, start)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def density_noise(dims, seed: int, amp: float = 1e-3) -> np.ndarray:
    """rho(x) = 1 + amp * xi with xi ~ U[-1, 1), one value per cell (x fastest)."""
    n = int(np.prod(dims))
    return 1.0 + amp * (2.0 * uniform(seed, STREAM_DENSITY, n) - 1.0)


@dataclass
class SpherePack:
    dims: tuple
    periodic: tuple
    centres: np.ndarray  # (nsph, 3) int64, in units of 1/unit cells
    radius: int  # in units of 1/unit cells
    unit: int
    porosity_target: float

    @property
    def nspheres(self) -> int:
        return int(self.centres.shape[0])


def sphere_count(dims, porosity: float, radius: float) -> int:
    """Boolean model of overlapping spheres: porosity = exp(-n v / V)."""
    vol = float(np.prod(dims))
    v = 4.0 / 3.0 * math.pi * radius ** 3
    return int(round(-math.log(porosity) * vol / v))


def sphere_pack(dims, porosity: float, radius: float = 8.0, seed: int = 3,
                periodic=(1, 1, 1), unit: int = 1024, stream: int = STREAM_SPHERES,
                start: int = 0) -> SpherePack:
    """Seeded overlapping spheres in a box; porosity is the fluid fraction."""
    dims = tuple(int(d) for d in dims)
    n = sphere_count(dims, porosity, radius)
    u = uniform(seed, stream, 3 * n, start).reshape(n, 3)
    scale = np.array(dims, dtype=np.float64) * unit
    centres = np.floor(u * scale).astype(np.int64)
    return SpherePack(dims, tuple(int(p) for p in periodic), centres,
                      int(round(radius * unit)), int(unit), float(porosity))


def paper_channel():
    """The empty channel of the paper's benchmarks (Sec. 10): 500 x 100 x 100
    cells, flow along x (periodic), bounce-back walls on the y and z faces;
    every cell is fluid (5.0 M)."""
    return (500, 100, 100), (1, 0, 0)


def paper_packed_bed(seed: int = 6, radius: float = 6.0, porosity: float = 0.42) -> SpherePack:
    """A packed bed of spheres in the paper's 500 x 100 x 100 box (Sec. 10,
    Fig. 7): overlapping spheres of radius 6 cells, porosity 0.42 so that the
    fluid cells number about 2.1 M as in the paper; periodic along the flow
    axis x, walls on the y and z faces."""
    return sphere_pack((500, 100, 100), porosity, radius, seed=seed, periodic=(1, 0, 0))


def duct(n: int = 32):
    """The 32^3 duct: periodic along x, bounce-back walls on the y and z faces."""
    return (n, n, n), (1, 0, 0)


@dataclass
class BatchItem:
    side: int
    porosity: float
    pack: SpherePack


def batch_packs(count: int = 64, seed: int = 4, side_range=(32, 192),
                porosity_range=(0.3, 0.8), radius: float = 8.0):
    """Uneven cubes for the batched permeability workload: side ~ U{lo..hi},
    porosity ~ U[lo, hi), each pack with its own sphere stream."""
    u = uniform(seed, STREAM_BATCH, 2 * count).reshape(count, 2)
    lo, hi = side_range
    items = []
    for k in range(count):
        side = lo + int(u[k, 0] * (hi - lo + 1))
        por = porosity_range[0] + u[k, 1] * (porosity_range[1] - porosity_range[0])
        pack = sphere_pack((side, side, side), por, radius, seed=seed * 1000 + k)
        items.append(BatchItem(side, float(por), pack))
    return items


def poisson_arrivals(count: int, rate: float, seed: int = 5):
    """Arrival times (s) of a Poisson process: exponential gaps, mean 1/rate."""
    u = uniform(seed, STREAM_ARRIVALS, count)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)
