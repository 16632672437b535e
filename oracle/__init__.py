"""Plain FP64 CPU oracle for the D3Q19 lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never calls it, and it shares no code with the CUDA path.

The arithmetic lives in ``lbm_oracle.c`` (plain loops, FP64, built with
``-ffp-contract=off``); this module only compiles it and marshals numpy
arrays.  Every PDF array is natural: ``f[i, node]`` with shape ``(19, n)``.

Parity status of each function (pins live in ``tests/test_oracle_*.py``):
  collide / push steps  pinned (Poiseuille closed form, conservation laws,
                        fixed points, shear-wave decay, streaming permutation)
  variants              pinned (all schemes equal after even step counts,
                        identity collision returns to the start)
  geometry, IDX         pinned (brute force on small boxes, porosity law)
  permeability          pinned through the Poiseuille slit (k = (H^2+8L-1)/12)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
VARIANTS = {"ts": 0, "os_push": 1, "os_pull": 2, "cg": 3, "swap": 4, "aa": 5, "et": 6}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        sig = {
            "ora_lattice": (None, [P, P]),
            "ora_collide": (None, [P, D, P, P]),
            "ora_node_moments": (None, [P, P, P, P]),
            "ora_equilibrium": (None, [D, P, P]),
            "ora_push_full": (None, [P, P, P, P, P, D, P, I]),
            "ora_build_nodes": (I64, [P, P, P, P, P]),
            "ora_build_idx": (None, [P, P, P, P, P, I64, P]),
            "ora_push_sparse": (None, [I64, P, P, P, D, P, I]),
            "ora_collide_nodes": (None, [I64, P, I64, P, D, P, P]),
            "ora_macroscopics": (None, [I64, P, P, P, P]),
            "ora_flux": (None, [I64, P, P, P, P, P]),
            "ora_sphere_mask": (None, [P, P, I64, P, I64, I64, P]),
            "ora_run_variant": (I, [I, P, P, P, P, P, I, D, P]),
            "ora_run_push_full": (None, [P, P, P, P, I, D, P, I]),
            "ora_run_push_sparse": (None, [I64, P, P, I, D, P, I]),
            "ora_collide_trt": (None, [P, D, D, P, P]),
            "ora_trt_lambda_minus": (D, [D, D]),
            "ora_run_push_full_trt": (None, [P, P, P, P, I, D, D, P, I]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _vec3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


def _mask(solid, n):
    if solid is None:
        return None
    m = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
    assert m.size == n
    return m


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def lattice():
    """(c, w): the oracle's velocity set (19, 3) int and weights (19,)."""
    lib = _load()
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q, np.float64)
    lib.ora_lattice(_p(c), _p(w))
    return c, w


def collide(f, omega, g=(0.0, 0.0, 0.0)):
    """Post-collision PDFs of one node (BGK + Guo force)."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(Q))
    out = np.zeros(Q)
    gv = _vec3(g)
    lib.ora_collide(_p(f), float(omega), _p(gv), _p(out))
    return out


def collide_trt(f, lam_p, lam_m, g=(0.0, 0.0, 0.0)):
    """Post-collision PDFs of one node with the two-relaxation-time model."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(Q))
    out = np.zeros(Q)
    gv = _vec3(g)
    lib.ora_collide_trt(_p(f), float(lam_p), float(lam_m), _p(gv), _p(out))
    return out


def trt_lambda_minus(lam_p, magic=3.0 / 16.0):
    return float(_load().ora_trt_lambda_minus(float(lam_p), float(magic)))


def run_push_trt(dims, periodic, solid, f, nsteps, lam_p, lam_m, g=(0.0, 0.0, 0.0), nthreads=None):
    """nsteps of the definition with the TRT collision on a full grid."""
    lib = _load()
    n = int(np.prod(dims))
    f = np.array(np.asarray(f, np.float64).reshape(Q, n), order="C", copy=True)
    gv = _vec3(g)
    lib.ora_run_push_full_trt(_p(_dims(dims)), _p(_dims(periodic)), _p(_mask(solid, n)), _p(f), int(nsteps),
                              float(lam_p), float(lam_m), _p(gv), int(nthreads or default_threads()))
    return f


def equilibrium(rho, u):
    lib = _load()
    uv = _vec3(u)
    out = np.zeros(Q)
    lib.ora_equilibrium(float(rho), _p(uv), _p(out))
    return out


def equilibrium_field(rho, u):
    """Natural state f_i = f_eq(rho(x), u(x)); rho (n,), u (n, 3)."""
    rho = np.asarray(rho, np.float64).reshape(-1)
    u = np.asarray(u, np.float64).reshape(-1, 3)
    out = np.zeros((Q, rho.size))
    for k in range(rho.size):
        out[:, k] = equilibrium(rho[k], u[k])
    return out


def rest_state(n, rho0=1.0):
    _, w = lattice()
    return np.ascontiguousarray(np.outer(w, np.full(n, rho0)))


def push_full(dims, periodic, solid, f, omega, g=(0.0, 0.0, 0.0), nthreads=None):
    """One time step f -> S(C(f)) on a full grid (the definition)."""
    lib = _load()
    n = int(np.prod(dims))
    f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(Q, n))
    out = np.empty_like(f)
    gv = _vec3(g)
    lib.ora_push_full(_p(_dims(dims)), _p(_dims(periodic)), _p(_mask(solid, n)), _p(f), _p(out),
                      float(omega), _p(gv), int(nthreads or default_threads()))
    return out


def build_nodes(dims, periodic, solid):
    """(cells, node_of): lexicographic fluid-node list and the dense map."""
    lib = _load()
    n = int(np.prod(dims))
    node_of = np.empty(n, np.int32)
    cells = np.empty(n, np.int32)
    cnt = lib.ora_build_nodes(_p(_dims(dims)), _p(_dims(periodic)), _p(_mask(solid, n)),
                              _p(node_of), _p(cells))
    return cells[:cnt].copy(), node_of


def build_idx(dims, periodic, solid, cells=None, node_of=None):
    """IDX array (18, N): neighbour node numbers along c_1..c_18, -1 = solid/wall."""
    lib = _load()
    if cells is None:
        cells, node_of = build_nodes(dims, periodic, solid)
    n = int(np.prod(dims))
    N = cells.size
    idx = np.empty((Q - 1, N), np.int32)
    lib.ora_build_idx(_p(_dims(dims)), _p(_dims(periodic)), _p(_mask(solid, n)), _p(node_of),
                      _p(np.ascontiguousarray(cells)), N, _p(idx))
    return idx


def push_sparse(idx, f, omega, g=(0.0, 0.0, 0.0), nthreads=None):
    """One time step on a node list with IDX (the same definition)."""
    lib = _load()
    idx = np.ascontiguousarray(idx, np.int32)
    N = idx.shape[1]
    f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(Q, N))
    out = np.empty_like(f)
    gv = _vec3(g)
    lib.ora_push_sparse(N, _p(idx), _p(f), _p(out), float(omega), _p(gv),
                        int(nthreads or default_threads()))
    return out


def collide_nodes(f, sample, omega, g=(0.0, 0.0, 0.0)):
    """Post-collision PDFs (len(sample), 19) of sampled nodes of state f (19, n)."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, np.float64))
    n = f.shape[1]
    s = np.ascontiguousarray(np.asarray(sample, np.int64))
    out = np.empty((s.size, Q))
    gv = _vec3(g)
    lib.ora_collide_nodes(n, _p(f), s.size, _p(s), float(omega), _p(gv), _p(out))
    return out


def macroscopics(f, g=(0.0, 0.0, 0.0)):
    """(rho (n,), u (n, 3)) of a natural state; u includes the half force."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, np.float64))
    n = f.shape[1]
    rho = np.empty(n)
    u = np.empty((n, 3))
    gv = _vec3(g)
    lib.ora_macroscopics(n, _p(f), _p(gv), _p(rho), _p(u))
    return rho, u


def flux(f, g=(0.0, 0.0, 0.0), skip=None):
    """(mass, jx) = (sum rho, sum rho u_x) over the nodes not flagged in skip."""
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f, np.float64))
    n = f.shape[1]
    m = ctypes.c_double()
    j = ctypes.c_double()
    gv = _vec3(g)
    sk = None if skip is None else np.ascontiguousarray(np.asarray(skip, np.uint8))
    lib.ora_flux(n, _p(f), _p(gv), _p(sk), ctypes.byref(m), ctypes.byref(j))
    return m.value, j.value


def sphere_mask(dims, periodic, centres, radius, unit):
    """Solid mask (uint8, x fastest) of overlapping spheres, exact integer test."""
    lib = _load()
    n = int(np.prod(dims))
    c = np.ascontiguousarray(np.asarray(centres, np.int64).reshape(-1, 3))
    out = np.empty(n, np.uint8)
    lib.ora_sphere_mask(_p(_dims(dims)), _p(_dims(periodic)), c.shape[0], _p(c), int(radius),
                        int(unit), _p(out))
    return out


def run_variant(variant, dims, periodic, solid, f, nsteps, omega, g=(0.0, 0.0, 0.0)):
    """Run nsteps with one of the paper's propagation schemes (serial form) and
    return the natural state.  variant: ts, os_push, os_pull, cg, swap, aa, et."""
    lib = _load()
    n = int(np.prod(dims))
    f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(Q, n))
    out = np.empty_like(f)
    gv = _vec3(g)
    rc = lib.ora_run_variant(VARIANTS[variant], _p(_dims(dims)), _p(_dims(periodic)),
                             _p(_mask(solid, n)), _p(f), _p(out), int(nsteps), float(omega), _p(gv))
    if rc != 0:
        raise ValueError("oracle variant %s rejected its arguments" % variant)
    return out


def run_push(dims, periodic, solid, f, nsteps, omega, g=(0.0, 0.0, 0.0), nthreads=None):
    """nsteps of the definition on a full grid; returns the new natural state."""
    lib = _load()
    n = int(np.prod(dims))
    f = np.array(np.asarray(f, np.float64).reshape(Q, n), order="C", copy=True)
    gv = _vec3(g)
    lib.ora_run_push_full(_p(_dims(dims)), _p(_dims(periodic)), _p(_mask(solid, n)), _p(f),
                          int(nsteps), float(omega), _p(gv), int(nthreads or default_threads()))
    return f


def run_sparse(idx, f, nsteps, omega, g=(0.0, 0.0, 0.0), nthreads=None):
    """nsteps of the definition on a node list; returns the new natural state."""
    lib = _load()
    idx = np.ascontiguousarray(idx, np.int32)
    N = idx.shape[1]
    f = np.array(np.asarray(f, np.float64).reshape(Q, N), order="C", copy=True)
    gv = _vec3(g)
    lib.ora_run_push_sparse(N, _p(idx), _p(f), int(nsteps), float(omega), _p(gv),
                            int(nthreads or default_threads()))
    return f


def permeability(jx_sum, n_box, omega, gx):
    """k = nu <u_x> / g with <u_x> the superficial velocity (sum over fluid
    nodes of rho u_x, divided by the number of cells of the box, rho ~ 1)."""
    nu = (1.0 / omega - 0.5) / 3.0
    return nu * (jx_sum / n_box) / gx
