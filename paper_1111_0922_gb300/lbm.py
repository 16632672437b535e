"""Thin ctypes binding of liblbm (include/lbm.h).

The functions here carry the C names and only marshal arguments: every step
of the computation runs in the library's CUDA kernels.  Loading fails loudly
when ``liblbm.so`` has not been built; there is no CPU fallback.

PyTorch is used only for plumbing: the default device allocator hands the
library PyTorch's caching allocator, and the default stream is PyTorch's
current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

# enums of include/lbm.h
LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_STATE, LBM_ERR_BOUNDS, \
    LBM_ERR_TIMEOUT, LBM_ERR_NOT_CONVERGED, LBM_ERR_UNSUPPORTED = range(9)
LBM_TS, LBM_OS_PUSH, LBM_OS_PULL, LBM_CG, LBM_SWAP, LBM_AA, LBM_ET = range(7)
LBM_DIRECT, LBM_INDIRECT = 0, 1
LBM_SOA, LBM_AOS = 0, 1
LBM_F64, LBM_F32, LBM_F16S = 0, 1, 2

VARIANTS = {"ts": LBM_TS, "os_push": LBM_OS_PUSH, "os_pull": LBM_OS_PULL, "cg": LBM_CG,
            "swap": LBM_SWAP, "aa": LBM_AA, "et": LBM_ET}
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S}
Q = 19

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class lbm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32 * 3),
                ("variant", ctypes.c_int32), ("addressing", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("omega", ctypes.c_double), ("force", ctypes.c_double * 3),
                ("f16_scale", ctypes.c_double), ("trt_magic", ctypes.c_double),
                ("block_size", ctypes.c_int32), ("nodes_per_thread", ctypes.c_int32),
                ("cg_shift", ctypes.c_int32),
                ("store_hint", ctypes.c_int32), ("swap_schedule", ctypes.c_int32),
                ("pair_z", ctypes.c_int32),
                ("stream", ctypes.c_void_p),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class lbm_info(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("storage_nodes", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
                ("index_bytes", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("natural", ctypes.c_int32), ("kernels_per_step", ctypes.c_int32),
                ("f16_scale", ctypes.c_double), ("reduce_blocks", ctypes.c_int32),
                ("tile_staged", ctypes.c_int32), ("pair_z", ctypes.c_int32)]


class lbm_batch_config(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("nodes_per_thread", ctypes.c_int32),
                ("capacity_slots", ctypes.c_int64), ("max_geometries", ctypes.c_int32),
                ("keep_idx", ctypes.c_int32), ("f16_scale", ctypes.c_double),
                ("tune_variant", ctypes.c_int32), ("round_mode", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p)]


class lbm_batch_info(ctypes.Structure):
    _fields_ = [("capacity_slots", ctypes.c_int64), ("free_slots", ctypes.c_int64),
                ("largest_free", ctypes.c_int64), ("active_nodes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("active_geometries", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("nodes_per_thread", ctypes.c_int32),
                ("work_chunks", ctypes.c_int32), ("variant", ctypes.c_int32), ("round_mode", ctypes.c_int32)]


# exported symbols and their signatures (every function declared in lbm.h)
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
SIGNATURES = {
    "lbm_config_default": (_I, [ctypes.POINTER(lbm_config)]),
    "lbm_create": (_I, [ctypes.POINTER(lbm_config), ctypes.POINTER(_P)]),
    "lbm_destroy": (_I, [_P]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_status_string": (ctypes.c_char_p, [_I]),
    "lbm_set_geometry": (_I, [_P, _P]),
    "lbm_set_geometry_spheres": (_I, [_P, _I64, _P, _I64, _I64]),
    "lbm_get_mask": (_I, [_P, _P]),
    "lbm_get_nodes": (_I, [_P, _P]),
    "lbm_get_idx": (_I, [_P, _P]),
    "lbm_get_info": (_I, [_P, ctypes.POINTER(lbm_info)]),
    "lbm_init": (_I, [_P, _P, _P, _I]),
    "lbm_set_pdfs": (_I, [_P, _P, _I]),
    "lbm_get_pdfs": (_I, [_P, _P, _I]),
    "lbm_step": (_I, [_P, _I]),
    "lbm_step_flux": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "lbm_flux": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "lbm_macroscopics": (_I, [_P, _P, _P, _I]),
    "lbm_sync": (_I, [_P]),
    "lbm_solve_permeability": (_I, [_P, ctypes.c_int32, ctypes.c_double, _I64, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int64)]),
    "lbm_batch_bytes_per_slot": (_I64, [ctypes.c_int32, ctypes.c_int32]),
    "lbm_batch_create": (_I, [ctypes.POINTER(lbm_batch_config), ctypes.POINTER(_P)]),
    "lbm_batch_destroy": (_I, [_P]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_batch_admit": (_I, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_double, _P,
                             ctypes.c_double, _I64, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_admit_spheres": (_I, [_P, _P, _P, _I64, _P, _I64, _I64, ctypes.c_double, _P, ctypes.c_double, _I64,
                                     ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_release": (_I, [_P, ctypes.c_int32]),
    "lbm_batch_round": (_I, [_P, ctypes.c_int32]),
    "lbm_batch_poll": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "lbm_batch_flux": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "lbm_batch_slot_info": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "lbm_batch_get_info": (_I, [_P, ctypes.POINTER(lbm_batch_info)]),
    "lbm_batch_get_pdfs": (_I, [_P, ctypes.c_int32, _P]),
    "lbm_batch_tune": (_I, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "lbm_flux_noalloc": (_I, [_P, ctypes.c_int32, ctypes.c_int32, _I64, _I64, ctypes.c_double,
                              ctypes.c_double, _P, _P]),
    "lbm_selftest_bounded_wait": (_I, [_I64, _P]),
}

_lib = None
_lock = threading.Lock()


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, msg))
        self.status = status


def _status_name(s):
    names = ["LBM_OK", "LBM_ERR_INVALID_ARG", "LBM_ERR_OOM", "LBM_ERR_CUDA", "LBM_ERR_STATE",
             "LBM_ERR_BOUNDS", "LBM_ERR_TIMEOUT", "LBM_ERR_NOT_CONVERGED", "LBM_ERR_UNSUPPORTED"]
    return names[s] if 0 <= s < len(names) else "status"


def load(path: str | None = None):
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("liblbm.so is not built (%s); run paper_1111_0922_gb300.build.build()" % p)
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(h, status):
    if status != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LBMError(status, msg.decode() if msg else "")


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):  # torch tensor on the device
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# C-named functions (argument marshalling only)

def lbm_config_default():
    cfg = lbm_config()
    _check(None, load().lbm_config_default(ctypes.byref(cfg)))
    return cfg


def lbm_create(cfg: lbm_config):
    h = ctypes.c_void_p()
    st = load().lbm_create(ctypes.byref(cfg), ctypes.byref(h))
    _check(None, st)
    return h


def lbm_destroy(h):
    _check(None, load().lbm_destroy(h))


def lbm_set_geometry(h, solid_mask=None):
    m = None if solid_mask is None else np.ascontiguousarray(solid_mask, dtype=np.uint8).reshape(-1)
    _check(h, load().lbm_set_geometry(h, _ptr(m)))


def lbm_set_geometry_spheres(h, centres, radius, unit):
    c = np.ascontiguousarray(np.asarray(centres, dtype=np.int64).reshape(-1, 3))
    _check(h, load().lbm_set_geometry_spheres(h, c.shape[0], _ptr(c), int(radius), int(unit)))


def lbm_get_info(h) -> lbm_info:
    info = lbm_info()
    _check(h, load().lbm_get_info(h, ctypes.byref(info)))
    return info


def lbm_get_mask(h, ncells):
    out = np.empty(ncells, np.uint8)
    _check(h, load().lbm_get_mask(h, _ptr(out)))
    return out


def lbm_get_nodes(h, nnodes):
    out = np.empty(nnodes, np.int32)
    _check(h, load().lbm_get_nodes(h, _ptr(out)))
    return out


def lbm_get_idx(h, nnodes):
    out = np.empty((18, nnodes), np.int32)
    _check(h, load().lbm_get_idx(h, _ptr(out)))
    return out


def lbm_init(h, rho=None, u=None, on_device=False):
    if not on_device:
        rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    _check(h, load().lbm_init(h, _ptr(rho), _ptr(u), int(bool(on_device))))


def lbm_set_pdfs(h, f, on_device=False):
    if not on_device:
        f = np.ascontiguousarray(f, dtype=np.float64)
    _check(h, load().lbm_set_pdfs(h, _ptr(f), int(bool(on_device))))


def lbm_get_pdfs(h, n=None, out=None, on_device=False):
    if out is None:
        out = np.empty((Q, n), np.float64)
    _check(h, load().lbm_get_pdfs(h, _ptr(out), int(bool(on_device))))
    return out


def lbm_step(h, n=1):
    _check(h, load().lbm_step(h, int(n)))


def lbm_step_flux(h, n=1):
    m = ctypes.c_double()
    j = ctypes.c_double()
    _check(h, load().lbm_step_flux(h, int(n), ctypes.byref(m), ctypes.byref(j)))
    return m.value, j.value


def lbm_flux(h):
    m = ctypes.c_double()
    j = ctypes.c_double()
    _check(h, load().lbm_flux(h, ctypes.byref(m), ctypes.byref(j)))
    return m.value, j.value


def lbm_macroscopics(h, n=None, rho=None, u=None, on_device=False, want_rho=True, want_u=True):
    if not on_device:
        rho = (np.empty(n, np.float64) if rho is None else rho) if want_rho else None
        u = (np.empty((n, 3), np.float64) if u is None else u) if want_u else None
    _check(h, load().lbm_macroscopics(h, _ptr(rho), _ptr(u), int(bool(on_device))))
    return rho, u


def lbm_sync(h):
    _check(h, load().lbm_sync(h))


def lbm_solve_permeability(h, check=100, tol=1e-6, max_steps=200000):
    """Run to a steady flux in the library (see include/lbm.h); returns
    (permeability, mass, flux, steps, converged)."""
    k, m, f, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    st = load().lbm_solve_permeability(h, int(check), float(tol), int(max_steps), ctypes.byref(k), ctypes.byref(m),
                                       ctypes.byref(f), ctypes.byref(n))
    if st not in (LBM_OK, LBM_ERR_NOT_CONVERGED):
        _check(h, st)
    return k.value, m.value, f.value, n.value, st == LBM_OK


def lbm_flux_noalloc(f_dev, precision, layout, n, npad, f16_scale, gx, out_dev, stream=None):
    """Mass and flux of a caller-owned natural PDF array into out_dev (2
    doubles on the device), for callers that cannot allocate device memory:
    the library allocates nothing for this call (its scratch is a fixed
    256 KiB array inside the library).  Calls that overlap on the GPU share
    that scratch and must be ordered by the caller; the first call on a
    device does a one-time set-up and should come before any stream capture."""
    st = load().lbm_flux_noalloc(_ptr(f_dev), int(precision), int(layout), int(n), int(npad),
                                 float(f16_scale), float(gx), _ptr(out_dev),
                                 ctypes.c_void_p(int(stream) if stream else 0))
    if st != LBM_OK:
        raise LBMError(st, "lbm_flux_noalloc rejected the call")


def lbm_selftest_bounded_wait(limit_ns, stream=None):
    """Run the bounded-wait self-test; returns the status (LBM_ERR_TIMEOUT is
    the expected result: the wait gave up after limit_ns)."""
    return int(load().lbm_selftest_bounded_wait(int(limit_ns), ctypes.c_void_p(int(stream) if stream else 0)))


# ---------------------------------------------------------------------------
# Convenience object over the same calls

class _TorchAllocator:
    """Device allocation through PyTorch's caching allocator (plumbing)."""

    def __init__(self, device, stream):
        import torch

        self.torch = torch
        self.device = device
        self.stream = stream

        def alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:  # noqa: BLE001 - report as a NULL allocation (LBM_ERR_OOM)
                return None

        def free(ptr, nbytes, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


class Lattice:
    """A D3Q19 lattice on one GPU: geometry, state and time stepping."""

    def __init__(self, dims, periodic=(1, 1, 1), variant="aa", addressing="direct",
                 layout="soa", precision="f32", omega=1.0, force=(0.0, 0.0, 0.0),
                 f16_scale=0.0, block_size=0, nodes_per_thread=0, cg_shift=0,
                 trt_magic=0.0, store_hint=0, swap_schedule=0, pair_z=0, stream=None, use_torch_allocator=True):
        self.cfg = lbm_config_default()
        c = self.cfg
        c.nx, c.ny, c.nz = (int(d) for d in dims)
        for a in range(3):
            c.periodic[a] = int(periodic[a])
            c.force[a] = float(force[a])
        c.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        c.addressing = {"direct": LBM_DIRECT, "indirect": LBM_INDIRECT}[addressing] \
            if isinstance(addressing, str) else int(addressing)
        c.layout = {"soa": LBM_SOA, "aos": LBM_AOS}[layout] if isinstance(layout, str) else int(layout)
        c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        c.omega = float(omega)
        c.f16_scale = float(f16_scale)
        c.trt_magic = float(trt_magic)
        c.block_size = int(block_size)
        c.nodes_per_thread = int(nodes_per_thread)
        c.cg_shift = int(cg_shift)
        c.store_hint = int(store_hint)
        c.swap_schedule = int(swap_schedule)
        c.pair_z = int(pair_z)
        self._alloc = None
        if stream is None or use_torch_allocator:
            import torch

            dev = torch.cuda.current_device()
            if stream is None:
                stream = torch.cuda.current_stream(dev).cuda_stream
            if use_torch_allocator:
                self._alloc = _TorchAllocator(dev, stream)
                c.dev_alloc = self._alloc.alloc
                c.dev_free = self._alloc.free
        c.stream = ctypes.c_void_p(int(stream) if stream else 0)
        self.dims = tuple(int(d) for d in dims)
        self.h = lbm_create(c)

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # geometry
    def set_geometry(self, solid=None):
        lbm_set_geometry(self.h, solid)

    def set_geometry_spheres(self, centres, radius, unit):
        lbm_set_geometry_spheres(self.h, centres, radius, unit)

    @property
    def info(self) -> lbm_info:
        return lbm_get_info(self.h)

    @property
    def n(self) -> int:
        """Length of natural arrays: cells (direct) or fluid nodes (indirect)."""
        i = self.info
        return int(i.cells if self.cfg.addressing == LBM_DIRECT else i.nodes)

    def mask(self):
        return lbm_get_mask(self.h, int(np.prod(self.dims)))

    def nodes(self):
        return lbm_get_nodes(self.h, self.info.nodes)

    def idx(self):
        return lbm_get_idx(self.h, self.info.nodes)

    # state
    def init(self, rho=None, u=None, on_device=False):
        lbm_init(self.h, rho, u, on_device)

    def set_pdfs(self, f, on_device=False):
        lbm_set_pdfs(self.h, f, on_device)

    def pdfs(self):
        return lbm_get_pdfs(self.h, self.n)

    def step(self, n=1):
        lbm_step(self.h, n)

    def step_flux(self, n=1):
        return lbm_step_flux(self.h, n)

    def flux(self):
        return lbm_flux(self.h)

    def macroscopics(self):
        return lbm_macroscopics(self.h, self.n)

    def sync(self):
        lbm_sync(self.h)

    def solve_permeability(self, check=100, tol=1e-6, max_steps=200000):
        return lbm_solve_permeability(self.h, check, tol, max_steps)


# ---------------------------------------------------------------------------
# Batches (continuous batching of many geometries)

def _bcheck(b, status):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error(b)
        raise LBMError(status, msg.decode() if msg else "")


def lbm_batch_bytes_per_slot(variant, precision):
    return int(load().lbm_batch_bytes_per_slot(int(variant), int(precision)))


def lbm_batch_create(cfg: lbm_batch_config):
    b = ctypes.c_void_p()
    _bcheck(None, load().lbm_batch_create(ctypes.byref(cfg), ctypes.byref(b)))
    return b


def lbm_batch_destroy(b):
    _bcheck(None, load().lbm_batch_destroy(b))


def lbm_batch_admit(b, mask, dims, periodic, omega, force, tol=1e-6, max_steps=0):
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
    if m.size != int(np.prod(dims)):
        raise ValueError("mask has %d cells, box %s" % (m.size, tuple(dims)))
    p = (ctypes.c_int32 * 3)(*[int(v) for v in periodic])
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    slot = ctypes.c_int32()
    _bcheck(b, load().lbm_batch_admit(b, _ptr(m), int(dims[0]), int(dims[1]), int(dims[2]), p, float(omega), f,
                                      float(tol), int(max_steps), ctypes.byref(slot)))
    return slot.value


def lbm_batch_admit_spheres(b, dims, periodic, centres, radius, unit, omega, force, tol=1e-6, max_steps=0):
    d = (ctypes.c_int32 * 3)(*[int(v) for v in dims])
    p = (ctypes.c_int32 * 3)(*[int(v) for v in periodic])
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    c = np.ascontiguousarray(np.asarray(centres, dtype=np.int64).reshape(-1, 3))
    slot = ctypes.c_int32()
    _bcheck(b, load().lbm_batch_admit_spheres(b, d, p, c.shape[0], _ptr(c), int(radius), int(unit),
                                              float(omega), f, float(tol), int(max_steps), ctypes.byref(slot)))
    return slot.value


def lbm_batch_release(b, slot):
    _bcheck(b, load().lbm_batch_release(b, int(slot)))


def lbm_batch_round(b, k):
    _bcheck(b, load().lbm_batch_round(b, int(k)))


def lbm_batch_poll(b, slot):
    """(done, permeability, steps): done 0 running, 1 steady, 2 step cap."""
    d, k, n = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int64()
    _bcheck(b, load().lbm_batch_poll(b, int(slot), ctypes.byref(d), ctypes.byref(k), ctypes.byref(n)))
    return d.value, k.value, n.value


def lbm_batch_flux(b, slot):
    """(mass, flux, steps) of the state the last round started from."""
    m, f, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _bcheck(b, load().lbm_batch_flux(b, int(slot), ctypes.byref(m), ctypes.byref(f), ctypes.byref(s)))
    return m.value, f.value, s.value


def lbm_batch_slot_info(b, slot):
    n, c, s = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _bcheck(b, load().lbm_batch_slot_info(b, int(slot), ctypes.byref(n), ctypes.byref(c), ctypes.byref(s)))
    return n.value, c.value, s.value


def lbm_batch_get_info(b) -> lbm_batch_info:
    info = lbm_batch_info()
    _bcheck(b, load().lbm_batch_get_info(b, ctypes.byref(info)))
    return info


def lbm_batch_get_pdfs(b, slot, nodes):
    out = np.empty((Q, nodes), np.float64)
    _bcheck(b, load().lbm_batch_get_pdfs(b, int(slot), _ptr(out)))
    return out


def lbm_batch_tune(b, rounds=2, k=10):
    """(variant, block size, nodes per thread, round mode, MFLUP/s) of the
    fastest candidate; every geometry restarts from rest."""
    v, bs, npt, mode, mf = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _bcheck(b, load().lbm_batch_tune(b, int(rounds), int(k), ctypes.byref(v), ctypes.byref(bs), ctypes.byref(npt),
                                     ctypes.byref(mode), ctypes.byref(mf)))
    return v.value, bs.value, npt.value, mode.value, mf.value


class Batch:
    """Many sphere-pack geometries on one GPU, advanced together in rounds."""

    def __init__(self, capacity_slots, variant="aa", precision="f32", max_geometries=1024,
                 f16_scale=0.0, block_size=0, nodes_per_thread=0, keep_idx=0, tune_variant=0, round_mode=0,
                 stream=None, use_torch_allocator=True):
        cfg = lbm_batch_config()
        cfg.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.block_size = int(block_size)
        cfg.nodes_per_thread = int(nodes_per_thread)
        cfg.capacity_slots = int(capacity_slots)
        cfg.max_geometries = int(max_geometries)
        cfg.f16_scale = float(f16_scale)
        cfg.keep_idx = int(keep_idx)
        cfg.tune_variant = int(tune_variant)
        cfg.round_mode = int(round_mode)
        self._alloc = None
        if stream is None or use_torch_allocator:
            import torch

            dev = torch.cuda.current_device()
            if stream is None:
                stream = torch.cuda.current_stream(dev).cuda_stream
            if use_torch_allocator:
                self._alloc = _TorchAllocator(dev, stream)
                cfg.dev_alloc = self._alloc.alloc
                cfg.dev_free = self._alloc.free
        cfg.stream = ctypes.c_void_p(int(stream) if stream else 0)
        self.cfg = cfg
        self.b = lbm_batch_create(cfg)

    def close(self):
        if self.b:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def admit(self, pack, omega, force, tol=1e-6, max_steps=0):
        """Admit a sphere pack (inputs.SpherePack)."""
        return lbm_batch_admit_spheres(self.b, pack.dims, pack.periodic, pack.centres, pack.radius,
                                       pack.unit, omega, force, tol, max_steps)

    def admit_mask(self, mask, dims, periodic, omega, force, tol=1e-6, max_steps=0):
        """Admit a geometry given as a solid mask (x fastest, nonzero = solid)."""
        return lbm_batch_admit(self.b, mask, dims, periodic, omega, force, tol, max_steps)

    def release(self, slot):
        lbm_batch_release(self.b, slot)

    def round(self, k):
        lbm_batch_round(self.b, k)

    def poll(self, slot):
        """(done, permeability, steps) after the last round."""
        return lbm_batch_poll(self.b, slot)

    def flux(self, slot):
        """(mass, flux, steps) of the state the last round started from."""
        return lbm_batch_flux(self.b, slot)

    def slot_info(self, slot):
        return lbm_batch_slot_info(self.b, slot)

    @property
    def info(self):
        return lbm_batch_get_info(self.b)

    def pdfs(self, slot):
        return lbm_batch_get_pdfs(self.b, slot, self.slot_info(slot)[0])

    def tune(self, rounds=2, k=10):
        """(variant, block size, nodes per thread, round mode, MFLUP/s)."""
        return lbm_batch_tune(self.b, rounds, k)
