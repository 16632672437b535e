"""Benchmark of the D3Q19 step on GB300.

Headline workload: a periodic 256^3 full grid (direct addressing), density
rho = 1 + 1e-3 U[-1, 1) (SplitMix64 seed 2), zero velocity, omega = 1.7,
AA pattern, SoA, in the paper's arithmetic: FP64 storage of f - w and FP64
collision.  One bench step is one time step of the whole lattice (one kernel
launch for the AA pattern).  The state (2.55 GB) is larger than L2 (129 MB),
so no flush is needed between steps.

Printed (rank 0, one JSON line): MFLUP/s of the headline run; the roofline of
its kernel, bound by the FP64 pipe (peak = SMs x FP64 instructions per SM
clock x the SM clock sampled during the timed region; instructions per update
from the committed ncu capture); the same workload with FP32 and FP16 storage
(each with its HBM roofline); an end-to-end figure through the C ABI with
host buffers; the FP64 CPU oracle timed on the host cores; SM clocks sampled
during the timed region; and a sweep over every propagation scheme x
FP64/FP32/FP16 x SoA/AoS with each one's fraction of its own roofline.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl gb300|reference]
N > 1 runs under torchrun as N independent replicas (weak scaling, no
collective on the data path); value = total node updates / max rank time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1111_0922_gb300 import inputs, model  # noqa: E402

METRIC = "D3Q19 MFLUP/s & % of HBM roofline per propagation variant; solves/s, p99"
DIMS = (256, 256, 256)
OMEGA = 1.7
SEED = 2
WORKLOAD = "periodic 256^3 full grid, rho = 1 + 1e-3 U[-1,1) (seed 2), u = 0, omega = 1.7, BGK"
FALLBACK_HBM = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM)), "measured"
    return FALLBACK_HBM, "fallback"


STEP_SOURCES = ("lbm_core.cuh", "lbm_dispatch.cuh", "lbm_steps.cuh")


def kernel_source_hash(precision="f32"):
    """Hash of the files that define the step kernels of one precision
    (k_aa_even/odd and the other one-lattice schemes): a profile's counters
    stay valid while this does not change."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1111_0922_gb300", "csrc")
    for name in STEP_SOURCES + ("lbm_steps_%s.cu" % precision,):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_records(directory=None):
    """Machine-readable lines of the committed ncu summaries (profiles/*.md):
      dram_bytes_per_launch <key> <bytes> source_hash <hash>
      fp64_inst_per_flup <collision kind> <count> source_hash <hash>
      fp64_inst_per_clk_sm <peak>
    returned as lists of fields."""
    recs = []
    for path in sorted(glob.glob(os.path.join(directory or os.path.join(ROOT, "profiles"), "*.md"))):
        with open(path) as f:
            for line in f:
                parts = line.split()
                if parts and parts[0] in ("dram_bytes_per_launch", "fp64_inst_per_flup", "fp64_inst_per_clk_sm"):
                    recs.append(parts)
    return recs


def profiled_traffic(kernel_key, precision, directory=None):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or
    None when the kernel sources changed since the capture."""
    want = kernel_source_hash(precision)
    for p in profile_records(directory):
        if len(p) == 5 and p[0] == "dram_bytes_per_launch" and p[1] == kernel_key and p[3] == "source_hash" \
                and p[4] == want:
            return float(p[2])
    return None


def profiled_fp64(directory=None):
    """(FP64 thread instructions per SM clock, {collision kind: FP64 thread
    instructions per update}) from the committed ncu capture; a count whose
    kernel sources changed since the capture is left out."""
    per_clk = None
    per_flup = {}
    for p in profile_records(directory):
        if p[0] == "fp64_inst_per_clk_sm" and len(p) == 2:
            per_clk = float(p[1])
        elif p[0] == "fp64_inst_per_flup" and len(p) == 5 and p[4] == kernel_source_hash("f64"):
            per_flup[p[1]] = float(p[2])
    return per_clk, per_flup


def fp64_pipe(torch, dev, clocks):
    """The FP64-pipe roof of this GPU from measured inputs (model.Fp64Pipe),
    or None when the capture is missing or stale."""
    per_clk, per_flup = profiled_fp64()
    if per_clk is None or set(per_flup) != set(model.COLLISIONS):
        return None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if clocks and clocks.get("sm_mhz"):
        ghz = clocks["sm_mhz"] / 1e3
    else:
        return None
    return model.Fp64Pipe(sms, ghz, per_clk, per_flup)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        import tempfile

        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = np.array([float(r[1]) for r in rows])
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        load = sm[sm > 0.5 * mx] if np.any(sm > 0.5 * mx) else sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": int(sm.size), "power_w_max": max(float(r[3]) for r in rows
                                                             if r[3].replace(".", "").isdigit())}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:  # noqa: BLE001
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


# ---------------------------------------------------------------------------
def max_over_ranks(torch, value: float, device) -> float:
    """Largest value over all ranks (the job time of N replicas)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(nodes_per_rank: int, steps: int, world: int, t_max: float) -> float:
    """Whole-job MFLUP/s of `world` replicas that each updated nodes_per_rank
    nodes `steps` times, the slowest taking t_max seconds."""
    return world * nodes_per_rank * steps / t_max / 1e6


def make_lattice(lbm, variant, precision, layout, addressing="direct", dims=DIMS, omega=OMEGA,
                 force=(0.0, 0.0, 0.0), **kw):
    return lbm.Lattice(dims, (1, 1, 1), variant=variant, addressing=addressing, layout=layout,
                       precision=precision, omega=omega, force=force, **kw)


def timed_steps(torch, lat, steps, per_launch=True):
    """Run `steps` steps between CUDA events on the lattice's stream.
    Returns (total seconds, mean seconds per launch-step)."""
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1 if per_launch else 2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for t in range(steps):
        lat.step(1)
        if per_launch:
            ev[t + 1].record(stream)
    if not per_launch:
        ev[1].record(stream)
    torch.cuda.synchronize()
    total = ev[0].elapsed_time(ev[-1]) / 1e3
    if per_launch:
        durs = [ev[t].elapsed_time(ev[t + 1]) / 1e3 for t in range(steps)]
        return total, float(np.mean(durs))
    return total, total / steps


def run_headline(torch, lbm, args, rank, world, precision="f64", sample_clocks=True):
    """The headline workload with the given storage precision (AA pattern,
    SoA, direct): W warm-up steps, then K steps between CUDA events on the
    launching stream, a barrier and a synchronize on both sides."""
    dev = torch.cuda.current_device()
    n = int(np.prod(DIMS))
    rho_host = inputs.density_noise(DIMS, seed=SEED)
    rho_dev = torch.from_numpy(rho_host).to(f"cuda:{dev}")
    lat = make_lattice(lbm, "aa", precision, "soa")
    lat.set_geometry(None)
    lat.init(rho_dev, on_device=True)
    lat.step(args.warmup if args.warmup % 2 == 0 else args.warmup + 1)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_smi_id(torch, dev)) if sample_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total, per_launch = timed_steps(torch, lat, args.steps)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    info = lat.info
    t_max = max_over_ranks(torch, total, f"cuda:{dev}")
    kernels = args.steps * info.kernels_per_step
    lat.close()
    del rho_dev
    torch.cuda.empty_cache()
    return {"total_s": t_max, "per_launch_s": per_launch, "nodes": n, "clocks": clocks,
            "kernels": kernels, "rho_host": rho_host, "paired": int(info.pair_z), "precision": precision}


def hbm_roofline(head, hbm, peak_kind, steps):
    """HBM roofline of an FP32 / FP16 headline run (its AA kernels)."""
    prec = head["precision"]
    bytes_launch = head["nodes"] * model.kernel_bytes_per_flup("aa", False, prec)
    achieved = bytes_launch / head["per_launch_s"] / 1e9
    key = "aa_%s_soa_direct_256" % prec
    codec = {"f32": "CodecF32", "f16s": "CodecF16S"}[prec]
    return {"mflups": round(head["nodes"] * steps / head["total_s"] / 1e6, 1),
            "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "peak_kind": peak_kind, "bytes_per_launch": int(bytes_launch),
            "traffic": profiled_traffic(key, prec),
            "kernel": ("k_aa_even_zp/k_aa_odd_zp<%s>" % codec if head["paired"]
                       else "k_aa_even/k_aa_odd<%s,SoA,direct>" % codec)}


def fp64_roofline(head, pipe, hbm, peak_kind):
    """FP64-pipe roofline of the FP64 headline run: achieved = FP64 thread
    instructions per launch (captured count per update x nodes) / mean
    CUDA-event launch duration; peak = SMs x FP64 instructions per SM clock
    x the SM clock sampled during the timed region."""
    n = head["nodes"]
    bytes_launch = n * model.kernel_bytes_per_flup("aa", False, "f64")
    hbm_achieved = bytes_launch / head["per_launch_s"] / 1e9
    out = {"bound": "alu", "unit": "G FP64 inst/s", "kernel": "k_aa_even/k_aa_odd<CodecF64,SoA,direct>",
           "bytes_per_launch": int(bytes_launch), "traffic": profiled_traffic("aa_f64_soa_direct_256", "f64"),
           "hbm": {"achieved": round(hbm_achieved, 1), "peak": hbm, "unit": "GB/s",
                   "frac": round(hbm_achieved / hbm, 4), "peak_kind": peak_kind}}
    if pipe is None:
        out.update({"achieved": None, "peak": None, "frac": None,
                    "peak_kind": "unavailable: FP64 capture missing or stale, or no clock samples"})
        return out
    inst = pipe.inst_per_flup["bgk"] * n
    achieved = inst / head["per_launch_s"] / 1e9
    peak = pipe.inst_rate() / 1e9
    out.update({"achieved": round(achieved, 1), "peak": round(peak, 1), "frac": round(achieved / peak, 4),
                "peak_kind": "measured (SM count: device attribute; SM clock: median sampled in the timed "
                             "region; FP64 instructions per clock and per update: ncu, profiles/)",
                "inst_per_launch": int(inst), "fp64_pipe": pipe.as_dict(),
                "roof_mflups": round(pipe.roof_mflups(), 1)})
    return out


def run_e2e(torch, lbm, args, rho_host, precision="f64"):
    """The same solve through the public API with host buffers: the initial
    density goes up from pinned host memory, the mass/flux come back every 100
    steps through the fused reduction, and the final density field comes back
    to pinned host memory, all inside the timed region."""
    n = rho_host.size
    pin_rho = torch.from_numpy(rho_host).pin_memory()
    pin_out = torch.empty(n, dtype=torch.float64).pin_memory()
    lat = make_lattice(lbm, "aa", precision, "soa")
    lat.set_geometry(None)
    check = 100
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.init(pin_rho.numpy())
    done = 0
    reads = 0
    while done < args.steps:
        k = min(check, args.steps - done)
        if k % 2 == 1 and k > 1:
            k -= 1
        lat.step_flux(k)
        reads += 1
        done += k
    if done % 2 == 1:  # AA pattern reads out after an even count
        lat.step(1)
        done += 1
    lbm.lbm_macroscopics(lat.h, n, rho=pin_out.numpy(), want_u=False)
    t1 = time.perf_counter()
    lat.close()
    secs = t1 - t0
    return {"value": n * done / secs / 1e6, "unit": "MFLUP/s",
            "h2d_bytes_per_step": int(8 * n / done), "d2h_bytes_per_step": int((8 * n + 16 * reads) / done),
            "seconds": secs, "precision": precision}


def run_cpu_baseline(target_s=10.0):
    """The FP64 oracle as it stands (push definition, OpenMP over cells) on
    the host cores: 256^3 periodic from the same initial state, whole steps
    until about target_s seconds have passed."""
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    rho = inputs.density_noise(DIMS, seed=SEED)
    _, w = oracle.lattice()
    f = np.ascontiguousarray(w[:, None] * rho[None, :])
    n = rho.size
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < target_s:
        f = oracle.push_full(DIMS, (1, 1, 1), None, f, OMEGA, nthreads=threads)
        steps += 1
    secs = time.perf_counter() - t0
    return {"value": n * steps / secs / 1e6, "unit": "MFLUP/s", "cores": threads, "kind": "oracle",
            "sample": "%d full steps of the 256^3 periodic box (%.1f s)" % (steps, secs)}


def run_sweep(torch, lbm, args, hbm, pipe):
    """Every scheme x FP64/FP32 x SoA/AoS, and FP16 storage in SoA, on the
    headline workload."""
    out = {}
    n = int(np.prod(DIMS))
    rho_dev = torch.from_numpy(inputs.density_noise(DIMS, seed=SEED)).cuda()
    for variant in model.VARIANTS:
        for precision in ("f64", "f32", "f16s"):
            for layout in (("soa",) if precision == "f16s" else ("soa", "aos")):
                key = "%s/%s/%s" % (variant, precision, layout)
                try:
                    lat = make_lattice(lbm, variant, precision, layout)
                    lat.set_geometry(None)
                    lat.init(rho_dev, on_device=True)
                    lat.step(4)
                    steps = args.sweep_steps
                    total, per = timed_steps(torch, lat, steps, per_launch=False)
                    mflups = n * steps / total / 1e6
                    bound, roof = model.bound_roof(variant, False, precision, hbm, pipe)
                    out[key] = {"mflups": round(mflups, 1), "bound": bound, "roof_mflups": round(roof, 1),
                                "frac": round(mflups / roof, 4),
                                "bytes_per_flup": model.gpu_bytes(variant, False, precision),
                                "kernels_per_step": lat.info.kernels_per_step}
                    if precision == "f16s":
                        out[key]["pair_z"] = int(lat.info.pair_z)
                    lat.close()
                except lbm.LBMError as e:
                    out[key] = {"unsupported": str(e).split(": ", 1)[-1][:120]}
                torch.cuda.empty_cache()
                log("sweep", key, out[key])
    del rho_dev
    torch.cuda.empty_cache()
    return out


def run_sparse(torch, lbm, args, hbm):
    """512^3 periodic sphere pack (r = 8, porosity 0.6, seed 3; g = 1e-6 x,
    omega 1): AA pattern and esoteric twist on the IDX node list, FP32 and FP16
    storage, SoA."""
    dims = (512, 512, 512)
    pack = inputs.sphere_pack(dims, 0.6, radius=8.0, seed=SEED + 1)
    out = {"workload": "periodic 512^3 sphere pack, r = 8, porosity 0.6 (seed 3), "
                       "%d spheres, g = 1e-6 x, omega 1.0, from rest" % pack.nspheres}
    for variant in ("aa", "et"):
        for precision in ("f32", "f16s"):
            key = "%s/%s/indirect" % (variant, precision)
            lat = lbm.Lattice(dims, (1, 1, 1), variant=variant, addressing="indirect", precision=precision,
                              omega=1.0, force=(1e-6, 0.0, 0.0))
            t0 = time.perf_counter()
            lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
            lat.init()
            torch.cuda.synchronize()
            t_geo = time.perf_counter() - t0
            lat.step(4)
            total, _ = timed_steps(torch, lat, args.sparse_steps, per_launch=False)
            info = lat.info
            n = int(info.nodes)
            mflups = n * args.sparse_steps / total / 1e6
            roof = model.roof_mflups(variant, True, precision, hbm)
            out[key] = {"mflups": round(mflups, 1), "roof_mflups": round(roof, 1), "frac": round(mflups / roof, 4),
                        "bytes_per_flup": model.gpu_bytes(variant, True, precision), "fluid_nodes": n,
                        "porosity": round(n / info.cells, 4), "ghost_slots": int(info.storage_nodes - n),
                        "setup_s": round(t_geo, 2)}
            lat.close()
            torch.cuda.empty_cache()
            log("sparse", key, out[key])
    return out


def run_sparse_solve(torch, lbm, args):
    """The 512^3 pack run to a steady flux (relative change < 1e-6 between
    rounds of 100 steps), AA pattern on the node list, FP32 and FP16 storage."""
    from paper_1111_0922_gb300 import permeability

    dims = (512, 512, 512)
    pack = inputs.sphere_pack(dims, 0.6, radius=8.0, seed=SEED + 1)
    out = {}
    for precision in ("f32", "f16s"):
        lat = lbm.Lattice(dims, (1, 1, 1), variant="aa", addressing="indirect", precision=precision, omega=1.0,
                          force=(1e-6, 0.0, 0.0))
        lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
        lat.init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = permeability.solve(lat, 100, 1e-6, max_steps=args.solve_max_steps)
        secs = time.perf_counter() - t0
        n = int(lat.info.nodes)
        out[precision] = {"k": res.k, "steps": res.steps, "converged": res.converged, "seconds": round(secs, 2),
                          "mflups": round(n * res.steps / secs / 1e6, 1), "f16_scale": lat.info.f16_scale}
        lat.close()
        torch.cuda.empty_cache()
        log("solve", precision, out[precision])
    if out["f32"]["converged"] and out["f16s"]["converged"]:
        out["k_rel_diff_f16s_vs_f32"] = abs(out["f16s"]["k"] - out["f32"]["k"]) / out["f32"]["k"]
    return out


def run_paper_shapes(torch, lbm, args, hbm, pipe):
    """The paper's benchmark geometries (Sec. 10): the 500x100x100 empty
    channel and a packed bed of spheres with about 2.1 M fluid cells, flow
    along x, walls on y/z; node-list addressing, SoA, TRT (magic 3/16) as the
    paper's solver, FP64 and FP32."""
    out = {}
    shapes = {"channel": (inputs.paper_channel(), None), "bed": (None, inputs.paper_packed_bed())}
    for name, (chan, pack) in shapes.items():
        for variant in ("os_push", "os_pull", "aa", "et"):
            for precision in ("f64", "f32"):
                dims, per = chan if chan else (pack.dims, pack.periodic)
                lat = lbm.Lattice(dims, per, variant=variant, addressing="indirect", precision=precision,
                                  omega=1.0, force=(1e-6, 0.0, 0.0), trt_magic=3.0 / 16.0)
                if pack is None:
                    lat.set_geometry(None)
                else:
                    lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
                lat.init()
                lat.step(4)
                total, _ = timed_steps(torch, lat, args.shape_steps, per_launch=False)
                n = int(lat.info.nodes)
                mflups = n * args.shape_steps / total / 1e6
                roof = model.roof_mflups(variant, True, precision, hbm)
                bound, broof = model.bound_roof(variant, True, precision, hbm, pipe, force=True, trt=True)
                out["%s/%s/%s" % (name, variant, precision)] = {
                    "fluid_nodes": n, "mflups": round(mflups, 1), "frac_of_hbm_roof": round(mflups / roof, 4),
                    "bound": bound, "frac": round(mflups / broof, 4)}
                lat.close()
                torch.cuda.empty_cache()
    log("paper_shapes", out)
    return out


def run_batch(torch, lbm, args):
    """64 sphere packs, cube sides U{32..192}, porosity U[0.3, 0.8), r = 8
    (seed 4); FP32 on concatenated node lists; the autotuner picks the
    variant (AA pattern or esoteric twist), block size, nodes per thread and
    round mode (per-step launches or one persistent launch); every geometry
    then advances in rounds of 100 steps until the library reports its flux
    steady (relative change below 1e-6 between rounds), then retires."""
    items = inputs.batch_packs(args.batch_count, seed=4)
    cap = sum(int(it.side ** 3) for it in items) + 4096 * (len(items) + 1)  # nodes + ghosts <= cells
    b = lbm.Batch(cap, variant="aa", precision="f32", max_geometries=len(items) + 1, tune_variant=1)
    g = (1e-6, 0.0, 0.0)
    t0 = time.perf_counter()
    slots = {b.admit(it.pack, 1.0, g, 1e-6, args.solve_max_steps): i for i, it in enumerate(items)}
    torch.cuda.synchronize()
    t_admit = time.perf_counter() - t0
    nodes_total = b.info.active_nodes
    t0 = time.perf_counter()
    variant, bs, npt, mode, tuned = b.tune(rounds=1, k=10)  # every geometry restarts from rest
    t_tune = time.perf_counter() - t0
    done = {}
    updates = 0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    while slots and time.perf_counter() - t1 < args.batch_seconds:
        active_nodes = b.info.active_nodes
        b.round(100)
        updates += 100 * active_nodes
        for slot in list(slots):
            state, k, steps = b.poll(slot)
            if state:
                done[slots[slot]] = (k, steps, state == 1)
                b.release(slot)
                del slots[slot]
    secs = time.perf_counter() - t1
    b.close()
    steps = [v[1] for v in done.values()]
    return {"workload": "64 sphere packs, side U{32..192}, porosity U[0.3,0.8), r = 8 (seed 4), FP32, "
                        "rounds of 100 steps, retire at relative flux change < 1e-6",
            "geometries": len(items), "fluid_nodes": int(nodes_total), "admit_s": round(t_admit, 2),
            "tuned": {"variant": "aa" if variant == lbm.LBM_AA else "et", "block_size": bs, "nodes_per_thread": npt,
                      "round_mode": "persistent" if mode == 1 else "per-step launches",
                      "mflups": round(tuned, 1), "tune_s": round(t_tune, 2)},
            "converged": sum(1 for v in done.values() if v[2]), "unfinished": len(items) - len(done),
            "solve_wall_s": round(secs, 2), "aggregate_mflups": round(updates / secs / 1e6, 1),
            "steps_to_converge": {"min": min(steps) if steps else None, "median": float(np.median(steps)) if steps else None,
                                  "max": max(steps) if steps else None},
            "k_range": [min(v[0] for v in done.values()), max(v[0] for v in done.values())] if done else None}


def run_serving(torch, lbm, args):
    """Poisson arrivals (20 requests/s, seed 5) of sphere packs with sides
    U{64..384} and porosity U[0.3, 0.8), r = 8, served by continuous batching
    with FP16-stored PDFs (FP32 collision, FP64 flux sums) within a 150 GB HBM
    budget.  Then a like-for-like comparison on a matched subset of the same
    trace (evenly spaced request ids, with their arrival times): served by
    the FP16 batch alone, and by the FP64 single-solve path one request at a
    time (each solve starts when the request has arrived and the previous
    solve is done).  Both report solves/s and latency over the same
    requests, and the permeability error of FP16 against FP64."""
    from paper_1111_0922_gb300 import permeability, serving

    budget = 150e9
    per_slot = lbm.lbm_batch_bytes_per_slot(lbm.LBM_AA, lbm.LBM_F16S)
    # below 2^30 slots (118 GB of the budget; the whole trace needs about
    # 0.6e9) the AA pattern's IDX holds the bounce-back slots, no branch per link
    cap = min(int(budget / per_slot), (1 << 30) - 8192)
    reqs = serving.poisson_requests(args.serve_requests, 20.0, seed=5)
    offered = sum(int(r.pack.dims[0] ** 3 * r.pack.porosity_target) for r in reqs) / (reqs[-1].arrival or 1.0)

    def fp16_serve(trace):
        # launch shape chosen by lbm_batch_tune on the 64-pack FP16 batch:
        # AA pattern, 512 threads x 4 nodes, per-step launches
        eng = serving.BatchEngine(cap, variant="aa", precision="f16s", f16_scale=2.0 ** 26,
                                  max_geometries=len(trace) + 1, block_size=512, nodes_per_thread=4)
        st = serving.serve(trace, eng, serving.RealClock(), k_round=100, tol=1e-6, max_steps=args.serve_max_steps)
        eng.close()
        torch.cuda.empty_cache()
        return st

    st = fp16_serve(reqs)
    summ = st.summary()
    # matched subset: every (n / m)-th request, with its arrival time
    m = max(1, min(args.serve_fp64, len(reqs)))
    subset = [reqs[i * len(reqs) // m] for i in range(m)]
    t0 = subset[0].arrival
    sub_trace = [serving.Request(r.rid, r.arrival - t0, r.pack, r.omega, r.force) for r in subset]
    sub16 = fp16_serve(sub_trace)
    by16 = {x.rid: x for x in sub16.results}
    # FP64, one solve at a time in arrival order
    clock = 0.0
    base = []
    for r in sub_trace:
        start = max(clock, r.arrival)
        lat = lbm.Lattice(r.pack.dims, r.pack.periodic, variant="aa", addressing="indirect", precision="f64",
                          omega=r.omega, force=r.force)
        t1 = time.perf_counter()
        lat.set_geometry_spheres(r.pack.centres, r.pack.radius, r.pack.unit)
        lat.init()
        res = permeability.solve(lat, 100, 1e-6, max_steps=args.serve_max_steps)
        service = time.perf_counter() - t1
        lat.close()
        torch.cuda.empty_cache()
        clock = start + service
        base.append((r.rid, res.k, service, res.steps, res.converged, clock - r.arrival, clock))
    lat64 = np.array([b[5] for b in base])
    k_err = {rid: abs(by16[rid].k - k) / k for rid, k, _, _, _, _, _ in base if by16[rid].converged}
    s16 = sub16.summary()
    return {"workload": "Poisson 20/s (seed 5), %d requests, side U{64..384}, porosity U[0.3,0.8), r = 8, "
                        "AA pattern, FP16 storage (S = 2^26), 150 GB budget" % len(reqs),
            "offered_node_rate_per_s": round(offered, 1), "capacity_slots": cap,
            **{k: (round(v, 4) if isinstance(v, float) else v) for k, v in summ.items()},
            "matched_subset": {
                "request_ids": [r.rid for r in subset],
                "fluid_nodes": [by16[r.rid].nodes for r in subset],
                "fp16_batched": {"solves_per_s": round(s16["solves_per_s"], 4),
                                 "p50_latency_s": round(s16["p50_latency_s"], 3),
                                 "p99_latency_s": round(s16["p99_latency_s"], 3),
                                 "steps": [by16[r.rid].steps for r in subset]},
                "fp64_one_at_a_time": {"solves_per_s": round(len(base) / (base[-1][6] - sub_trace[0].arrival), 4),
                                       "p50_latency_s": round(float(np.percentile(lat64, 50)), 3),
                                       "p99_latency_s": round(float(np.percentile(lat64, 99)), 3),
                                       "service_s": [round(b[2], 3) for b in base], "steps": [b[3] for b in base],
                                       "converged": all(b[4] for b in base)},
                "k_rel_err_fp16_vs_fp64": {str(r): float("%.3g" % e) for r, e in k_err.items()},
                "k_rel_err_max": max(k_err.values()) if k_err else None}}


def main_gb300(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1111_0922_gb300 import build, lbm

    build.build()
    lbm.load()
    hbm, peak_kind = measured_peaks()
    dev = torch.cuda.current_device()
    head = run_headline(torch, lbm, args, rank, world, "f64")
    n = head["nodes"]
    value = replica_value(n, args.steps, world, head["total_s"])
    pipe = fp64_pipe(torch, dev, head["clocks"])
    roof = fp64_roofline(head, pipe, hbm, peak_kind)
    by_prec = {}
    if not args.no_side:
        for prec in ("f32", "f16s"):
            side = run_headline(torch, lbm, args, rank, world, prec, sample_clocks=False)
            by_prec[prec] = hbm_roofline(side, hbm, peak_kind, args.steps)
            by_prec[prec]["gpu_launches"] = side["kernels"]
    roof["by_precision"] = by_prec
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": "MFLUP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(head["total_s"] / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "variant": "aa", "precision": "f64 (f - w stored, FP64 collision)",
                   "layout": "soa", "addressing": "direct", "nodes_per_gpu": n,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "state 2.55 GB > 129 MB L2, no flush needed",
                   "side_runs": "roofline.by_precision: the same workload with FP32 and FP16 storage "
                                "(FP32 collision), timed the same way after the headline"},
        "roofline": roof,
        "gpu_launches": head["kernels"],
        "clocks": head["clocks"],
    }
    if rank == 0 and not args.no_e2e:
        result["e2e"] = run_e2e(torch, lbm, args, head["rho_host"])
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = run_cpu_baseline(args.cpu_seconds)
    if rank == 0 and not args.no_sweep:
        result["variants"] = run_sweep(torch, lbm, args, hbm, pipe)
    if rank == 0 and not args.no_sparse:
        result["sparse"] = run_sparse(torch, lbm, args, hbm)
        if not args.no_solve:
            result["sparse"]["steady_flux"] = run_sparse_solve(torch, lbm, args)
    if rank == 0 and not args.no_shapes:
        result["paper_shapes"] = run_paper_shapes(torch, lbm, args, hbm, pipe)
    if rank == 0 and not args.no_batch:
        result["batch"] = run_batch(torch, lbm, args)
        log("batch", result["batch"])
    if rank == 0 and not args.no_serving:
        result["serving"] = run_serving(torch, lbm, args)
        log("serving", result["serving"])
    result["roofline"]["per_variant"] = per_variant_table(result)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def per_variant_table(result):
    """Compact table of every measured row: {name: [MFLUP/s, fraction of its
    own roof]} (full grid: scheme/precision/layout; node lists: sparse/...,
    paper shapes: channel/... and bed/...)."""
    table = {}
    for key, row in result.get("variants", {}).items():
        if "mflups" in row:
            table[key] = [row["mflups"], row["frac"]]
    for key, row in result.get("sparse", {}).items():
        if isinstance(row, dict) and "mflups" in row and "frac" in row:
            table["sparse/" + key] = [row["mflups"], row["frac"]]
    for key, row in result.get("paper_shapes", {}).items():
        table[key] = [row["mflups"], row["frac"]]
    return table


def main_reference(args):
    """The FP64 CPU oracle on the host cores, same workload, metric and
    arithmetic: each step is one oracle step (the push definition, OpenMP
    over cells) of the whole periodic 256^3 box from the same initial state
    (about 0.2 s per step on 16 cores)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    rho = inputs.density_noise(DIMS, seed=SEED)
    _, w = oracle.lattice()
    f = np.ascontiguousarray(w[:, None] * rho[None, :])
    for _ in range(args.warmup):
        f = oracle.push_full(DIMS, (1, 1, 1), None, f, OMEGA, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.push_full(DIMS, (1, 1, 1), None, f, OMEGA, nthreads=threads)
    secs = time.perf_counter() - t0
    n = int(np.prod(DIMS))
    value = n * args.steps / secs / 1e6
    sample = "each step: one oracle step of the whole 256^3 periodic box (%d nodes)" % n
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MFLUP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(secs / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "variant": "push definition (oracle)", "sample": sample},
        "cpu_baseline": {"value": round(value, 3), "unit": "MFLUP/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MFLUP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--sweep-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the FP32 / FP16 headline side runs")
    ap.add_argument("--no-sparse", action="store_true")
    ap.add_argument("--sparse-steps", type=int, default=50)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--solve-max-steps", type=int, default=20000)
    ap.add_argument("--no-shapes", action="store_true")
    ap.add_argument("--shape-steps", type=int, default=50)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-seconds", type=float, default=60.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-fp64", type=int, default=4)
    ap.add_argument("--serve-max-steps", type=int, default=30000)
    a = ap.parse_args(argv)
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    if a.steps < 1:
        ap.error("--steps must be >= 1")
    return a


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        main_reference(args)
    else:
        main_gb300(args)
