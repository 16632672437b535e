"""Run one workload case through the C ABI and print its throughput.

    python -m paper_1111_0922_gb300.run_case --variant aa --precision f32 \
        --addressing direct --workload dense256 --steps 100

Workloads:
  dense<N>   periodic N^3 full grid, rho = 1 + 1e-3 U[-1,1) (seed 2), omega 1.7
  pack<N>    periodic N^3 sphere pack, r = 8, porosity 0.6 (seed 3),
             g = 1e-6 along x, omega 1.0, from rest
  duct<N>    N^3 duct, periodic x, walls y/z, g = 1e-6 x, omega 1.0
  channel    the paper's 500x100x100 empty channel (walls y/z), g = 1e-6 x
  bed        the paper-shaped 500x100x100 packed bed (about 2.1 M fluid cells)
Prints one JSON line: nodes, steps, seconds, MFLUP/s, bytes per FLUP, roof.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

from . import inputs, lbm, model


def measured_hbm_gbs(default: float = 6800.0) -> float:
    """HBM copy bandwidth measured on this machine pool, else the fallback."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f).get("hbm_gbs", default))
    return default


def setup(args):
    import torch

    kind = "".join(c for c in args.workload if c.isalpha())
    size = int("".join(c for c in args.workload if c.isdigit()) or "256")
    dims = (size, size, size)
    common = dict(variant=args.variant, addressing=args.addressing, layout=args.layout,
                  precision=args.precision, block_size=args.block_size,
                  nodes_per_thread=args.nodes_per_thread,
                  store_hint=args.store_hint, swap_schedule=args.swap_schedule, pair_z=args.pair_z,
                  trt_magic=3.0 / 16.0 if args.trt else 0.0)
    if kind == "dense":
        lat = lbm.Lattice(dims, (1, 1, 1), omega=1.7, **common)
        lat.set_geometry(None)
        rho = torch.from_numpy(inputs.density_noise(dims, seed=2)).cuda()
        lat.init(rho, on_device=True)  # with IDX every cell is a node, in cell order
        return lat
    if kind == "pack":
        pack = inputs.sphere_pack(dims, 0.6, radius=8.0, seed=3)
        lat = lbm.Lattice(dims, (1, 1, 1), omega=1.0, force=(1e-6, 0, 0), **common)
        lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
        lat.init()
        return lat
    if kind == "channel":
        d, per = inputs.paper_channel()
        lat = lbm.Lattice(d, per, omega=1.0, force=(1e-6, 0, 0), **common)
        lat.set_geometry(None)
        lat.init()
        return lat
    if kind == "bed":
        pack = inputs.paper_packed_bed()
        lat = lbm.Lattice(pack.dims, pack.periodic, omega=1.0, force=(1e-6, 0, 0), **common)
        lat.set_geometry_spheres(pack.centres, pack.radius, pack.unit)
        lat.init()
        return lat
    if kind == "duct":
        d, per = inputs.duct(size)
        lat = lbm.Lattice(d, per, omega=1.0, force=(1e-6, 0, 0), **common)
        lat.set_geometry(None)
        lat.init()
        return lat
    raise SystemExit("unknown workload %s" % args.workload)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--variant", default="aa", choices=list(lbm.VARIANTS))
    ap.add_argument("--precision", default="f32", choices=list(lbm.PRECISIONS))
    ap.add_argument("--addressing", default="direct", choices=["direct", "indirect"])
    ap.add_argument("--layout", default="soa", choices=["soa", "aos"])
    ap.add_argument("--workload", default="dense256")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--block-size", type=int, default=0)
    ap.add_argument("--nodes-per-thread", type=int, default=0)
    ap.add_argument("--store-hint", type=int, default=0,
                    help="OS push/pull, SoA: 1 = cache-streaming stores of the second lattice (OS-NT analogue)")
    ap.add_argument("--swap-schedule", type=int, default=0,
                    help="swap, full grid: 0 default, 1 coloured passes, 2 coloured with tensor-copy staging")
    ap.add_argument("--pair-z", type=int, default=0,
                    help="AA, FP16 storage, full grid: 0 default (z pairs where allowed), 2 one node per thread")
    ap.add_argument("--trt", action="store_true", help="two-relaxation-time collision, magic 3/16")
    args = ap.parse_args(argv)
    import torch

    from . import build

    build.build()
    lbm.load()
    torch.cuda.set_device(0)
    lat = setup(args)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    lat.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    info = lat.info
    n = int(info.nodes)
    ind = args.addressing == "indirect"
    bpf = model.gpu_bytes(args.variant, ind, args.precision)
    peak = measured_hbm_gbs()
    mflups = n * args.steps / secs / 1e6
    roof = peak * 1e9 / bpf / 1e6
    print(json.dumps({"case": vars(args), "nodes": n, "seconds": secs, "mflups": round(mflups, 1),
                      "bytes_per_flup": bpf, "roof_mflups": round(roof, 1), "frac": round(mflups / roof, 4),
                      "kernels_per_step": info.kernels_per_step}))
    lat.close()


if __name__ == "__main__":
    sys.exit(main())
