"""Host-side logic of bench.py (no GPU): the FP64-pipe roofline, the
profile lines it reads (a count or a traffic figure whose kernel sources
changed is ignored), and the per-variant table."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1111_0922_gb300 import model  # noqa: E402


def test_profile_lines_are_gated_by_source_hash(tmp_path):
    h64 = bench.kernel_source_hash("f64")
    (tmp_path / "a.md").write_text(
        "text\n"
        "fp64_inst_per_clk_sm 2\n"
        "fp64_inst_per_flup bgk 114.0 source_hash %s\n"
        "fp64_inst_per_flup bgk_force 127.0 source_hash 0000000000000000\n"
        "dram_bytes_per_launch aa_f64_soa_direct_256 111 source_hash 0000000000000000\n"
        "dram_bytes_per_launch aa_f64_soa_direct_256 222 source_hash %s\n" % (h64, h64))
    per_clk, per_flup = bench.profiled_fp64(str(tmp_path))
    assert per_clk == 2.0 and per_flup == {"bgk": 114.0}  # the stale count is ignored
    assert bench.profiled_traffic("aa_f64_soa_direct_256", "f64", str(tmp_path)) == 222.0
    assert bench.profiled_traffic("aa_f32_soa_direct_256", "f32", str(tmp_path)) is None


def test_fp64_roofline_from_measured_inputs():
    pipe = model.Fp64Pipe(152, 2.07, 2.0, {"bgk": 114.0, "bgk_force": 127.0, "trt_force": 145.0})
    head = {"nodes": 256 ** 3, "per_launch_s": 3.54e-3}
    r = bench.fp64_roofline(head, pipe, 6780.0, "measured")
    assert r["bound"] == "alu" and r["peak"] == round(152 * 2 * 2.07, 1)
    assert abs(r["achieved"] - 114 * 256 ** 3 / 3.54e-3 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert r["hbm"]["frac"] < 0.25  # the FP64 step moves 304 B per update at a fifth of the copy rate
    none = bench.fp64_roofline(head, None, 6780.0, "measured")
    assert none["frac"] is None and none["peak_kind"].startswith("unavailable")


def test_per_variant_table():
    res = {"variants": {"aa/f32/soa": {"mflups": 45000.0, "frac": 1.01}, "swap/f64/aos": {"unsupported": "x"}},
           "sparse": {"aa/f16s/indirect": {"mflups": 45100.0, "frac": 0.745}, "steady_flux": {"f32": {}}},
           "paper_shapes": {"bed/et/f32": {"mflups": 24000.0, "frac": 0.66}}}
    t = bench.per_variant_table(res)
    assert t == {"aa/f32/soa": [45000.0, 1.01], "sparse/aa/f16s/indirect": [45100.0, 0.745],
                 "bed/et/f32": [24000.0, 0.66]}
