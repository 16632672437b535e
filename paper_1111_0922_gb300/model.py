"""Bytes-per-update performance model (Sec. 9, Eq. 1-2, Tab. 1-8) and its
adaptation to HBM on GB300.

The paper counts, per lattice-node update of D3Q19 (q = 19), the PDF and IDX
transfers of each propagation scheme, including the write-allocate (read for
ownership) of every store that misses the cache (Tab. 1-6), and divides the
bytes by about 200 FLOP (its TRT collision) to get the code balance B_code
(Eq. 1, Tab. 8).  Performance is bounded by memory bandwidth / bytes per
update when B_code exceeds the machine balance (Eq. 2).

On a GPU a store of a whole 32-byte sector allocates in L2 without reading
DRAM, so the write-allocate terms drop.  ``gpu_counts`` gives the PDF and IDX
words each kernel of this library moves per fluid-node update (FLUP); the
roofline of a variant is HBM bandwidth / (PDFs * sizeof(PDF) + IDX * 4).
"""
from __future__ import annotations

Q = 19
FLOP_PER_LUP_PAPER = 200  # TRT, Sec. 9

PDF_BYTES = {"f64": 8, "f32": 4, "f16s": 2}
IDX_BYTES = 4

VARIANTS = ("ts", "os_push", "os_pull", "cg", "swap", "aa", "et")


def paper_counts(variant: str, indirect: bool):
    """(PDF transfers, IDX transfers) per update as in Tab. 1-6, with the
    write-allocate transfers of a cache-based CPU."""
    q = Q
    pdfs = {"ts": 6 * q, "os": 3 * q, "os-nt": 2 * q, "cg": 3 * q - 1, "swap": 3 * q - 1,
            "aap": 2 * q, "et": 2 * q}[variant]
    if not indirect:
        return pdfs, 0
    idx = {"ts": 2 * (q - 1), "os": q - 1, "os-nt": q - 1, "cg": q - 1, "swap": (q - 1) // 2,
           "aap": (q - 1) // 2, "et": (q + 1) // 2}[variant]
    return pdfs, idx


def paper_bytes(variant: str, indirect: bool, pdf_bytes: int = 8, idx_bytes: int = 4) -> int:
    p, i = paper_counts(variant, indirect)
    return p * pdf_bytes + i * idx_bytes


def paper_bcode(variant: str, indirect: bool, flop: int = FLOP_PER_LUP_PAPER) -> float:
    """Code balance B_code = bytes / FLOP (Eq. 1)."""
    return paper_bytes(variant, indirect) / flop


def gpu_counts(variant: str, indirect: bool):
    """(PDF words, IDX words) per FLUP that this library's kernels move
    through DRAM at best (no write-allocate).

    ts       collide kernel q loads + q stores, stream kernel q + q, and the
             stream kernel's q-1 neighbour lookups
    os_*     q loads + q stores; q-1 lookups
    cg       as one-step, plus the periodic ghost-plane copies (not counted)
    swap     q loads + q stores at best (link exchanges across tile faces
             re-touch a few slots, not counted); q-1 lookups per update
    aa       q loads + q stores every step; q-1 lookups on odd steps only,
             so (q-1)/2 on average (Tab. 5)
    et       q loads + q stores; (q-1)/2 lookups: the neighbours along the
             nine 'positive' directions, with the solid flags of the nine
             opposite links packed into their top bits (the paper counts
             (q+1)/2, Tab. 6)
    """
    q = Q
    pdfs = {"ts": 4 * q}.get(variant, 2 * q)
    if not indirect:
        return pdfs, 0
    idx = {"ts": q - 1, "os_push": q - 1, "os_pull": q - 1, "cg": q - 1, "swap": q - 1,
           "aa": (q - 1) / 2, "et": (q - 1) / 2}[variant]
    return pdfs, idx


def gpu_bytes(variant: str, indirect: bool, precision: str) -> float:
    p, i = gpu_counts(variant, indirect)
    return p * PDF_BYTES[precision] + i * IDX_BYTES


def roof_mflups(variant: str, indirect: bool, precision: str, hbm_gbs: float) -> float:
    """HBM roofline in MFLUP/s: bandwidth / bytes per FLUP."""
    return hbm_gbs * 1e9 / gpu_bytes(variant, indirect, precision) / 1e6


# FP64-pipe roof.  GB300 runs FP64 arithmetic on a narrow pipe (two thread
# instructions per SM clock), so every FP64 step kernel is bound by its FP64
# instruction count per update, not by HBM.  Every input of this roof is
# measured, none is a constant of this module: the SM count is the device's
# attribute, the SM clock the median sampled during the timed region, and
# the pipe's peak rate and the instructions per update (DADD + DMUL + DFMA
# thread instructions of the collision, one count per collision kind) come
# from an ncu capture whose summary is committed under profiles/.
COLLISIONS = ("bgk", "bgk_force", "trt_force")


def collision_kind(force: bool = False, trt: bool = False) -> str:
    if trt and not force:
        raise ValueError("no captured FP64 count for TRT without a body force")
    return "trt_force" if trt else ("bgk_force" if force else "bgk")


class Fp64Pipe:
    """FP64-pipe roof from measured inputs.

    sms              streaming multiprocessors (device attribute)
    sm_ghz           SM clock during the timed region (GHz)
    inst_per_clk_sm  peak FP64 thread instructions per SM clock (ncu's
                     sm__thread_inst_executed_pipe_fp64_pred_on peak)
    inst_per_flup    {collision kind: FP64 thread instructions per update}
                     (ncu: the kernel's DADD + DMUL + DFMA thread instructions
                     divided by the nodes of the launch)
    """

    def __init__(self, sms: int, sm_ghz: float, inst_per_clk_sm: float, inst_per_flup: dict):
        self.sms = int(sms)
        self.sm_ghz = float(sm_ghz)
        self.inst_per_clk_sm = float(inst_per_clk_sm)
        self.inst_per_flup = dict(inst_per_flup)

    def inst_rate(self) -> float:
        """Peak FP64 thread instructions per second of the whole GPU."""
        return self.sms * self.inst_per_clk_sm * self.sm_ghz * 1e9

    def roof_mflups(self, force: bool = False, trt: bool = False) -> float:
        return self.inst_rate() / self.inst_per_flup[collision_kind(force, trt)] / 1e6

    def as_dict(self) -> dict:
        return {"sms": self.sms, "sm_ghz": self.sm_ghz, "inst_per_clk_sm": self.inst_per_clk_sm,
                "inst_per_flup": self.inst_per_flup}


def bound_roof(variant: str, indirect: bool, precision: str, hbm_gbs: float, fp64: Fp64Pipe | None = None,
               force: bool = False, trt: bool = False):
    """(bound, roof MFLUP/s): the lower of the HBM and, for FP64, FP64-pipe
    roofs (the latter only when `fp64` is given).  The two-step scheme's
    FP64 roof adds the time of its stream kernel (pure data movement, half
    of its bytes at HBM speed) to the collide kernel's FP64-pipe time, since
    the two kernels run one after the other."""
    hbm = roof_mflups(variant, indirect, precision, hbm_gbs)
    if precision == "f64" and fp64 is not None:
        alu = fp64.roof_mflups(force, trt)
        if variant == "ts":
            stream_s = gpu_bytes(variant, indirect, precision) / 2 / (hbm_gbs * 1e9)
            alu = 1.0 / (1.0 / (alu * 1e6) + stream_s) / 1e6
        if alu < hbm:
            return "alu", alu
    return "hbm", hbm


def kernel_bytes_per_flup(variant: str, indirect: bool, precision: str, odd: bool = False) -> float:
    """Algorithmic DRAM bytes per FLUP of ONE launch of the variant's main
    kernel (the AA pattern's even and odd kernels differ)."""
    pb = PDF_BYTES[precision]
    if variant == "aa":
        return 2 * Q * pb + ((Q - 1) * IDX_BYTES if (indirect and odd) else 0)
    if variant == "ts":
        # one of its two kernels; the stream kernel carries the lookups
        return 2 * Q * pb + ((Q - 1) * IDX_BYTES if (indirect and odd) else 0)
    return gpu_bytes(variant, indirect, precision)
