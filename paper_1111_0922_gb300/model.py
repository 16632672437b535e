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


# FP64 instruction roof on GB300: 2 FP64 thread-instructions per clock per SM
# (ncu's sm__sass_thread_inst_executed_op_dfma_pred_on peak) on 152 SMs at the
# 2.07 GHz maximum SM clock.  The BGK collision issues 127 FP64 instructions
# per update without a body force (ncu, AA pattern on 256^3: 46 DADD, 63
# DFMA, 18 DMUL per node); counted from the source, a force adds 16 (u, u.g,
# one more operation per opposite pair) and TRT adds 18 (two more operations
# per opposite pair).
FP64_INST_PER_CLK_SM = 2
GB300_SMS = 152
GB300_SM_GHZ = 2.07
FP64_INST_BGK = 127


def fp64_inst_per_flup(force: bool = False, trt: bool = False) -> int:
    return FP64_INST_BGK + (16 if force else 0) + (18 if trt else 0)


def fp64_roof_mflups(force: bool = False, trt: bool = False) -> float:
    """FP64-pipe roofline in MFLUP/s of an FP64 step (any scheme)."""
    rate = FP64_INST_PER_CLK_SM * GB300_SMS * GB300_SM_GHZ * 1e9
    return rate / fp64_inst_per_flup(force, trt) / 1e6


def bound_roof(variant: str, indirect: bool, precision: str, hbm_gbs: float, force: bool = False,
               trt: bool = False):
    """(bound, roof MFLUP/s): the lower of the HBM and, for FP64, FP64-pipe
    roofs.  The two-step scheme's FP64 roof adds the time of its stream
    kernel (pure data movement, half of its bytes at HBM speed) to the
    collide kernel's FP64-pipe time, since the two kernels run one after the
    other."""
    hbm = roof_mflups(variant, indirect, precision, hbm_gbs)
    if precision == "f64":
        alu = fp64_roof_mflups(force, trt)
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
