"""Algorithmic bytes of one SpMV per kernel variant (HBM roofline).

SpMV moves ~12 bytes per 2 flops in FP64, far below any tensor or ALU ridge,
so HBM bandwidth bounds every variant.  The bytes a variant must move are its
format's index and value arrays read once, x read once (it stays in L2), and
y written once (plus read when beta != 0):

  CSR (scalar / vector / merge)  (s_v + 4) NNZ + 4 (M + 1)
  ELL                            (s_v + 4) K M            (pad slots counted)
  DIA                            s_v Ndiags M + 4 Ndiags  (fill counted)
  COO                            (s_v + 8) NNZ
  HYB                            (s_v + 4) K M + (s_v + 8) Ncoo
  SELL                           (s_v + 4) slots + 4 Mp + 12 Nslices + 8
                                 (perm 4 B / position, width and pointer per slice)
  BCSR                           (s_v b^2 + 4) Nblocks + 4 (ceil(M/b) + 1)
  SPLIT                          (s_v + 4) (NNZ - Nshort) + 12 Nchunks + (s_v + 8) Nshort
                                 + 4 empty rows (+ 8 per long row, at most Nchunks: counted as Nchunks)
  every variant                  + s_x N + s_y M (1 + [beta != 0])

The HYB / SELL / BCSR / SPLIT sizes come from the built format
(SpMatrix.features() adds hyb_K, hyb_ncoo, sell_ns, sell_slots, bcsr_b,
bcsr_nb, split_nc and split_ns once built).

GFLOP/s counts 2 NNZ flops per product (true nonzeros only).

On random-column matrices the binding roof is the rate of L2 sector requests:
every stored product gathers one random x element (a whole 32-byte sector)
besides the format's streamed bytes.  ``l2_sectors`` counts them; the bench
compares the count per second with a measured rate (random gathers plus
their streamed 4-byte indices, 1.125 sectors per gather).

GB300 runs FP64 arithmetic at about 2 operations per clock per SM, so an
FP64 product that spends one fused multiply-add per stored slot can be bound
by the FP64 pipe instead of HBM; ``bound`` picks whichever roof binds.
"""
from __future__ import annotations

ELEM = {"f64": 8, "f32": 4, "bf16": 2}
CSR_VARIANTS = (0, 1, 2, 3, 4, 8)
V_ELL, V_DIA, V_COO = 5, 6, 7
V_HYB, V_SELL, V_BCSR, V_SPLIT = 9, 10, 11, 12


def algorithmic_bytes(f: dict, variant: int, dtype: str, beta_nonzero: bool = False) -> float:
    sv = ELEM[dtype]
    sx = 8 if dtype == "f64" else 4
    m, n, nnz = f["m"], f["n"], f["nnz"]
    if variant in CSR_VARIANTS:
        mat = (sv + 4) * nnz + 4 * (m + 1)
    elif variant == V_ELL:
        mat = (sv + 4) * f["max_rd"] * m
    elif variant == V_DIA:
        mat = sv * f["ndiags"] * m + 4 * f["ndiags"]
    elif variant == V_COO:
        mat = (sv + 8) * nnz
    elif variant == V_HYB:
        mat = (sv + 4) * f["hyb_K"] * m + (sv + 8) * f["hyb_ncoo"]
    elif variant == V_SELL:
        mat = (sv + 4) * f["sell_slots"] + 4 * 32 * f["sell_ns"] + 12 * f["sell_ns"] + 8
    elif variant == V_BCSR:
        b = f["bcsr_b"]
        mat = (sv * b * b + 4) * f["bcsr_nb"] + 4 * ((m + b - 1) // b + 1)
    elif variant == V_SPLIT:
        ns, nc = f["split_ns"], f["split_nc"]
        mat = (sv + 4) * (nnz - ns) + 12 * nc + 8 * nc + (sv + 8) * ns + 4 * f["empty_rows"]
    else:
        raise ValueError(variant)
    return float(mat + sx * n + sx * m * (2 if beta_nonzero else 1))


def flops(f: dict) -> float:
    return 2.0 * f["nnz"]


# FP64 arithmetic on GB300: 152 SMs x 2 FP64 operations per clock x 2.07 GHz
# (one fused multiply-add counts as one operation, i.e. 2 flops):
# 629.3 G operations/s = 1.2586 TFLOP/s.  FP32 units are 64x wider, so only
# FP64 kernels can be bound by arithmetic.
SMS, FP64_OPS_PER_CLK_PER_SM, SM_CLOCK_GHZ = 152, 2, 2.07
FP64_PEAK_TFLOPS = SMS * FP64_OPS_PER_CLK_PER_SM * 2 * SM_CLOCK_GHZ / 1e3


def fp64_ops(f: dict, variant: int) -> float:
    """FP64 fused multiply-adds one product needs in this format: one per
    stored slot the kernel multiplies (fill and padding included)."""
    if variant == V_ELL:
        return float(f["max_rd"] * f["m"])
    if variant == V_DIA:
        return float(f["ndiags"] * f["m"])
    if variant == V_HYB:
        return float(f["hyb_K"] * f["m"] + f["hyb_ncoo"])
    if variant == V_SELL:
        return float(f["sell_slots"])
    if variant == V_BCSR:
        return float(f["bcsr_nb"] * f["bcsr_b"] ** 2)
    return float(f["nnz"])


def l2_sectors(f: dict, variant: int, dtype: str) -> float:
    """32-byte L2 sector requests of one product on a matrix with random
    columns (a lower bound):
    - one per gathered slot (a random x element is one sector that L1 does
      not hold);
    - the format's streamed index and value bytes, in sectors;
    - y: formats that write rows one at a time from lanes far apart (COO and
      SPLIT tiles, SELL through its row permutation) spend a whole sector per
      row; the others write y in full sectors;
    - FP32 / BF16 COO and SPLIT tiles also load each thread's next row (one
      sector per 8 entries; FP64 takes it from the next lane).
    Banded matrices gather x in coalesced runs, so this count holds for
    random-column matrices only."""
    sy = 8 if dtype == "f64" else 4
    byts = algorithmic_bytes(f, variant, dtype) - sy * f["n"]   # x comes by gathers
    extra = 0.0
    if variant == V_SELL:
        gathers = f["sell_slots"]
    elif variant == V_HYB:
        gathers = f["hyb_K"] * f["m"] + f["hyb_ncoo"]
    elif variant == V_ELL:
        gathers = f["max_rd"] * f["m"]
    else:
        gathers = f["nnz"]
    if variant in (V_COO, V_SPLIT, V_SELL):
        byts -= sy * f["m"]
        extra += f["m"]
    if variant in (V_COO, V_SPLIT) and dtype != "f64":
        extra += (f["nnz"] if variant == V_COO else f["split_ns"]) / 8.0
    return float(gathers) + byts / 32.0 + extra


def bound(f: dict, variant: int, dtype: str, seconds: float, hbm_gbs: float,
          fp64_tflops: float | None = None) -> dict:
    """The binding roofline of one launch: HBM bytes, or (FP64 storage) FP64
    arithmetic, whichever needs more time at peak; achieved/peak for it.
    fp64_tflops is the measured FP64 roof (smat_measure_fp64_rate x 2);
    without it the derived FP64_PEAK_TFLOPS serves."""
    byts = algorithmic_bytes(f, variant, dtype)
    t_hbm = byts / (hbm_gbs * 1e9)
    out = {"bound": "hbm", "achieved": byts / seconds / 1e9, "peak": hbm_gbs, "unit": "GB/s",
           "alg_bytes": byts}
    if dtype == "f64":
        roof = fp64_tflops if fp64_tflops else FP64_PEAK_TFLOPS
        ops = fp64_ops(f, variant)
        t_alu = 2.0 * ops / (roof * 1e12)
        out["fp64_frac"] = t_alu / seconds
        if t_alu > t_hbm:
            out.update(bound="alu", achieved=2.0 * ops / seconds / 1e12, peak=roof, unit="TFLOP/s",
                       alg_fp64_fma=ops)
    out["hbm_frac"] = t_hbm / seconds
    out["frac"] = out["achieved"] / out["peak"]
    return out
