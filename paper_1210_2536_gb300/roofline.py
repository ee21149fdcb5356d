"""Algorithmic bytes of one SpMV per kernel variant (HBM roofline).

SpMV moves ~12 bytes per 2 flops in FP64, far below any tensor or ALU ridge,
so HBM bandwidth bounds every variant.  The bytes a variant must move are its
format's index and value arrays read once, x read once (it stays in L2), and
y written once (plus read when beta != 0):

  CSR (scalar / vector / merge)  (s_v + 4) NNZ + 4 (M + 1)
  ELL                            (s_v + 4) K M            (pad slots counted)
  DIA                            s_v Ndiags M + 4 Ndiags  (fill counted)
  COO                            (s_v + 8) NNZ
  every variant                  + s_x N + s_y M (1 + [beta != 0])

GFLOP/s counts 2 NNZ flops per product (true nonzeros only).
"""
from __future__ import annotations

ELEM = {"f64": 8, "f32": 4, "bf16": 2}
CSR_VARIANTS = (0, 1, 2, 3, 4)
V_ELL, V_DIA, V_COO = 5, 6, 7


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
    else:
        raise ValueError(variant)
    return float(mat + sx * n + sx * m * (2 if beta_nonzero else 1))


def flops(f: dict) -> float:
    return 2.0 * f["nnz"]
