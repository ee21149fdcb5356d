"""Shared helpers for the parity tests: build library handles from the seeded
inputs, run the oracle on the same inputs, and compare with the stated bars."""
import numpy as np

import oracle
from paper_1210_2536_gb300.synth import CSR

# Per-row bars: |y - y_ref| <= TOL * (|alpha| * sum_j |a_ij x_j| + |beta y_i|)
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5}


def stored_values(A: CSR, dtype: str):
    """(values to hand to the library, the same stored values widened to FP64)."""
    if dtype == "f64":
        return A.val, A.val
    if dtype == "f32":
        v = A.val.astype(np.float32)
        return v, v.astype(np.float64)
    b = oracle.round_bf16(A.val)
    return b, oracle.bf16_to_double(b)


def vec(v, dtype):
    return np.asarray(v, dtype=np.float64 if dtype == "f64" else np.float32)


def reference(A: CSR, vals64, x, alpha, beta, y0):
    """Oracle product and the per-row error scale on the stored values."""
    x64 = np.asarray(x, dtype=np.float64)
    y64 = None if y0 is None else np.asarray(y0, dtype=np.float64)
    ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, vals64, x64, alpha, beta, y64, threads=8)
    scale = abs(alpha) * oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(vals64), np.abs(x64), threads=8)
    if beta != 0 and y64 is not None:
        scale = scale + abs(beta) * np.abs(y64)
    return ref, scale


def assert_close_rows(y, ref, scale, tol, what=""):
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - ref)
    bad = err > tol * scale
    if np.any(bad):
        i = int(np.argmax(np.where(bad, err / np.maximum(scale, 1e-300), 0)))
        raise AssertionError(f"{what}: {int(bad.sum())} rows out of bound; row {i}: y={y[i]!r} ref={ref[i]!r} "
                             f"scale={scale[i]!r} tol={tol}")


def csr_from_degrees(deg, n, seed):
    """A CSR matrix whose rows have the given lengths, columns drawn uniformly
    without replacement from [0, n), values 1."""
    rng = np.random.default_rng(seed)
    deg = np.asarray(deg, dtype=np.int64)
    rowptr = np.zeros(len(deg) + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(deg)
    cols = [np.sort(rng.choice(n, size=int(d), replace=False)) for d in deg]
    colidx = np.concatenate(cols).astype(np.int32) if len(cols) else np.zeros(0, np.int32)
    return CSR(len(deg), n, rowptr, colidx, np.ones(len(colidx)))
