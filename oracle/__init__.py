"""CPU oracle for the SMAT hot path (arXiv 1210.2536) -- TEST INFRASTRUCTURE.

Thin ctypes/numpy front end to ``oracle.c`` (plain C, FP64, no FMA
contraction).  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg and reference arm (``--impl reference``) of ``bench.py`` may import this
package; the library under ``paper_1210_2536_gb300`` never does, and the two
share no code.

Every function restates a definition of the paper:
  spmv_csr        y = alpha*A*x + beta*y in CSR, fixed ascending order (Sec. 2.1, 3)
  spmv_csr_threads  the same on T threads, nonzero-balanced row split (Sec. 6)
  segment_starts  that split on 8-row boundaries, for per-segment plans (Sec. 6)
  features        Table "Feature parameters of a sparse matrix" (Sec. 4)
  to_ell/to_dia/to_coo  the four basic storage formats (Sec. 2.1)
  to_hyb/sell_layout/to_sell/to_bcsr  further GPU formats left to future work
                  in Sec. 8 (HYB, SELL-C-sigma, BCSR; published definitions)
  split_rows      rows split by length: long rows in chunks, short rows as COO
  mlp_*           the learned replacement of the ruleset classifier (Sec. 5)
  admissible      the 20x fill rule plus a byte cap and a diagonal-count cap (Sec. 2.3)
  rules_select    the observations of Sec. 4 as an ordered rule set (Sec. 6)
  selector_inputs/learned_select  the learned selector's inputs and pick
Readings taken where the paper is silent are listed in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MLP_IN, MLP_H, MLP_OUT = 12, 64, 8


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, -O2 -ffp-contract=off: every FP op is one rounding)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=gnu11", "-o", tmp, _SRC, "-lm", "-pthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Features(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("m", "n", "nnz", "max_rd", "min_rd", "ndiags", "ntdiags", "empty_rows", "s2_lo", "s2_hi")] + \
               [(n, ctypes.c_double) for n in
                ("aver_rd", "var_rd", "er_dia", "er_ell", "ntdiags_ratio", "r")] + [("r_valid", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.oracle_spmv_csr.argtypes = [i64, vp, vp, vp, vp, f64, f64, vp]
        L.oracle_spmv_csr_threads.argtypes = [i64, vp, vp, vp, vp, f64, f64, vp, ctypes.c_int]
        L.oracle_partition_rows.argtypes = [i64, vp, ctypes.c_int, vp]
        L.oracle_max_rd.argtypes = [i64, vp]
        L.oracle_max_rd.restype = i64
        L.oracle_features.argtypes = [i64, i64, vp, vp, i64, i64, vp, vp, ctypes.POINTER(_Features)]
        L.oracle_to_ell.argtypes = [i64, vp, vp, vp, i64, i64, i64, vp, vp]
        L.oracle_dia_offsets.argtypes = [i64, i64, vp, vp, vp]
        L.oracle_dia_offsets.restype = i64
        L.oracle_to_dia.argtypes = [i64, vp, vp, vp, i64, vp, i64, i64, vp]
        L.oracle_to_coo.argtypes = [i64, vp, vp]
        L.oracle_hyb_width.argtypes = [i64, vp]
        L.oracle_hyb_width.restype = i64
        L.oracle_to_hyb.argtypes = [i64, vp, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp]
        L.oracle_to_hyb.restype = i64
        L.oracle_sell_layout.argtypes = [i64, vp, i64, i64, vp, vp, vp]
        L.oracle_sell_layout.restype = i64
        L.oracle_to_sell.argtypes = [i64, vp, vp, vp, i64, i64, vp, vp, vp, vp, vp]
        L.oracle_to_bcsr.argtypes = [i64, i64, vp, vp, vp, i64, i64, vp, vp, vp]
        L.oracle_to_bcsr.restype = i64
        L.oracle_bcsr_choose.argtypes = [i64, i64, vp, vp, i64, vp]
        L.oracle_bcsr_choose.restype = i64
        L.oracle_split.argtypes = [i64, vp, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_round_bf16.argtypes = [i64, vp, vp]
        L.oracle_bf16_to_double.argtypes = [i64, vp, vp]
        L.oracle_mlp_param_count.restype = i64
        L.oracle_mlp_forward.argtypes = [vp, i64, vp, vp]
        L.oracle_mlp_loss_grad.argtypes = [vp, i64, vp, vp, vp]
        L.oracle_mlp_loss_grad.restype = f64
        L.oracle_adam.argtypes = [i64, vp, vp, vp, vp, i64, f64, f64, f64, f64]
        _lib = L
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


# ---------------------------------------------------------------------------
# SpMV (Sec. 2.1 / Sec. 3: CSR is the unified interface and default format)
# ---------------------------------------------------------------------------

def spmv_csr(m, rowptr, colidx, val, x, alpha=1.0, beta=0.0, y=None, threads: int = 1):
    """y = alpha*A*x + beta*y with FP64 accumulation in ascending storage order.
    ``val`` and ``x`` are widened to FP64 first (exact for FP32 / BF16 storage).
    Returns a new array; ``y`` is read only when beta != 0."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v, pv = _c(val, np.float64)
    xx, px = _c(x, np.float64)
    out = np.zeros(m, dtype=np.float64) if y is None else np.array(y, dtype=np.float64, copy=True)
    if threads <= 1:
        lib().oracle_spmv_csr(m, prp, pci, pv, px, float(alpha), float(beta), out.ctypes.data)
    else:
        lib().oracle_spmv_csr_threads(m, prp, pci, pv, px, float(alpha), float(beta), out.ctypes.data,
                                      int(threads))
    return out


def spmv_csr_rows(rowptr, colidx, val, x, r0, r1, alpha, beta, y, threads: int = 1):
    """Rows [r0, r1) of y = alpha*A*x + beta*y, written into ``y`` in place.
    All arrays must already be contiguous (int32 indices, float64 values)."""
    for a, t in ((rowptr, np.int32), (colidx, np.int32), (val, np.float64), (x, np.float64), (y, np.float64)):
        assert a.dtype == t and a.flags.c_contiguous
    m = int(r1 - r0)
    if m <= 0:
        return
    prp = rowptr.ctypes.data + 4 * int(r0)
    py = y.ctypes.data + 8 * int(r0)
    if threads <= 1:
        lib().oracle_spmv_csr(m, prp, colidx.ctypes.data, val.ctypes.data, x.ctypes.data, float(alpha),
                              float(beta), py)
    else:
        lib().oracle_spmv_csr_threads(m, prp, colidx.ctypes.data, val.ctypes.data, x.ctypes.data, float(alpha),
                                      float(beta), py, int(threads))


def partition_rows(m, rowptr, nthreads):
    rp, prp = _c(rowptr, np.int32)
    b = np.zeros(nthreads + 1, dtype=np.int64)
    lib().oracle_partition_rows(m, prp, nthreads, b.ctypes.data)
    return b


def segment_starts(m, rowptr, nseg):
    """Row starts of the per-segment plans (Sec. 6: the nonzeros divided
    evenly, at whole rows): the nonzero-balanced bounds of ``partition_rows``,
    each moved down to a multiple of 8 rows; a bound that does not pass the
    previous one, or reaches M, is dropped.  Returns [0, ..., M]."""
    b = partition_rows(m, rowptr, nseg)
    starts = [0]
    for r in b[1:-1]:
        r8 = int(r) // 8 * 8
        if starts[-1] < r8 < m:
            starts.append(r8)
    return starts + [m]


def spmv_rows_sampled(rowptr, colidx, val, x, rows, alpha=1.0, beta=0.0, y_in=None):
    """The oracle product for selected rows only (for full-size parity checks):
    builds the sub-CSR of those rows and runs ``spmv_csr`` on it."""
    rows = np.asarray(rows, dtype=np.int64)
    rp = np.asarray(rowptr, dtype=np.int64)
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    sub_rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=sub_rp[1:])
    idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if len(rows) else np.zeros(0, np.int64)
    yb = None if y_in is None else np.asarray(y_in, dtype=np.float64)[rows]
    return spmv_csr(len(rows), sub_rp.astype(np.int32), np.asarray(colidx)[idx], np.asarray(val)[idx], x,
                    alpha, beta, yb)


# ---------------------------------------------------------------------------
# Features (Sec. 4)
# ---------------------------------------------------------------------------

def features(m, n, rowptr, colidx, tau=(3, 5)):
    """All feature parameters plus the row-degree histogram and the per-diagonal
    counts (index d + M - 1 for diagonal d = j - i)."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    mx = int(lib().oracle_max_rd(m, prp)) if m > 0 else 0
    hist = np.zeros(mx + 1, dtype=np.int64)
    dcnt = np.zeros(max(m + n - 1, 1), dtype=np.int64)
    f = _Features()
    lib().oracle_features(m, n, prp, pci, int(tau[0]), int(tau[1]), hist.ctypes.data, dcnt.ctypes.data,
                          ctypes.byref(f))
    d = {name: getattr(f, name) for name, _ in _Features._fields_}
    d["s2"] = (d.pop("s2_hi") << 64) | (d.pop("s2_lo") & 0xFFFFFFFFFFFFFFFF)
    d["hist"] = hist
    d["diag_cnt"] = dcnt[: m + n - 1] if m + n > 0 else dcnt[:0]
    return d


# ---------------------------------------------------------------------------
# Conversions (Sec. 2.1)
# ---------------------------------------------------------------------------

def pitch(m: int) -> int:
    """Row pitch of the ELL and DIA arrays: M rounded up to a multiple of 32."""
    return (m + 31) // 32 * 32


def to_ell(m, rowptr, colidx, val, K=None, P=None):
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v = np.ascontiguousarray(val)
    if K is None:
        K = int(np.max(np.diff(rp))) if m > 0 else 0
    P = pitch(m) if P is None else P
    col = np.empty(K * P, dtype=np.int32)
    out = np.empty(K * P, dtype=v.dtype)
    lib().oracle_to_ell(m, prp, pci, v.ctypes.data, v.itemsize, K, P, col.ctypes.data, out.ctypes.data)
    return col, out, K, P


def dia_offsets(m, n, rowptr, colidx):
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    nd = int(lib().oracle_dia_offsets(m, n, prp, pci, None))
    off = np.empty(nd, dtype=np.int32)
    lib().oracle_dia_offsets(m, n, prp, pci, off.ctypes.data)
    return off


def to_dia(m, n, rowptr, colidx, val, P=None):
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v = np.ascontiguousarray(val)
    off = dia_offsets(m, n, rp, ci)
    P = pitch(m) if P is None else P
    out = np.empty(len(off) * P, dtype=v.dtype)
    lib().oracle_to_dia(m, prp, pci, v.ctypes.data, v.itemsize, off.ctypes.data, len(off), P, out.ctypes.data)
    return off, out, P


def to_coo(m, rowptr):
    rp, prp = _c(rowptr, np.int32)
    nnz = int(rp[-1]) if m > 0 else 0
    row = np.empty(nnz, dtype=np.int32)
    lib().oracle_to_coo(m, prp, row.ctypes.data)
    return row


def hyb_width(m, rowptr) -> int:
    """HYB's ELL width K: the largest k with 3 * #{rows with >= k entries} >= M."""
    rp, prp = _c(rowptr, np.int32)
    return int(lib().oracle_hyb_width(m, prp))


def to_hyb(m, rowptr, colidx, val, K=None, P=None):
    """HYB = ELL part (K x P, column-major) + COO part (row, col, val) of the
    entries past each row's first K.  Returns (ell_col, ell_val, coo_row,
    coo_col, coo_val, K, P)."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v = np.ascontiguousarray(val)
    K = hyb_width(m, rp) if K is None else K
    P = pitch(m) if P is None else P
    ncoo = int(lib().oracle_to_hyb(m, prp, pci, v.ctypes.data, v.itemsize, K, P, None, None, None, None, None))
    ecol = np.empty(K * P, dtype=np.int32)
    ev = np.empty(K * P, dtype=v.dtype)
    crow = np.empty(ncoo, dtype=np.int32)
    ccol = np.empty(ncoo, dtype=np.int32)
    cv = np.empty(ncoo, dtype=v.dtype)
    lib().oracle_to_hyb(m, prp, pci, v.ctypes.data, v.itemsize, K, P, ecol.ctypes.data, ev.ctypes.data,
                        crow.ctypes.data, ccol.ctypes.data, cv.ctypes.data)
    return ecol, ev, crow, ccol, cv, K, P


SELL_C = 32


def sell_layout(m, rowptr, sigma, C=SELL_C):
    """SELL-C-sigma slice structure: (perm[Mp], width[Mp/C], slice_ptr[Mp/C + 1])."""
    rp, prp = _c(rowptr, np.int32)
    mp = (m + C - 1) // C * C
    perm = np.empty(mp, dtype=np.int32)
    width = np.empty(mp // C, dtype=np.int32)
    sptr = np.empty(mp // C + 1, dtype=np.int64)
    lib().oracle_sell_layout(m, prp, C, sigma, perm.ctypes.data, width.ctypes.data, sptr.ctypes.data)
    return perm, width, sptr


def to_sell(m, rowptr, colidx, val, sigma, C=SELL_C):
    """SELL-C-sigma arrays: (perm, width, slice_ptr, col, val)."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v = np.ascontiguousarray(val)
    perm, width, sptr = sell_layout(m, rp, sigma, C)
    slots = int(sptr[-1])
    col = np.empty(slots, dtype=np.int32)
    out = np.empty(slots, dtype=v.dtype)
    lib().oracle_to_sell(m, prp, pci, v.ctypes.data, v.itemsize, C, perm.ctypes.data, width.ctypes.data,
                         sptr.ctypes.data, col.ctypes.data, out.ctypes.data)
    return perm, width, sptr, col, out


def to_bcsr(m, n, rowptr, colidx, val, b):
    """BCSR with b x b blocks: (browptr[ceil(M/b)+1], bcol[nb], bval[nb*b*b])."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v = np.ascontiguousarray(val)
    mb = (m + b - 1) // b
    brp = np.empty(mb + 1, dtype=np.int32)
    nb = int(lib().oracle_to_bcsr(m, n, prp, pci, None, v.itemsize, b, brp.ctypes.data, None, None))
    bcol = np.empty(nb, dtype=np.int32)
    bval = np.empty(nb * b * b, dtype=v.dtype)
    lib().oracle_to_bcsr(m, n, prp, pci, v.ctypes.data, v.itemsize, b, brp.ctypes.data, bcol.ctypes.data,
                         bval.ctypes.data)
    return brp, bcol, bval


def bcsr_choose(m, n, rowptr, colidx, elem_size):
    """(b, nblocks) for the b in {2, 4, 8} with the fewest BCSR bytes."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    nb = np.zeros(1, dtype=np.int64)
    b = int(lib().oracle_bcsr_choose(m, n, prp, pci, elem_size, nb.ctypes.data))
    return b, int(nb[0])


def split_rows(m, rowptr, colidx, val, L=256, CK=4096):
    """SPLIT layout: long rows (>= L entries) in chunks of <= CK entries, a COO
    of the short rows' entries, the empty rows.  Returns a dict of arrays."""
    rp, prp = _c(rowptr, np.int32)
    ci, pci = _c(colidx, np.int32)
    v = np.ascontiguousarray(val)
    cnt = np.zeros(4, dtype=np.int64)
    lib().oracle_split(m, prp, pci, v.ctypes.data, v.itemsize, L, CK, None, None, None, None, None, None, None, None,
                       cnt.ctypes.data)
    nl, nc, ns, ne = (int(c) for c in cnt)
    out = {"lrows": np.empty(nl, np.int32), "crow": np.empty(nc, np.int32), "cstart": np.empty(nc, np.int32),
           "cend": np.empty(nc, np.int32), "srow": np.empty(ns, np.int32), "scol": np.empty(ns, np.int32),
           "sval": np.empty(ns, v.dtype), "empty": np.empty(ne, np.int32)}
    lib().oracle_split(m, prp, pci, v.ctypes.data, v.itemsize, L, CK, *(out[k].ctypes.data for k in
                       ("lrows", "crow", "cstart", "cend", "srow", "scol", "sval", "empty")), cnt.ctypes.data)
    return out


# ---------------------------------------------------------------------------
# Value storage precision
# ---------------------------------------------------------------------------

def round_bf16(x) -> np.ndarray:
    """FP64 -> bfloat16 bit patterns (uint16), round to nearest even."""
    xx, px = _c(x, np.float64)
    out = np.empty(xx.shape, dtype=np.uint16)
    lib().oracle_round_bf16(xx.size, px, out.ctypes.data)
    return out


def bf16_to_double(b) -> np.ndarray:
    bb, pb = _c(b, np.uint16)
    out = np.empty(bb.shape, dtype=np.float64)
    lib().oracle_bf16_to_double(bb.size, pb, out.ctypes.data)
    return out


# ---------------------------------------------------------------------------
# MLP selector (Sec. 5 replacement) and its optimizer
# ---------------------------------------------------------------------------

def mlp_param_count() -> int:
    return int(lib().oracle_mlp_param_count())


def mlp_forward(params, X) -> np.ndarray:
    p, pp = _c(params, np.float64)
    x, px = _c(X, np.float64)
    B = x.shape[0]
    out = np.empty((B, MLP_OUT), dtype=np.float64)
    lib().oracle_mlp_forward(pp, B, px, out.ctypes.data)
    return out


def mlp_loss_grad(params, X, T):
    p, pp = _c(params, np.float64)
    x, px = _c(X, np.float64)
    t, pt = _c(T, np.float64)
    g = np.empty_like(p)
    loss = lib().oracle_mlp_loss_grad(pp, x.shape[0], px, pt, g.ctypes.data)
    return float(loss), g


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays p, m, v given gradient g."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg, pg = _c(g, np.float64)
    lib().oracle_adam(p.size, p.ctypes.data, pg, m.ctypes.data, v.ctypes.data, int(t), lr, b1, b2, eps)


# ---------------------------------------------------------------------------
# Admissible formats and the paper's rule set (Sec. 2.3, Sec. 4, Sec. 6)
# ---------------------------------------------------------------------------

#: the eight classes a format is chosen from, in the order of their ids
CLASSES = ("csr_scalar", "csr_vec4", "csr_vec8", "csr_vec32", "csr_merge", "ell", "dia", "coo")


# Reading: the paper bounds the diagonals only through the 20x fill rule; a
# GPU DIA product keeps its offsets in on-chip memory, and this build's reading
# caps them at 8192 (32 KB of int32 offsets) however the fill rule falls.
DIA_MAX_OFFSETS = 8192


def admissible(m, nnz, max_rd, ndiags, value_bytes, fill_ratio_max=20, bytes_cap=4.0,
               dia_max_offsets=DIA_MAX_OFFSETS) -> int:
    """Bit mask over CLASSES (bit c set = class c may be used).

    CSR, in every kernel, and COO store only the entries: always admissible.
    Sec. 2.3 keeps the zero-filling formats only while the slots they store
    are at most 20 times the entries (one stored slot in twenty at least is an
    entry): ELL while max_RD * M <= 20 NNZ, DIA while Ndiags * M <= 20 NNZ,
    both tested in integers.  Besides, their arrays, padded to the pitch P =
    roundup(M, 32) rows, may move at most ``bytes_cap`` times the bytes of the
    CSR arrays (values, int32 columns, int32 row pointers):
      ELL  (value_bytes + 4) * max_RD * P
      DIA  value_bytes * Ndiags * P + 4 * Ndiags   (values plus the offsets)
    and DIA takes at most ``dia_max_offsets`` diagonals (8192 by default), a
    reading stated beside DIA_MAX_OFFSETS: the paper sets no such number.
    """
    mask = 0
    for c in ("csr_scalar", "csr_vec4", "csr_vec8", "csr_vec32", "csr_merge", "coo"):
        mask |= 1 << CLASSES.index(c)
    P = pitch(m)
    csr_bytes = max((value_bytes + 4) * nnz + 4 * (m + 1), 1)
    if m > 0 and max_rd > 0 and max_rd * m <= fill_ratio_max * nnz and \
            (value_bytes + 4) * max_rd * P <= bytes_cap * csr_bytes:
        mask |= 1 << CLASSES.index("ell")
    if m > 0 and 0 < ndiags <= dia_max_offsets and ndiags * m <= fill_ratio_max * nnz and \
            value_bytes * ndiags * P + 4 * ndiags <= bytes_cap * csr_bytes:
        mask |= 1 << CLASSES.index("dia")
    return mask


def rules_select(f, mask) -> int:
    """The format the observations of Sec. 4 choose, tried in the order Sec. 6
    gives the rule subsets (DIA, ELL, then CSR and COO); returns a class id.

    ``f`` holds the features of ``features()`` (aver_rd, max_rd, var_rd,
    ndiags, er_dia, er_ell, ntdiags_ratio, r, r_valid); ``mask`` is
    ``admissible()``.  Readings:
      DIA  at most 500 diagonals (few matrices gain beyond), and any of: fewer
           than 25 diagonals, ER_DIA above 60 %, NTdiags_ratio above 40 %;
      ELL  max_RD below 5 or ER_ELL above 90 %, and var_RD below 0.5 in
           either case;
      CSR or COO: the observations give no CSR rule, so R decides between
           them: a row-degree histogram fitted by a power law with R in
           [1, 4) marks a small-world matrix, stored as COO; otherwise CSR,
           whose GPU kernel is CSR-vector with the lane count that fits the
           mean row length (4 below 8 entries, 8 below 24, else 32).
    A rule whose format is not admissible does not fire; when none fires and
    the CSR-vector width is not admissible either, the lowest admissible id
    is the pick (ValueError when no class is admissible)."""
    def ok(name):
        return (mask >> CLASSES.index(name)) & 1

    nd = f["ndiags"]
    if ok("dia") and nd <= 500 and (nd < 25 or f["er_dia"] > 0.6 or f["ntdiags_ratio"] > 0.4):
        return CLASSES.index("dia")
    if ok("ell") and (f["max_rd"] < 5 or f["er_ell"] > 0.9) and f["var_rd"] < 0.5:
        return CLASSES.index("ell")
    if ok("coo") and f["r_valid"] and 1.0 <= f["r"] < 4.0:
        return CLASSES.index("coo")
    lanes = "csr_vec4" if f["aver_rd"] < 8.0 else ("csr_vec8" if f["aver_rd"] < 24.0 else "csr_vec32")
    if ok(lanes):
        return CLASSES.index(lanes)
    live = [c for c in range(len(CLASSES)) if (mask >> c) & 1]
    if not live:
        raise ValueError("no admissible class")   # the library refuses to tune then
    return live[0]


# ---------------------------------------------------------------------------
# The learned selector's decision (replacing the ruleset search of Sec. 6)
# ---------------------------------------------------------------------------

def selector_inputs(f) -> np.ndarray:
    """The 12 network inputs from the features of Table "Feature parameters"
    (Sec. 4) plus N and aver_RD, in FP64: log(1 + v) of M, N, NNZ, aver_RD,
    max_RD, min_RD, var_RD and Ndiags (counts spanning decades), then
    NTdiags_ratio, ER_DIA and ER_ELL as they are (already in [0, 1]), then R,
    limited to [-100, 100], or 0 when the fit is undefined (``r_valid`` 0)."""
    logs = [f[k] for k in ("m", "n", "nnz", "aver_rd", "max_rd", "min_rd", "var_rd", "ndiags")]
    r = min(100.0, max(-100.0, f["r"])) if f["r_valid"] else 0.0
    return np.array([np.log1p(float(v)) for v in logs] + [f["ntdiags_ratio"], f["er_dia"], f["er_ell"], r])


def learned_select(f, mask, params, mean, std):
    """(class id, probabilities over CLASSES): the inputs standardised by the
    model's mean and standard deviation (a deviation of 0 leaves the input
    unscaled), the network's logits, a softmax over the admissible classes
    only (others get probability 0), and the most probable class (the lowest
    id among equals; with no admissible class, all probabilities are 0 and
    the id is 0, a case the library refuses).  FP64 throughout."""
    x = selector_inputs(f)
    sd = np.where(np.asarray(std, np.float64) > 0, np.asarray(std, np.float64), 1.0)
    xs = (x - np.asarray(mean, np.float64)) / sd
    z = mlp_forward(np.asarray(params, np.float64), xs.reshape(1, -1))[0]
    live = np.array([(mask >> c) & 1 for c in range(len(CLASSES))], dtype=bool)
    p = np.zeros(len(CLASSES))
    if live.any():
        e = np.exp(z[live] - z[live].max())
        p[live] = e / e.sum()
    best = int(np.argmax(np.where(live, p, -1.0)))
    return best, p
