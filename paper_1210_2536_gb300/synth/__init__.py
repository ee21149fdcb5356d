"""Seeded synthetic sparse matrices (inputs only).

The generators stand in for the structure classes of the sparse-matrix
collection the paper trains and tests on (arXiv 1210.2536, Sec. 2.2 and the
table of application areas): PDE stencils, uniform random graphs, power-law
(small-world) graphs and dense block structure.  None of the auto-tuning
method's arithmetic lives here, so the oracle and the CUDA library can both be
fed from this module.  The C side (``synth.c``) draws every random number from
Philox4x32-10 (Salmon et al., SC'11) keyed by (seed, row, purpose, index).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsmatsynth.so")

STENCIL2D5, STENCIL3D7, STENCIL3D27, UNIFORM, POWERLAW, BLOCKDIAG, BOX3D = range(7)
KIND_NAMES = ["stencil2d5", "stencil3d7", "stencil3d27", "uniform", "powerlaw", "blockdiag", "box3d"]


def build(force: bool = False) -> str:
    """Compile ``libsmatsynth.so`` beside its source (plain C, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                               "-o", tmp, _SRC, "-lm", "-pthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.synth_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.synth_dims.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_int64)]
        L.synth_dims.restype = ctypes.c_int64
        L.synth_rowlen.argtypes = [ctypes.c_int, P(ctypes.c_double), ctypes.c_uint64, ctypes.c_void_p,
                                   ctypes.c_int]
        L.synth_fill.argtypes = [ctypes.c_int, P(ctypes.c_double), ctypes.c_uint64, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_void_p]
        L.synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p]
        L.synth_zipf_mean.argtypes = [ctypes.c_double, ctypes.c_int64]
        L.synth_zipf_mean.restype = ctypes.c_double
        _lib = L
    return _lib


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: 4 counter words and 2 key words -> 4 words."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().synth_philox4x32_10(c, k, o)
    return [int(v) for v in o]


@dataclass
class CSR:
    """A CSR matrix on the host: int32 rowptr[M+1], int32 colidx[NNZ], float64 val[NNZ]."""

    m: int
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if self.m > 0 else 0

    def row_of_nnz(self) -> np.ndarray:
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.rowptr.astype(np.int64)))

    def todense(self) -> np.ndarray:
        d = np.zeros((self.m, self.n), dtype=np.float64)
        d[self.row_of_nnz(), self.colidx.astype(np.int64)] = self.val
        return d


def generate(kind: int, params, seed: int = 0, nthreads: int = 0, name: str = "") -> CSR:
    """Build one matrix of the given kind (see ``synth.c`` for the parameters)."""
    L = lib()
    p = (ctypes.c_double * 4)(*(list(map(float, params)) + [0.0] * (4 - len(params))))
    nr, nc = ctypes.c_int64(), ctypes.c_int64()
    if L.synth_dims(kind, p, ctypes.byref(nr), ctypes.byref(nc)) < 0:
        raise ValueError(f"bad generator kind {kind}")
    m, n = nr.value, nc.value
    rowlen = np.empty(m, dtype=np.int32)
    if L.synth_rowlen(kind, p, seed, rowlen.ctypes.data, nthreads) != 0:
        raise MemoryError("synth_rowlen failed")
    rp64 = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(rowlen, out=rp64[1:])
    nnz = int(rp64[-1])
    if nnz > 2**31 - 1:
        raise ValueError(f"nnz {nnz} exceeds int32 indexing")
    colidx = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    if L.synth_fill(kind, p, seed, rp64.ctypes.data, colidx.ctypes.data, val.ctypes.data, nthreads) != 0:
        raise MemoryError("synth_fill failed")
    return CSR(m, n, rp64.astype(np.int32), colidx, val, name or KIND_NAMES[kind])


def uniform(seed: int, stream: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n values uniform on [lo, hi) (the x vectors of the workloads: U[-1,1], seed 0)."""
    out = np.empty(n, dtype=np.float64)
    lib().synth_uniform(seed, stream, n, lo, hi, out.ctypes.data)
    return out


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    lib().synth_normal(seed, stream, n, out.ctypes.data)
    return out


def zipf_mean(alpha: float, kmax: int) -> float:
    return float(lib().synth_zipf_mean(alpha, kmax))


# ---------------------------------------------------------------------------
# Named builders
# ---------------------------------------------------------------------------

def stencil2d5(mx: int, my: int | None = None) -> CSR:
    my = mx if my is None else my
    return generate(STENCIL2D5, [mx, my], 0, name=f"stencil2d5_{mx}x{my}")


def stencil3d7(m: int) -> CSR:
    return generate(STENCIL3D7, [m], 0, name=f"stencil3d7_{m}^3")


def stencil3d27(m: int) -> CSR:
    return generate(STENCIL3D27, [m], 0, name=f"stencil3d27_{m}^3")


def uniform_random(n: int, lam: float = 16.0, seed: int = 0) -> CSR:
    return generate(UNIFORM, [n, lam], seed, name=f"uniform_{n}_poisson{lam:g}")


def powerlaw(n: int, alpha: float = 1.8, kmax: int = 10000, seed: int = 0) -> CSR:
    return generate(POWERLAW, [n, alpha, kmax], seed, name=f"powerlaw_{n}_zipf{alpha:g}_cap{kmax}")


def blockdiag(n: int, b: int = 8, seed: int = 0) -> CSR:
    return generate(BLOCKDIAG, [n, b], seed, name=f"blockdiag_{n}_b{b}")


def box3d(m: int, r: int = 2) -> CSR:
    """The (2r+1)^3-point box stencil on an m^3 grid (r = 1: the 27-point
    stencil), rows truncated at the grid's boundary: the shape of the Galerkin
    operators on coarse multigrid levels, whose stencils widen level by level."""
    return generate(BOX3D, [m, r], 0, name=f"box3d_{m}^3_r{r}")


# ---------------------------------------------------------------------------
# Workload recipes (sizes of the paper-shaped synthetic workloads)
# ---------------------------------------------------------------------------

def poisson_2d_64() -> CSR:
    """2-D 5-point Laplacian on a 64x64 grid: n = 4096, nnz = 20224."""
    return stencil2d5(64, 64)


def structures_suite(scale: float = 1.0, seed: int = 0):
    """The four structure classes at full size (scale = 1):
    3-D 7-point 128^3; uniform random n = 1e6 with Poisson(16) rows;
    power-law n = 2e6 with Zipf(1.8) rows capped at 1e4; 8x8 block diagonal n = 1e6.
    ``scale`` shrinks the row counts for small test cases."""
    m3 = max(4, int(round(128 * scale ** (1.0 / 3.0))))
    return [
        stencil3d7(m3),
        uniform_random(max(64, int(1_000_000 * scale)), 16.0, seed),
        powerlaw(max(64, int(2_000_000 * scale)), 1.8, 10000, seed),
        blockdiag(max(64, int(1_000_000 * scale)), 8, seed),
    ]


def _meta_uniforms(matrix_id: int, count: int) -> np.ndarray:
    return uniform(0x5EED0000 + matrix_id, 7, count, 0.0, 1.0)


# The labelled set: matrices 0 .. DATASET_PRIMARY-1 over the six structure
# classes above, then DATASET_SIZE - DATASET_PRIMARY box stencils, which cover
# the banded operators with hundreds to thousands of entries per row on small
# grids that coarse multigrid levels produce (none of the six classes has
# that shape, and a selector trained without it mispicks there).
DATASET_PRIMARY = 2000
DATASET_SIZE = 2400


def dataset_spec(matrix_id: int, n_lo: float = 1e3, n_hi: float = 4e6, nnz_lo: float = 1e4,
                 nnz_hi: float = 5e7):
    """Generator kind and parameters of matrix ``matrix_id`` of the labelled
    training/held-out set.  Below DATASET_PRIMARY the kind is uniform over the
    six structures (block diagonal with b in {2,4,8,16}), n log-uniform on
    [n_lo, n_hi] and the target nnz log-uniform on [nnz_lo, nnz_hi], clipped to
    what the kind can realise at that n.  From DATASET_PRIMARY on: box stencils
    of radius r uniform in 2..6 on m^3 grids, n = m^3 log-uniform on
    [512, min(n_hi, nnz_hi / (2r+1)^3)].  Returns (kind, params, seed)."""
    u = _meta_uniforms(matrix_id, 4)
    if matrix_id >= DATASET_PRIMARY:
        r = 2 + min(4, int(u[0] * 5))
        hi = min(n_hi, nnz_hi / float((2 * r + 1) ** 3))
        n = math.exp(math.log(512.0) + u[1] * (math.log(hi) - math.log(512.0)))
        return BOX3D, [max(8, int(round(n ** (1.0 / 3.0)))), r], matrix_id
    kind = min(5, int(u[0] * 6))
    n = int(round(math.exp(math.log(n_lo) + u[1] * (math.log(n_hi) - math.log(n_lo)))))
    target = math.exp(math.log(nnz_lo) + u[2] * (math.log(nnz_hi) - math.log(nnz_lo)))
    seed = matrix_id
    if kind == STENCIL2D5:
        mx = max(2, int(round(math.sqrt(n))))
        return kind, [mx, mx], seed
    if kind in (STENCIL3D7, STENCIL3D27):
        m = max(2, int(round(n ** (1.0 / 3.0))))
        return kind, [m], seed
    if kind == UNIFORM:
        lam = min(max(target / n, 1.0), n / 4.0, 2000.0)
        return kind, [n, lam], seed
    if kind == POWERLAW:
        kmax = min(10000, n)
        want = min(max(target / n, 1.2), kmax / 3.0)
        lo, hi = 0.3, 4.0  # mean decreases in alpha
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            if zipf_mean(mid, kmax) > want:
                lo = mid
            else:
                hi = mid
        return kind, [n, 0.5 * (lo + hi), kmax], seed
    b = [2, 4, 8, 16][min(3, int(u[3] * 4))]
    return kind, [n, b], seed


def dataset_matrix(matrix_id: int, nthreads: int = 0, **kw) -> CSR:
    kind, params, seed = dataset_spec(matrix_id, **kw)
    return generate(kind, params, seed, nthreads, name=f"ds{matrix_id}_{KIND_NAMES[kind]}")


def amg_like_hierarchy(top: int = 192):
    """27-point stencils on top^3, (top/2)^3, ... five levels (multigrid levels)."""
    return [stencil3d27(top >> lvl) for lvl in range(5)]


def stencil_over_powerlaw(m: int = 128, kmax: int = 10000, seed: int = 5) -> CSR:
    """The 3-D 7-point stencil on m^3 (banded) stacked over as many rows of a
    power-law graph (Zipf(1.8) rows, uniform columns) on the same m^3 columns:
    a matrix whose structure changes halfway down, the case per-segment
    formats are for."""
    top = stencil3d7(m)
    bot = powerlaw(top.n, 1.8, kmax, seed)
    rp = np.concatenate([top.rowptr[:-1].astype(np.int64), bot.rowptr.astype(np.int64) + top.nnz])
    return CSR(top.m + bot.m, top.n, rp.astype(np.int32), np.concatenate([top.colidx, bot.colidx]),
               np.concatenate([top.val, bot.val]), f"stencil3d7_{m}^3_over_powerlaw_cap{kmax}")


def aggregation_prolongator(m: int, A: CSR, omega: float = 2.0 / 3.0) -> "scipy.sparse.csr_matrix":
    """Smoothed-aggregation prolongator of an m x m x m grid operator A (points
    ordered x fastest): the tentative P0 maps each point to its 2 x 2 x 2 box
    aggregate ((x//2) + mc (y//2) + mc^2 (z//2), mc = ceil(m/2)) with weight 1,
    and one damped-Jacobi step smooths it: P = (I - omega D^-1 A) P0."""
    import scipy.sparse as sp
    mc = (m + 1) // 2
    i = np.arange(A.m, dtype=np.int64)
    x, y, z = i % m, (i // m) % m, i // (m * m)
    agg = (x // 2) + mc * (y // 2) + mc * mc * (z // 2)
    P0 = sp.csr_matrix((np.ones(A.m), (i, agg)), shape=(A.m, mc ** 3))
    As = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.m, A.n))
    dinv = 1.0 / As.diagonal()
    return (P0 - omega * sp.diags(dinv) @ (As @ P0)).tocsr()


def galerkin_hierarchy(m: int = 96, levels: int = 5, omega: float = 2.0 / 3.0):
    """An algebraic-multigrid hierarchy with Galerkin coarse operators: level 0
    is the 27-point operator (26 / -1) on m^3; level l+1 is P^T A_l P with the
    smoothed-aggregation prolongator of level l (``aggregation_prolongator``).
    Each coarse stencil is wider than the last (125 points on level 1 where
    the grid allows, then wider still), so the levels differ in structure the
    way the operators of an AMG solve do.  Host-side input generation
    (scipy.sparse products), FP64 values, canonical CSR."""
    import scipy.sparse as sp
    A = stencil3d27(m)
    out = [A]
    g = m
    for lvl in range(1, levels):
        if g < 2:
            break
        P = aggregation_prolongator(g, A, omega)
        As = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.m, A.n))
        Ac = (P.T.tocsr() @ (As @ P)).tocsr()
        Ac.sum_duplicates()
        Ac.sort_indices()
        g = (g + 1) // 2
        A = CSR(Ac.shape[0], Ac.shape[1], Ac.indptr.astype(np.int32), Ac.indices.astype(np.int32),
                Ac.data.astype(np.float64), f"galerkin_L{lvl}_{g}^3_from_27pt_{m}^3")
        out.append(A)
    return out


def mixed_batch(count: int = 64, n_lo: float = 1e3, n_hi: float = 1e6, base_seed: int = 0):
    """``count`` independent matrices, n log-uniform on [n_lo, n_hi], structure
    cycling through uniform random, power-law, block diagonal and 3-D 7-point."""
    out = []
    for i in range(count):
        u = uniform(0xBA7C0000 + base_seed + i, 3, 1, 0.0, 1.0)[0]
        n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
        c = i % 4
        if c == 0:
            out.append(uniform_random(n, 16.0, base_seed + i))
        elif c == 1:
            out.append(powerlaw(n, 1.8, min(10000, n), base_seed + i))
        elif c == 2:
            out.append(blockdiag(n, 8, base_seed + i))
        else:
            out.append(stencil3d7(max(2, int(round(n ** (1.0 / 3.0))))))
    return out
