"""Pins of the oracle's format conversions (Sec. 2.1: DIA, ELL, COO from CSR)
and of its bfloat16 rounding."""
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth

MAKERS = [lambda: synth.stencil2d5(9, 7), lambda: synth.uniform_random(150, 4.0, 1),
          lambda: synth.powerlaw(200, 1.8, 60, 2), lambda: synth.blockdiag(53, 4, 3),
          lambda: synth.stencil3d27(4)]


@pytest.mark.parametrize("mk", MAKERS)
def test_ell_reconstructs_dense(mk):
    A = mk()
    col, val, K, P = oracle.to_ell(A.m, A.rowptr, A.colidx, A.val)
    assert K == np.diff(A.rowptr).max() and P % 32 == 0 and P >= A.m
    col, val = col.reshape(K, P), val.reshape(K, P)
    d = np.zeros((A.m, A.n))
    for s in range(K):
        for i in range(P):
            if col[s, i] >= 0:
                assert i < A.m
                d[i, col[s, i]] += val[s, i]
            else:
                assert val[s, i].view(np.uint64) == 0  # +0.0 pads
    assert np.array_equal(d, A.todense())
    rl = np.diff(A.rowptr)
    for i in range(A.m):  # pads only after the row's entries
        assert np.all(col[:rl[i], i] >= 0) and np.all(col[rl[i]:, i] == -1)


@pytest.mark.parametrize("mk", MAKERS)
def test_dia_reconstructs_dense(mk):
    A = mk()
    off, val, P = oracle.to_dia(A.m, A.n, A.rowptr, A.colidx, A.val)
    dense = A.todense()
    nz_off = sorted({j - i for i, j in zip(*np.nonzero(dense))})
    assert list(off) == nz_off
    val = val.reshape(len(off), P)
    rec = np.zeros_like(dense)
    for t, o in enumerate(off):
        for i in range(P):
            j = i + o
            if i < A.m and 0 <= j < A.n:
                rec[i, j] = val[t, i]
            else:
                assert val[t, i].view(np.uint64) == 0
    assert np.array_equal(rec, dense)


@pytest.mark.parametrize("mk", MAKERS)
def test_coo_rows(mk):
    A = mk()
    assert np.array_equal(oracle.to_coo(A.m, A.rowptr), A.row_of_nnz().astype(np.int32))


def test_conversions_copy_narrow_values_bitwise():
    A = synth.uniform_random(100, 5.0, 4)
    v32 = A.val.astype(np.float32)
    col, val, K, P = oracle.to_ell(A.m, A.rowptr, A.colidx, v32)
    assert val.dtype == np.float32
    c64, val64, _, _ = oracle.to_ell(A.m, A.rowptr, A.colidx, A.val)
    assert np.array_equal(val, val64.astype(np.float32))
    b16 = oracle.round_bf16(A.val)
    off, dv, P = oracle.to_dia(A.m, A.n, A.rowptr, A.colidx, b16)
    off2, dv64, _ = oracle.to_dia(A.m, A.n, A.rowptr, A.colidx, oracle.bf16_to_double(b16))
    assert np.array_equal(oracle.bf16_to_double(dv), dv64)


# ---------------------------------------------------------------------------
# bfloat16 round-to-nearest-even against exact rational arithmetic
# ---------------------------------------------------------------------------

def _bf16_grid_value(bits):
    return oracle.bf16_to_double(np.array([bits], np.uint16))[0]


def _rne_bf16_exact(x: float) -> int:
    """Nearest bfloat16 by exact comparison with its two neighbours."""
    if x == 0:
        return 0x8000 if struct.pack(">d", x)[0] & 0x80 else 0
    neg = x < 0
    a = abs(x)
    fx = Fraction(a)
    # largest non-negative finite pattern <= a
    lo = 0
    for bit in range(14, -1, -1):
        cand = lo | (1 << bit)
        if cand <= 0x7F7F and Fraction(_bf16_grid_value(cand)) <= fx:
            lo = cand
    if lo == 0x7F7F:
        top = Fraction(2) ** 128  # the next step would be 2^128 -> overflow
        mid = (Fraction(_bf16_grid_value(0x7F7F)) + top) / 2
        r = 0x7F80 if fx >= mid else 0x7F7F
    else:
        vlo, vhi = Fraction(_bf16_grid_value(lo)), Fraction(_bf16_grid_value(lo + 1))
        dl, dh = fx - vlo, vhi - fx
        r = lo if dl < dh else lo + 1 if dh < dl else (lo if lo % 2 == 0 else lo + 1)
    return r | (0x8000 if neg else 0)


def test_bf16_rounding_against_exact():
    rng = np.random.default_rng(0)
    xs = list(rng.standard_normal(300))
    xs += list(rng.standard_normal(100) * 1e-39)   # bfloat16 subnormal range
    xs += list(rng.standard_normal(50) * 1e38)     # near overflow
    # exact ties between neighbours, both parities, and one ulp around them
    for bits in [0x3F80, 0x3F81, 0x4049, 0x0001, 0x0002, 0x007F, 0x0080, 0x7F7E, 0x7F7F]:
        a = Fraction(_bf16_grid_value(bits))
        b = Fraction(_bf16_grid_value(bits + 1)) if bits < 0x7F7F else Fraction(2) ** 128
        mid = float((a + b) / 2)
        xs += [mid, np.nextafter(mid, 0), np.nextafter(mid, np.inf), -mid]
    xs += [3.3895313892515355e38, 3.4e38, 1e300, -1e300, 5e-324, -5e-324, 0.0, -0.0, 1.0, -2.0]
    got = oracle.round_bf16(np.array(xs))
    for x, g in zip(xs, got):
        assert int(g) == _rne_bf16_exact(float(x)), (x, hex(int(g)))


def test_bf16_specials():
    got = oracle.round_bf16(np.array([np.inf, -np.inf, np.nan]))
    assert got[0] == 0x7F80 and got[1] == 0xFF80 and (got[2] & 0x7F80) == 0x7F80 and (got[2] & 0x7F)


def test_bf16_overflow_boundary():
    # the largest finite bfloat16 is (2 - 2^-7) 2^127 (0x7F7F); the halfway
    # point to 2^128, (2 - 2^-8) 2^127, ties to the even neighbour, which is
    # 2^128 and therefore +inf; anything in [2^128, 2^129) is +inf too
    top = (2.0 - 2.0 ** -7) * 2.0 ** 127
    half = (2.0 - 2.0 ** -8) * 2.0 ** 127
    got = oracle.round_bf16(np.array([top, np.nextafter(half, 0.0), half, 2.0 ** 128, 1.5 * 2.0 ** 128,
                                      -1.5 * 2.0 ** 128]))
    assert got.tolist() == [0x7F7F, 0x7F7F, 0x7F80, 0x7F80, 0x7F80, 0xFF80]
