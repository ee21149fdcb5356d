"""Pins of the oracle SpMV (Sec. 2.1 / Sec. 3) to facts other than itself:
dense products on tiny inputs, closed-form stencil actions, invariants."""
import math

import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR


def _from_dense(d):
    m, n = d.shape
    rows, cols = np.nonzero(d)
    rp = np.zeros(m + 1, dtype=np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return CSR(m, n, rp, cols.astype(np.int32), d[rows, cols].astype(np.float64))


def _spmv(A, x, alpha=1.0, beta=0.0, y=None, threads=1):
    return oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x, alpha, beta, y, threads)


@pytest.mark.parametrize("seed", range(8))
def test_integer_matrices_exact_against_dense(seed):
    # small integers: every partial sum is exact, so any order gives the same bits
    rng = np.random.default_rng(seed)
    m, n = rng.integers(1, 64, size=2)
    d = rng.integers(-9, 10, size=(m, n)).astype(np.float64)
    d[rng.random((m, n)) < 0.7] = 0.0
    A = _from_dense(d)
    x = rng.integers(-5, 6, size=n).astype(np.float64)
    y0 = rng.integers(-5, 6, size=m).astype(np.float64)
    assert np.array_equal(_spmv(A, x), d @ x)
    assert np.array_equal(_spmv(A, x, 2.0, -1.0, y0), 2.0 * (d @ x) - y0)


@pytest.mark.parametrize("seed", range(4))
def test_real_matrices_against_dense(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 57, 41
    d = rng.standard_normal((m, n))
    d[rng.random((m, n)) < 0.6] = 0.0
    A = _from_dense(d)
    x = rng.uniform(-1, 1, n)
    ref = d @ x
    bound = 64 * np.finfo(float).eps * (np.abs(d) @ np.abs(x))
    assert np.all(np.abs(_spmv(A, x) - ref) <= bound)


def test_row_sums_closed_form_5pt():
    # A*1 for the 4/-1 5-point operator: 0 inside, 1 on edges, 2 at corners
    A = synth.stencil2d5(64, 64)
    y = _spmv(A, np.ones(A.n)).reshape(64, 64)
    want = np.zeros((64, 64))
    want[0, :] += 1; want[-1, :] += 1; want[:, 0] += 1; want[:, -1] += 1
    assert np.array_equal(y, want)


def test_linear_field_is_harmonic_inside():
    A = synth.stencil2d5(30, 20)
    ix = np.tile(np.arange(30, dtype=np.float64), 20)
    y = _spmv(A, ix).reshape(20, 30)
    assert np.all(y[1:-1, 1:-1] == 0.0)


@pytest.mark.parametrize("a,b", [(1, 1), (3, 5), (17, 2)])
def test_eigenvector_action_2d(a, b):
    mx = my = 33
    h = math.pi / (mx + 1)
    X, Y = np.meshgrid(np.arange(1, mx + 1), np.arange(1, my + 1))
    v = (np.sin(a * X * h) * np.sin(b * Y * h)).ravel()
    lam = 4 - 2 * math.cos(a * h) - 2 * math.cos(b * h)
    y = _spmv(synth.stencil2d5(mx, my), v)
    assert np.max(np.abs(y - lam * v)) < 1e-13


def test_eigenvector_action_3d7():
    m = 12
    h = math.pi / (m + 1)
    g = np.arange(1, m + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    a, b, c = 2, 5, 7
    v = (np.sin(a * X * h) * np.sin(b * Y * h) * np.sin(c * Z * h)).ravel()
    lam = 6 - 2 * (math.cos(a * h) + math.cos(b * h) + math.cos(c * h))
    y = _spmv(synth.stencil3d7(m), v)
    assert np.max(np.abs(y - lam * v)) < 1e-13


def test_block_diagonal_equals_block_products():
    A = synth.blockdiag(45, 8, 2)
    x = synth.uniform(0, 9, A.n)
    y = _spmv(A, x)
    d = A.todense()
    for s in range(0, 45, 8):
        e = min(s + 8, 45)
        ref = d[s:e, s:e] @ x[s:e]
        assert np.all(np.abs(y[s:e] - ref) <= 16 * np.finfo(float).eps * (np.abs(d[s:e, s:e]) @ np.abs(x[s:e])))


def test_alpha_beta_semantics():
    A = synth.uniform_random(200, 5.0, 1)
    x = synth.uniform(0, 1, A.n)
    ax = _spmv(A, x)
    y_nan = np.full(A.m, np.nan)
    assert np.array_equal(_spmv(A, x, 1.0, 0.0, y_nan), ax)  # beta = 0: y never read
    y0 = synth.uniform(3, 1, A.m)
    assert np.array_equal(_spmv(A, x, 0.0, 2.5, y0), 2.5 * y0)
    both = _spmv(A, x, 2.0, -1.0, y0)
    assert np.array_equal(both, 2.0 * ax + (-1.0) * y0)  # separately rounded, as defined


def test_empty_matrix_and_empty_rows():
    A = CSR(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    y0 = np.arange(5, dtype=np.float64)
    assert np.array_equal(_spmv(A, np.ones(7), 1.0, 3.0, y0), 3.0 * y0)
    assert np.array_equal(_spmv(A, np.ones(7)), np.zeros(5))


def test_threaded_is_bitwise_serial_and_balanced():
    A = synth.powerlaw(30000, 1.8, 3000, 7)
    x = synth.uniform(0, 1, A.n)
    y0 = synth.uniform(1, 1, A.m)
    s = _spmv(A, x, 1.5, 0.5, y0)
    for t in (2, 3, 8):
        p = _spmv(A, x, 1.5, 0.5, y0, threads=t)
        assert np.array_equal(s.view(np.uint64), p.view(np.uint64))
    b = oracle.partition_rows(A.m, A.rowptr, 8)
    nnz_per = np.diff(A.rowptr.astype(np.int64)[b])
    assert nnz_per.sum() == A.nnz
    assert nnz_per.max() <= A.nnz / 8 + np.diff(A.rowptr).max()


def test_sampled_rows_match_full():
    A = synth.uniform_random(1000, 7.0, 2)
    x = synth.uniform(0, 1, A.n)
    y0 = synth.uniform(1, 1, A.m)
    full = _spmv(A, x, 1.25, -0.5, y0)
    rows = np.array([0, 5, 999, 500, 17])
    part = oracle.spmv_rows_sampled(A.rowptr, A.colidx, A.val, x, rows, 1.25, -0.5, y0)
    assert np.array_equal(full[rows], part)


def test_segment_starts_closed_forms():
    # constant rows: the balanced bounds are M t / k, already on 8-row multiples
    A = synth.blockdiag(4096, 8, 0)
    assert oracle.segment_starts(A.m, A.rowptr, 4) == [0, 1024, 2048, 3072, 4096]
    # bounds off the 8-row grid move down: 1000 rows of 5 entries, 3 parts ->
    # targets 1666, 3333 entries reached at rows 334, 667 -> 328, 664
    rp = np.arange(1001, dtype=np.int32) * 5
    assert oracle.segment_starts(1000, rp, 3) == [0, 328, 664, 1000]
    # every entry in the first row: each bound is row 1, moved down to 0 and dropped
    rp = np.array([0] + [100] * 50, dtype=np.int32)
    assert oracle.segment_starts(50, rp, 4) == [0, 50]
    # every entry in the last of 16 rows: each bound is row 16 = M, dropped
    rp = np.array([0] * 16 + [100], dtype=np.int32)
    assert oracle.segment_starts(16, rp, 4) == [0, 16]
    # fewer than 8 rows: one segment
    assert oracle.segment_starts(7, np.arange(8, dtype=np.int32), 3) == [0, 7]


def test_segment_starts_stay_within_eight_rows_of_balance():
    A = synth.powerlaw(50000, 1.8, 2000, 9)
    for k in (2, 3, 4, 7, 16):
        s = oracle.segment_starts(A.m, A.rowptr, k)
        assert s[0] == 0 and s[-1] == A.m and all(a < b for a, b in zip(s, s[1:]))
        assert all(r % 8 == 0 for r in s[:-1])
        for r in s[1:-1]:
            # some balanced bound t NNZ / k is first reached within the 8 rows from r
            hit = [t for t in range(1, k) if r <= np.searchsorted(A.rowptr, A.nnz * t // k) < r + 8]
            assert hit, (k, r)


def test_partition_bounds_round_targets_down():
    # one entry per row, 10 rows over 3 threads: the bounds are the first rows
    # whose start reaches floor(10 t / 3) = 3 and 6 entries
    assert oracle.partition_rows(10, np.arange(11, dtype=np.int32), 3).tolist() == [0, 3, 6, 10]
    # rows of 1, 5, 1, 1, 1, 1 entries (10 in all), 4 threads: targets 2, 5, 7
    # are first reached at rows 2 (start 6), 2 and 3 (start 7)
    rp = np.array([0, 1, 6, 7, 8, 9, 10], dtype=np.int32)
    assert oracle.partition_rows(6, rp, 4).tolist() == [0, 2, 2, 3, 6]
