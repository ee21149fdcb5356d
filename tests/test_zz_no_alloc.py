"""The allocation-free merge-path product, for callers that cannot allocate
device memory (a memory manager owns it, allocation may synchronise the
device, or allocation is forbidden inside a time-critical loop).

It is called through the C ABI and compared with the handle-based merge-path
product and with the oracle on the same inputs, within the per-row bars the
parity tests use, on two calls in a row over matrices of different sizes: a
larger matrix then a smaller one (fewer tiles: the second call must not read
carries or tile coordinates the first call left in the shared array), and the
reverse.  alpha == 0 must give y = beta*y without reading x, as smat_spmv
does.  This file sorts last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

LARGE = lambda: synth.powerlaw(60000, 1.8, 5000, 11)   # ~430 tiles
SMALL = lambda: synth.stencil3d7(8)                    # 2 tiles


def _scalar(dtype, v):
    return ctypes.c_double(v) if dtype == "f64" else ctypes.c_float(v)


def _noalloc(A, rp, ci, vv, dtype, alpha, xd, beta, yd):
    a, b = _scalar(dtype, alpha), _scalar(dtype, beta)
    # any device allocation inside the call would now fail
    smat.lib().smat_test_fail_alloc_after(1)
    try:
        st = smat.smat_spmv_csr_merge_noalloc(A.m, A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), vv.data_ptr(),
                                              smat.DTYPES[dtype], ctypes.addressof(a), xd.data_ptr(),
                                              ctypes.addressof(b), yd.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    finally:
        smat.lib().smat_test_fail_alloc_after(0)
    assert st == smat.SMAT_OK, smat.smat_status_string(st)


def _device_csr(A, dtype):
    vals, vals64 = stored_values(A, dtype)
    if dtype == "bf16":
        vals = vals.view(np.int16)
    return (torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
            torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), vals64)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("order", [(LARGE, SMALL), (SMALL, LARGE)], ids=["large_then_small", "small_then_large"])
def test_noalloc_matches_handle_path_twice(dtype, order):
    np_t = np.float64 if dtype == "f64" else np.float32
    for call, (maker, alpha, beta, seed) in enumerate([(order[0], 1.0, 0.0, 0), (order[1], -0.5, 2.0, 1)]):
        A = maker()
        rp, ci, vv, vals64 = _device_csr(A, dtype)
        M = smat.SpMatrix(A.m, A.n, rp, ci, vv, dtype)
        x = synth.uniform(seed, 1, A.n).astype(np_t)
        y0 = synth.uniform(seed, 2, A.m).astype(np_t)
        xd = torch.from_numpy(x).to(DEV)
        y_ref = M.spmv(xd, torch.from_numpy(y0.copy()).to(DEV), alpha, beta, variant=smat.SMAT_V_CSR_MERGE)
        y_new = torch.from_numpy(y0.copy()).to(DEV)
        _noalloc(A, rp, ci, vv, dtype, alpha, xd, beta, y_new)
        torch.cuda.synchronize()
        got = y_new.cpu().numpy().astype(np.float64)
        want = y_ref.cpu().numpy().astype(np.float64)
        ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
        assert_close_rows(got, want, scale, TOL[dtype], f"call {call} ({A.name}): no-alloc vs handle path")
        assert_close_rows(got, ref, scale, TOL[dtype], f"call {call} ({A.name}): no-alloc vs oracle")
        M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_noalloc_alpha_zero_reads_neither_a_nor_x(dtype):
    # NaN and Inf in x must not reach y when alpha == 0: y = beta*y, one
    # rounding per row, and exactly 0 when beta == 0 (NaN in y ignored)
    A = SMALL()
    rp, ci, vv, _ = _device_csr(A, dtype)
    np_t = np.float64 if dtype == "f64" else np.float32
    x = synth.uniform(3, 1, A.n).astype(np_t)
    x[::7] = np.nan
    x[3::11] = np.inf
    xd = torch.from_numpy(x).to(DEV)
    y0 = synth.uniform(3, 2, A.m).astype(np_t)
    beta = -1.5
    y = torch.from_numpy(y0.copy()).to(DEV)
    _noalloc(A, rp, ci, vv, dtype, 0.0, xd, beta, y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), np_t(beta) * y0)
    y0[::5] = np.nan
    y = torch.from_numpy(y0.copy()).to(DEV)
    _noalloc(A, rp, ci, vv, dtype, 0.0, xd, 0.0, y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), np.zeros(A.m, np_t))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # the size check comes before any use of the pointers, which are never
    # dereferenced here
    a, b = ctypes.c_double(1.0), ctypes.c_double(0.0)
    m, nnz = 1 << 20, (1 << 27)  # ceil((m + nnz) / 2048) > 65536 tiles
    st = smat.smat_spmv_csr_merge_noalloc(m, m, nnz, 16, 16, 16, smat.SMAT_F64, ctypes.addressof(a), 16,
                                          ctypes.addressof(b), 16, 0)
    assert st == smat.SMAT_ERR_UNSUPPORTED
