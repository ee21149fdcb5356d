"""The allocation-free merge-path product, for callers that cannot allocate
device memory (a memory manager owns it, allocation may synchronise the
device, or allocation is forbidden inside a time-critical loop).

It is called through the C ABI and compared with the handle-based merge-path
product on the same inputs, within the per-row bars the parity tests use, on
two calls in a row (the second call must not see the first call's carries).
This file sorts last so that a failure here never hides another test.
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


def _scalar(dtype, v):
    return ctypes.c_double(v) if dtype == "f64" else ctypes.c_float(v)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("maker", [lambda: synth.powerlaw(60000, 1.8, 5000, 11),
                                   lambda: synth.stencil3d7(24)])
def test_noalloc_matches_handle_path_twice(dtype, maker):
    A = maker()
    vals, vals64 = stored_values(A, dtype)
    if dtype == "bf16":
        vals = vals.view(np.int16)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    rp = torch.from_numpy(A.rowptr).to(DEV)
    ci = torch.from_numpy(A.colidx).to(DEV)
    vv = torch.from_numpy(np.ascontiguousarray(vals)).to(DEV)
    M = smat.SpMatrix(A.m, A.n, rp, ci, vv, dtype)
    for call, (alpha, beta, seed) in enumerate([(1.0, 0.0, 0), (-0.5, 2.0, 1)]):
        x = synth.uniform(seed, 1, A.n).astype(np.float64 if dtype == "f64" else np.float32)
        y0 = synth.uniform(seed, 2, A.m).astype(np.float64 if dtype == "f64" else np.float32)
        xd = torch.from_numpy(x).to(DEV)
        y_ref = M.spmv(xd, torch.from_numpy(y0.copy()).to(DEV), alpha, beta, variant=smat.SMAT_V_CSR_MERGE)
        y_new = torch.from_numpy(y0.copy()).to(DEV)
        a, b = _scalar(dtype, alpha), _scalar(dtype, beta)
        # any device allocation inside the call would now fail
        smat.lib().smat_test_fail_alloc_after(1)
        try:
            st = smat.smat_spmv_csr_merge_noalloc(A.m, A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), vv.data_ptr(),
                                                  smat.DTYPES[dtype], ctypes.addressof(a), xd.data_ptr(),
                                                  ctypes.addressof(b), y_new.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream)
        finally:
            smat.lib().smat_test_fail_alloc_after(0)
        assert st == smat.SMAT_OK, smat.smat_status_string(st)
        torch.cuda.synchronize()
        got = y_new.cpu().numpy().astype(np.float64)
        want = y_ref.cpu().numpy().astype(np.float64)
        ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
        assert_close_rows(got, want, scale, TOL[dtype], f"call {call}: no-alloc vs handle path")
        assert_close_rows(got, ref, scale, TOL[dtype], f"call {call}: no-alloc vs oracle")
    M.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    a, b = ctypes.c_double(1.0), ctypes.c_double(0.0)
    m, nnz = 1 << 20, (1 << 27)  # ceil((m + nnz) / 2048) > 65536 tiles
    st = smat.smat_spmv_csr_merge_noalloc(m, m, nnz, 16, 16, 16, smat.SMAT_F64, ctypes.addressof(a), 16,
                                          ctypes.addressof(b), 16, 0)
    assert st == smat.SMAT_ERR_UNSUPPORTED
