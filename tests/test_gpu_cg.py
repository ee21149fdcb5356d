"""Mixed-precision CG: FP32/BF16 inner solves, FP64 residual and update.
The final residual is recomputed on the host by the oracle's FP64 SpMV."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def handles(A, inner="f32", tune=True):
    def mk(dt):
        vals, _ = stored_values(A, dt)
        if dt == "bf16":
            vals = vals.view(np.int16)
        M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, np.ascontiguousarray(vals), dt)
        if tune:
            M.tune("exhaustive", trial_reps=3)
        return M
    return mk("f64"), mk(inner)


def oracle_relres(A, x, b):
    r = b - oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x, threads=8)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("maker,inner", [(lambda: synth.poisson_2d_64(), "f32"),
                                         (lambda: synth.stencil3d7(20), "bf16"),
                                         (lambda: synth.stencil3d7(32), "f32")])
def test_cg_reaches_fp64_residual(maker, inner):
    A = maker()
    x_true = synth.uniform(0, 5, A.n)
    b = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x_true, threads=8)
    A64, A32 = handles(A, inner)
    bd = torch.from_numpy(b).to(DEV)
    xd = torch.zeros(A.n, dtype=torch.float64, device=DEV)
    info = smat.cg_mixed(A64, A32, bd, xd, rtol=1e-10, max_inner=2000)
    assert info["converged"] and info["status"] == smat.SMAT_OK, info
    x = xd.cpu().numpy()
    rr = oracle_relres(A, x, b)
    assert rr <= 1e-10, rr
    assert abs(rr - info["relres"]) <= 0.05 * rr + 1e-16
    assert info["outer"] >= 2  # FP32 alone cannot reach 1e-10: refinement did the rest
    A64.close(), A32.close()


def test_graph_and_plain_launches_agree_bitwise():
    A = synth.stencil3d7(16)
    b = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, synth.uniform(1, 5, A.n))
    A64, A32 = handles(A, "f32")
    bd = torch.from_numpy(b).to(DEV)
    out = []
    for g in (1, 0):
        xd = torch.zeros(A.n, dtype=torch.float64, device=DEV)
        info = smat.cg_mixed(A64, A32, bd, xd, use_graph=g, rtol=1e-11)
        out.append((xd.cpu().numpy(), info["inner_total"]))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0].view(np.uint64), out[1][0].view(np.uint64))


def test_limits_and_degenerate_cases():
    A = synth.poisson_2d_64()
    b = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, synth.uniform(2, 5, A.n))
    A64, A32 = handles(A, "f32", tune=False)
    bd = torch.from_numpy(b).to(DEV)
    xd = torch.zeros(A.n, dtype=torch.float64, device=DEV)
    info = smat.cg_mixed(A64, A32, bd, xd, max_total_inner=5)
    assert info["status"] == smat.SMAT_ERR_NOT_CONVERGED and info["inner_total"] <= 5 and not info["converged"]
    # b = 0: x = 0 is returned at once
    xd.fill_(3.0)
    info = smat.cg_mixed(A64, A32, torch.zeros_like(bd), xd)
    assert info["converged"] and torch.count_nonzero(xd).item() == 0
    # an FP64 handle cannot be the inner operator
    st, _ = smat.smat_cg_mixed(A64.h, A64.h, bd.data_ptr(), xd.data_ptr(), None, 0)
    assert st == smat.SMAT_ERR_INVALID_ARG
    R = synth.CSR(3, 4, np.array([0, 1, 2, 3], np.int32), np.array([0, 1, 2], np.int32), np.ones(3))
    N64 = smat.SpMatrix(3, 4, R.rowptr, R.colidx, R.val, "f64")
    N32 = smat.SpMatrix(3, 4, R.rowptr, R.colidx, R.val.astype(np.float32), "f32")
    st, _ = smat.smat_cg_mixed(N64.h, N32.h, bd.data_ptr(), xd.data_ptr(), None, 0)
    assert st == smat.SMAT_ERR_INVALID_ARG
    for M in (A64, A32, N64, N32):
        M.close()
