"""The configurations at their full sizes, in the launch configuration the
configuration benchmarks time, every output row against the oracle: the
batched multigrid-like hierarchy with 64 further matrices, the power-law
matrix with 8e6 rows in three storage types, and the mixed-precision CG on the
7-point 256^3 Laplacian."""
import os

import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
THREADS = os.cpu_count() or 1


@pytest.fixture(autouse=True)
def _model():
    assert smat.smat_load_model(smat.MODEL_PATH) == smat.SMAT_OK


def _handle(A, dtype):
    vals, v64 = stored_values(A, dtype)
    if dtype == "bf16":
        vals = vals.view(np.int16)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)
    return M, v64


@pytest.mark.parametrize("mode", [smat.SMAT_BATCH_AUTO, smat.SMAT_BATCH_GRAPH])
def test_batched_hierarchy_full_size(mode):
    # 27-point stencils on 192^3 .. 12^3 (215.8 M stored entries) and 64
    # matrices of mixed structure, each with its learned plan, in one batch
    mats = synth.amg_like_hierarchy(192) + synth.mixed_batch(64)
    hs, v64s = [], []
    for A in mats:
        M, v64 = _handle(A, "f64")
        M.tune("learned")
        hs.append(M)
        v64s.append(v64)
    B = smat.Batch(hs).tune(mode=mode)
    xs = [torch.from_numpy(synth.uniform(i, 1, A.n)).to(DEV) for i, A in enumerate(mats)]
    y0 = [synth.uniform(i, 2, A.m) for i, A in enumerate(mats)]
    ys = [torch.from_numpy(v.copy()).to(DEV) for v in y0]
    alphas = [1.0 if i % 3 else -0.5 for i in range(len(mats))]
    betas = [0.0 if i % 2 else 0.25 for i in range(len(mats))]
    B.spmv(xs, ys, alphas, betas)
    torch.cuda.synchronize()
    for i, A in enumerate(mats):
        ref, scale = reference(A, v64s[i], xs[i].cpu().numpy(), alphas[i], betas[i], y0[i] if betas[i] else None)
        assert_close_rows(ys[i].cpu().numpy(), ref, scale, TOL["f64"],
                          f"member {i} ({A.name}, {hs[i].plan()['name']}, mode {B.info()['per_matrix']})")
    B.close()
    for M in hs:
        M.close()


@pytest.fixture(scope="module")
def powerlaw_8m():
    return synth.powerlaw(8_000_000, 1.8, 10000, 0)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_powerlaw_8m_full_size(powerlaw_8m, dtype):
    # the precision workload: per row within the bar against the stored
    # values, and against the FP64 matrix within what the storage rounding
    # allows (each value moves by at most 2^-24 (FP32) or 2^-8 (BF16) of itself)
    A = powerlaw_8m
    M, v64 = _handle(A, dtype)
    M.tune("learned")
    x = synth.uniform(0, 1, A.n)
    xs = x if dtype == "f64" else x.astype(np.float32)
    y = M.spmv(torch.from_numpy(xs).to(DEV)).cpu().numpy().astype(np.float64)
    ref, scale = reference(A, v64, xs, 1.0, 0.0, None)
    assert_close_rows(y, ref, scale, TOL[dtype], f"powerlaw 8e6 {dtype} {M.plan()['name']} vs stored values")
    if dtype != "f64":
        x64 = np.asarray(xs, np.float64)
        ref64 = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x64, threads=THREADS)
        sc64 = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(A.val), np.abs(x64), threads=THREADS)
        err = np.abs(y - ref64) / np.maximum(sc64, 1e-300)
        storage = 2.0 ** -24 if dtype == "f32" else 2.0 ** -8
        assert float(err.max()) <= storage + TOL[dtype], (dtype, float(err.max()))
    M.close()


def test_mixed_cg_256_full_size():
    # the CG of the precision workload: FP32 inner solve, FP64 residual and
    # update, to a relative residual of 1e-10 that the oracle recomputes
    L = synth.stencil3d7(256)
    xt = synth.uniform(0, 5, L.n)
    b = oracle.spmv_csr(L.m, L.rowptr, L.colidx, L.val, xt, threads=THREADS)
    H64, _ = _handle(L, "f64")
    H32, _ = _handle(L, "f32")
    H64.tune("learned")
    H32.tune("learned")
    bd = torch.from_numpy(b).to(DEV)
    xd = torch.zeros(L.n, dtype=torch.float64, device=DEV)
    info = smat.cg_mixed(H64, H32, bd, xd, max_total_inner=5000, rtol=1e-10, max_inner=2000)
    assert info["converged"], info
    r = b - oracle.spmv_csr(L.m, L.rowptr, L.colidx, L.val, xd.cpu().numpy(), threads=THREADS)
    relres = float(np.linalg.norm(r) / np.linalg.norm(b))
    assert relres <= 1e-10, relres
    assert abs(relres - info["relres"]) <= 1e-3 * relres + 1e-15   # the solver's own FP64 residual agrees
    H64.close()
    H32.close()
