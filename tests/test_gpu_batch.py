"""Batched persistent SpMV (one graph launch for many matrices) against the
oracle and against the per-matrix products."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _members():
    mats = synth.amg_like_hierarchy(16)[:3] + synth.mixed_batch(12, 1e3, 3e4, base_seed=7)
    mats.append(CSR(40, 40, np.zeros(41, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty40"))
    mats.append(CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]), "one"))
    return mats


def _handles(mats, dtype):
    hs = []
    for A in mats:
        vals, _ = stored_values(A, dtype)
        M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, np.ascontiguousarray(vals), dtype)
        M.tune("exhaustive", trial_reps=3)
        hs.append(M)
    return hs


@pytest.mark.parametrize("mode", [smat.SMAT_BATCH_GRAPH, smat.SMAT_BATCH_PER_MATRIX, smat.SMAT_BATCH_AUTO])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_matches_oracle_and_single_products(dtype, mode):
    mats = _members()
    hs = _handles(mats, dtype)
    B = smat.Batch(hs).tune(trial_reps=3, mode=mode)
    info = B.info()
    assert info["count"] == len(mats) and info["tuned_ms"] > 0
    if mode == smat.SMAT_BATCH_GRAPH:
        assert info["per_matrix"] == 0 and info["tiles"] > 0 and info["grid"] > 0 and info["per_matrix_ms"] == -1.0
        assert info["tuned_ms"] == info["graph_ms"]
    elif mode == smat.SMAT_BATCH_PER_MATRIX:
        assert info["per_matrix"] == 1 and info["graph_ms"] == -1.0 and info["tuned_ms"] == info["per_matrix_ms"]
    else:  # both timed, the faster kept
        assert info["graph_ms"] > 0 and info["per_matrix_ms"] > 0
        assert info["tuned_ms"] == min(info["graph_ms"], info["per_matrix_ms"])
        assert info["per_matrix"] == (1 if info["per_matrix_ms"] < info["graph_ms"] else 0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    for call, seed in enumerate((0, 3)):
        xs = [torch.from_numpy(synth.uniform(seed + i, 1, A.n).astype(npdt)).to(DEV) for i, A in enumerate(mats)]
        y0 = [synth.uniform(seed + i, 2, A.m).astype(npdt) for i, A in enumerate(mats)]
        ys = [torch.from_numpy(v.copy()).to(DEV) for v in y0]
        alphas = [1.0 + 0.5 * i for i in range(len(mats))]
        betas = [0.0 if (i + call) % 2 == 0 else -0.75 for i in range(len(mats))]
        B.spmv(xs, ys, alphas, betas)
        torch.cuda.synchronize()
        for i, A in enumerate(mats):
            _, v64 = stored_values(A, dtype)
            ref, scale = reference(A, v64, xs[i].cpu().numpy(), alphas[i], betas[i], y0[i] if betas[i] else None)
            got = ys[i].cpu().numpy().astype(np.float64)
            assert_close_rows(got, ref, scale, TOL[dtype], f"call {call} member {i} ({A.name}) vs oracle")
            single = hs[i].spmv(xs[i], torch.from_numpy(y0[i].copy()).to(DEV), alphas[i], betas[i])
            assert_close_rows(got, single.cpu().numpy().astype(np.float64), scale, TOL[dtype],
                              f"call {call} member {i} vs its own plan")
    B.close()
    for M in hs:
        M.close()


@pytest.mark.parametrize("own", [0, 1, 2])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_own_launches_on_side_branches(dtype, own):
    # members whose plan has no batch kind (here COO, merge-path and, when
    # admissible, SPLIT) run their own kernels on side branches of the graph
    # (own = 1), or every member does (own = 2); the graph is captured again
    # when those members' vectors or scalars change between calls
    mats = _members()
    hs = _handles(mats, dtype)
    hs[4].tune("fixed", variant=smat.SMAT_V_COO)
    hs[5].tune("fixed", variant=smat.SMAT_V_CSR_MERGE)
    for M in hs[6:]:
        if (M.features()["admissible"] >> smat.SMAT_V_SPLIT) & 1:
            M.tune("fixed", variant=smat.SMAT_V_SPLIT)
            break
    B = smat.Batch(hs).tune(trial_reps=3, mode=smat.SMAT_BATCH_GRAPH, own_launches=own)
    info = B.info()
    assert info["per_matrix"] == 0 and info["own_launches"] == own
    npdt = np.float64 if dtype == "f64" else np.float32
    for call, seed in enumerate((1, 4, 4)):
        xs = [torch.from_numpy(synth.uniform(seed + i, 1, A.n).astype(npdt)).to(DEV) for i, A in enumerate(mats)]
        y0 = [synth.uniform(seed + i, 2, A.m).astype(npdt) for i, A in enumerate(mats)]
        ys = [torch.from_numpy(v.copy()).to(DEV) for v in y0]
        alphas = [0.5 + 0.25 * i for i in range(len(mats))]
        betas = [0.0 if (i + call) % 2 else 1.5 for i in range(len(mats))]
        B.spmv(xs, ys, alphas, betas)
        torch.cuda.synchronize()
        for i, A in enumerate(mats):
            _, v64 = stored_values(A, dtype)
            ref, scale = reference(A, v64, xs[i].cpu().numpy(), alphas[i], betas[i], y0[i] if betas[i] else None)
            assert_close_rows(ys[i].cpu().numpy().astype(np.float64), ref, scale, TOL[dtype],
                              f"own {own} call {call} member {i} ({A.name}, {hs[i].plan()['name']})")
    B.close()
    for M in hs:
        M.close()


def test_batch_rejects_mixed_dtypes_and_untuned_use():
    A = synth.stencil3d7(6)
    h64 = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, "f64")
    h32 = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val.astype(np.float32), "f32")
    import ctypes
    arr = (ctypes.c_void_p * 2)(h64.h, h32.h)
    b = ctypes.c_void_p()
    assert smat.lib().smat_batch_create(ctypes.byref(b), arr, 2) == smat.SMAT_ERR_INVALID_ARG
    B = smat.Batch([h64])
    x = torch.zeros(A.n, dtype=torch.float64, device=DEV)
    y = torch.zeros(A.m, dtype=torch.float64, device=DEV)
    with pytest.raises(smat.SmatError):
        B.spmv([x], [y])  # not tuned yet
    B.close()
    h64.close(), h32.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_galerkin_hierarchy(dtype):
    # the AMG setting: Galerkin coarse operators (P^T A P, smoothed
    # aggregation) of a 27-point operator, every level planned on its own and
    # all levels in one batched launch
    pytest.importorskip("scipy")
    mats = synth.galerkin_hierarchy(24, 5)
    hs = _handles(mats, dtype)
    B = smat.Batch(hs).tune(trial_reps=3, mode=smat.SMAT_BATCH_GRAPH)
    npdt = np.float64 if dtype == "f64" else np.float32
    xs = [torch.from_numpy(synth.uniform(40 + i, 1, A.n).astype(npdt)).to(DEV) for i, A in enumerate(mats)]
    y0 = [synth.uniform(50 + i, 2, A.m).astype(npdt) for i, A in enumerate(mats)]
    ys = [torch.from_numpy(v.copy()).to(DEV) for v in y0]
    B.spmv(xs, ys, [1.0] * len(mats), [0.5] * len(mats))
    torch.cuda.synchronize()
    for i, A in enumerate(mats):
        _, v64 = stored_values(A, dtype)
        ref, scale = reference(A, v64, xs[i].cpu().numpy(), 1.0, 0.5, y0[i])
        assert_close_rows(ys[i].cpu().numpy().astype(np.float64), ref, scale, TOL[dtype], f"level {i} ({A.name})")
        single = hs[i].spmv(xs[i]).cpu().numpy().astype(np.float64)
        ref1, scale1 = reference(A, v64, xs[i].cpu().numpy(), 1.0, 0.0, None)
        assert_close_rows(single, ref1, scale1, TOL[dtype], f"level {i} ({A.name}) own plan {hs[i].plan()['name']}")
    B.close()
    for M in hs:
        M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_batch_dia_members(dtype):
    # DIA members run the single-matrix kernel's bodies inside the persistent
    # kernel (FP64 lane-striped rows, FP32/BF16 the unchecked interior path
    # with 16-byte x loads); small tiles give every matrix several tiles and
    # ragged ends, and the sizes leave partial warps at the tails
    mats = [synth.stencil3d7(21), synth.stencil3d27(13), synth.box3d(9, 2), synth.box3d(5, 3),
            synth.stencil2d5(37, 29), synth.stencil3d7(3)]
    hs = []
    for A in mats:
        vals, _ = stored_values(A, dtype)
        M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, np.ascontiguousarray(vals), dtype)
        M.tune("fixed", variant=smat.SMAT_V_DIA)
        assert M.plan()["variant"] == smat.SMAT_V_DIA
        hs.append(M)
    B = smat.Batch(hs).tune(trial_reps=2, tile_scale=1, ctas_per_sm=2, mode=smat.SMAT_BATCH_GRAPH)
    assert B.info()["per_matrix"] == 0
    tdt = np.float64 if dtype == "f64" else np.float32
    for call, beta in enumerate((0.0, 1.5)):
        xs = [torch.from_numpy(synth.uniform(70 + i, 1, A.n).astype(tdt)).to(DEV) for i, A in enumerate(mats)]
        y0 = [synth.uniform(80 + i, 2, A.m).astype(tdt) for i, A in enumerate(mats)]
        ys = [torch.from_numpy(v.copy()).to(DEV) for v in y0]
        B.spmv(xs, ys, [0.75] * len(mats), [beta] * len(mats))
        torch.cuda.synchronize()
        for i, A in enumerate(mats):
            _, v64 = stored_values(A, dtype)
            ref, scale = reference(A, v64, xs[i].cpu().numpy(), 0.75, beta, y0[i] if beta else None)
            assert_close_rows(ys[i].cpu().numpy().astype(np.float64), ref, scale, TOL[dtype],
                              f"call {call} {A.name} ({dtype})")
    B.close()
    for M in hs:
        M.close()
