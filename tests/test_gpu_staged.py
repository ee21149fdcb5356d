"""The DIA product whose stripes are staged in shared memory by bulk copies
(Sec. 2.1's DIA format, one CTA per SM, a ring of stages fed several tiles
ahead), against the oracle within the per-row bars, on shapes chosen to reach
every path of its pipeline: more tiles per CTA than stages (the ring wraps
and its stages are reused), more than 32 stripes (each producer lane issues
several copies), a ragged last tile, non-square matrices whose offsets reach
outside x, and the three epilogue forms; in every storage type.  Also: the
result equals the direct DIA kernel's within the bars, a matrix whose
stripes do not fit the stage is refused, and no bounded wait ever ran out."""
import numpy as np
import pytest

import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
AB = [(1.0, 0.0), (2.5, 0.0), (-0.5, 2.0)]
STAGED_SHAPES = (1, 2)   # launch shapes of the staged kernel (smat_set_kernel ids)


def banded(m, n, offsets, keep, seed):
    """Rows i hold columns i + d for the offsets d that land in [0, n), each
    kept with probability `keep`; values N(0, 1)."""
    rng = np.random.default_rng(seed)
    offs = np.sort(np.asarray(offsets))
    rows, cols = [], []
    for i in range(m):
        c = i + offs
        c = c[(c >= 0) & (c < n)]
        c = c[rng.random(len(c)) < keep]
        rows.append(len(c))
        cols.append(c)
    rowptr = np.zeros(m + 1, np.int32)
    rowptr[1:] = np.cumsum(rows)
    colidx = np.concatenate(cols).astype(np.int32)
    return CSR(m, n, rowptr, colidx, rng.standard_normal(len(colidx)), name=f"banded_{m}x{n}_{len(offs)}")


CASES = {
    # ring wraps: ceil(rows / tile) > 4 stages x 152 CTAs in each storage type
    "stencil3d7_82": (lambda: synth.stencil3d7(82), ("f64",)),
    "stencil3d7_104": (lambda: synth.stencil3d7(104), ("f32",)),
    "stencil3d7_130": (lambda: synth.stencil3d7(130), ("bf16",)),
    # 27 stripes, ring wraps in FP32 (tiles of 448 rows)
    "stencil3d27_68": (lambda: synth.stencil3d27(68), ("f32", "f64", "bf16")),
    # 45 stripes: two copies per producer lane; tall, wide and ragged
    "banded_tall": (lambda: banded(70001, 50000, list(range(-30, 15)), 0.7, 3), ("f64", "f32", "bf16")),
    "banded_wide": (lambda: banded(20011, 90000, [-5000, -7, -1, 0, 1, 33, 800, 65000], 0.9, 4),
                    ("f64", "f32", "bf16")),
    # fewer tiles than SMs, tiny
    "stencil2d5_64": (lambda: synth.stencil2d5(64), ("f64", "f32", "bf16")),
    "banded_small": (lambda: banded(45, 45, [-3, 0, 2], 1.0, 5), ("f64", "f32", "bf16")),
}


def _handle(A, dtype):
    vals, vals64 = stored_values(A, dtype)
    if dtype == "bf16":
        vals = vals.view(np.int16)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)
    return M, vals64


def _product(M, A, dtype, x, y0, alpha, beta):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    y = torch.from_numpy(y0.copy()).to(DEV)
    M.spmv(torch.from_numpy(x).to(DEV).to(tdt), y, alpha, beta, variant=smat.SMAT_V_DIA)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_staged_dia_matches_the_oracle(name):
    make, dtypes = CASES[name]
    A = make()
    timeouts0 = smat.smat_get_wait_timeouts()
    for dtype in dtypes:
        M, vals64 = _handle(A, dtype)
        assert (M.features()["admissible"] >> smat.SMAT_V_DIA) & 1, (name, dtype)
        np_t = np.float64 if dtype == "f64" else np.float32
        x = synth.uniform(7, 1, A.n).astype(np_t)
        y0 = synth.uniform(7, 2, A.m).astype(np_t)
        _product(M, A, dtype, x, y0, 1.0, 0.0)   # builds DIA and measures its kernels
        M.set_kernel(smat.SMAT_V_DIA, 0)
        direct = _product(M, A, dtype, x, y0, -0.5, 2.0)
        _, scale_d = reference(A, vals64, x, -0.5, 2.0, y0)
        for k in STAGED_SHAPES:
            M.set_kernel(smat.SMAT_V_DIA, k)
            assert M.kernel(smat.SMAT_V_DIA) == k
            for alpha, beta in AB:
                got = _product(M, A, dtype, x, y0, alpha, beta)
                ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
                assert_close_rows(got, ref, scale, TOL[dtype], f"{name} {dtype} staged {k} a={alpha} b={beta}")
            staged = _product(M, A, dtype, x, y0, -0.5, 2.0)
            assert_close_rows(staged, direct, scale_d, 2 * TOL[dtype], f"{name} {dtype} staged {k} vs direct")
        M.close()
    assert smat.smat_get_wait_timeouts() == timeouts0


def full_bands(m, offsets, seed):
    """Every row i holds the columns i + d, d in `offsets`, that land in [0, m); values N(0, 1)."""
    offs = np.sort(np.asarray(offsets, dtype=np.int64))
    cols = np.arange(m, dtype=np.int64)[:, None] + offs[None, :]
    keep = (cols >= 0) & (cols < m)
    rowptr = np.zeros(m + 1, np.int32)
    rowptr[1:] = np.cumsum(keep.sum(axis=1))
    colidx = cols[keep].astype(np.int32)
    val = np.random.default_rng(seed).standard_normal(len(colidx))
    return CSR(m, m, rowptr, colidx, val, name=f"bands_{m}_{len(offs)}")


LIGHT = {
    # one or two stripes over millions of rows: a consumer does little work per
    # stage, so a released stage is refilled within microseconds, and every CTA
    # reuses each stage of its ring several times (5 to 18 tiles per CTA)
    "diag_f32": (1 << 24, [0], "f32"),
    "bidiag_f64": (1 << 23, [-1, 0], "f64"),
    "diag_bf16": (1 << 24, [0], "bf16"),
}


@pytest.mark.parametrize("name", list(LIGHT))
def test_staged_dia_light_stages_repeated(name):
    # a stage released by the consumers and refilled by the next bulk copy
    # must never hand a consumer data of another tile: repeated products on
    # the lightest stages, every row checked each time
    m, offsets, dtype = LIGHT[name]
    A = full_bands(m, offsets, 11)
    M, vals64 = _handle(A, dtype)
    np_t = np.float64 if dtype == "f64" else np.float32
    x = synth.uniform(13, 1, A.n).astype(np_t)
    y0 = np.zeros(A.m, np_t)
    _product(M, A, dtype, x, y0, 1.0, 0.0)
    ref, scale = reference(A, vals64, x, 1.0, 0.0, None)
    timeouts0 = smat.smat_get_wait_timeouts()
    for k in STAGED_SHAPES:
        M.set_kernel(smat.SMAT_V_DIA, k)
        for rep in range(6):
            got = _product(M, A, dtype, x, y0, 1.0, 0.0)
            assert_close_rows(got, ref, scale, TOL[dtype], f"{name} staged {k} repeat {rep}")
    assert smat.smat_get_wait_timeouts() == timeouts0
    M.close()


def test_staged_waits_that_run_out_leave_the_context_usable():
    # the test hook makes the consumers wait on a barrier nothing arrives on,
    # for 2e6 cycles (~1 ms): the kernel gives up, waits for its own copies,
    # counts the timeout and returns; the next products are correct
    A = synth.stencil3d7(64)
    M, vals64 = _handle(A, "f32")
    x = synth.uniform(9, 1, A.n).astype(np.float32)
    y0 = np.zeros(A.m, np.float32)
    _product(M, A, "f32", x, y0, 1.0, 0.0)
    for k in STAGED_SHAPES:
        M.set_kernel(smat.SMAT_V_DIA, k)
        before = smat.smat_get_wait_timeouts()
        smat.lib().smat_test_stall_pipelines(1, 2_000_000)
        try:
            _product(M, A, "f32", x, y0, 1.0, 0.0)
        finally:
            smat.lib().smat_test_stall_pipelines(0, 0)
        assert smat.smat_get_wait_timeouts() > before, k
        got = _product(M, A, "f32", x, y0, 1.0, 0.0)
        ref, scale = reference(A, vals64, x, 1.0, 0.0, None)
        assert_close_rows(got, ref, scale, TOL["f32"], f"staged {k} after a run-out wait")
    M.close()


def test_staged_dia_is_deterministic():
    A = synth.stencil3d27(40)
    M, _ = _handle(A, "f64")
    x = torch.from_numpy(synth.uniform(1, 1, A.n)).to(DEV)
    y = torch.zeros(A.m, dtype=torch.float64, device=DEV)
    M.spmv(x, y, variant=smat.SMAT_V_DIA)
    for k in STAGED_SHAPES:
        M.set_kernel(smat.SMAT_V_DIA, k)
        first = M.spmv(x, y.clone(), variant=smat.SMAT_V_DIA).cpu().numpy()
        for _ in range(3):
            again = M.spmv(x, y.clone(), variant=smat.SMAT_V_DIA).cpu().numpy()
            assert np.array_equal(first.view(np.int64), again.view(np.int64)), k
    M.close()


def test_staged_dia_refuses_stripes_that_do_not_fit():
    # 343 diagonals: 32 FP64 rows of every stripe take 86 KB, above the 48 KB
    # stage; the direct kernel still runs the product
    A = synth.box3d(12, 3)
    M, _ = _handle(A, "f64")
    if not (M.features()["admissible"] >> smat.SMAT_V_DIA) & 1:
        pytest.skip("DIA not admissible for this matrix")
    x = torch.from_numpy(synth.uniform(2, 1, A.n)).to(DEV)
    M.spmv(x, torch.zeros(A.m, dtype=torch.float64, device=DEV), variant=smat.SMAT_V_DIA)
    assert M.kernel(smat.SMAT_V_DIA) == 0
    for k in STAGED_SHAPES:
        with pytest.raises(smat.SmatError):
            M.set_kernel(smat.SMAT_V_DIA, k)
    M.close()


def test_kernel_choice_needs_a_built_format():
    A = synth.stencil2d5(16)
    M, _ = _handle(A, "f64")
    with pytest.raises(smat.SmatError):
        M.kernel(smat.SMAT_V_DIA)
    with pytest.raises(smat.SmatError):
        M.set_kernel(smat.SMAT_V_COO, 0)
    M.close()
