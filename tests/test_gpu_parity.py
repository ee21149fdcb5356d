"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs -- features and conversions bit for bit, every SpMV kernel
variant within the per-row bars (bit for bit where the operation sequence is
the CSR definition's)."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR
from helpers import TOL, assert_close_rows, reference, stored_values, vec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _long_row():
    # one dense row of 10k entries among short rows (rows longer than 32 * W)
    rl = np.array([3] * 50 + [10000] + [1] * 200 + [0] * 5 + [40] * 30, dtype=np.int64)
    rng = np.random.default_rng(9)
    n = 12000
    rp = np.concatenate([[0], np.cumsum(rl)]).astype(np.int32)
    col = np.concatenate([np.sort(rng.choice(n, r, replace=False)) for r in rl]).astype(np.int32)
    return CSR(len(rl), n, rp, col, rng.standard_normal(len(col)), "long_row")


def _nonsquare():
    rng = np.random.default_rng(3)
    m, n = 700, 2300
    d = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.01)
    d[50:60] = 0.0  # empty rows
    r, c = np.nonzero(d)
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return CSR(m, n, np.cumsum(rp).astype(np.int32), c.astype(np.int32), d[r, c], "nonsquare")


def _tiny(m, n, entries):
    rows = [[] for _ in range(m)]
    for i, j, v in entries:
        rows[i].append((j, v))
    rp = [0]
    cols, vals = [], []
    for r in rows:
        for j, v in sorted(r):
            cols.append(j)
            vals.append(v)
        rp.append(len(cols))
    return CSR(m, n, np.array(rp, np.int32), np.array(cols, np.int32), np.array(vals, np.float64), f"tiny{m}x{n}")


CASES = {
    "poisson2d_64": lambda: synth.poisson_2d_64(),
    "stencil3d7_20": lambda: synth.stencil3d7(20),
    "stencil3d27_9": lambda: synth.stencil3d27(9),
    "uniform_5000": lambda: synth.uniform_random(5000, 16.0, 1),
    "powerlaw_20000": lambda: synth.powerlaw(20000, 1.8, 3000, 2),
    "blockdiag_10001": lambda: synth.blockdiag(10001, 8, 3),
    "long_row": _long_row,
    "nonsquare_empty_rows": _nonsquare,
    "one_by_one": lambda: _tiny(1, 1, [(0, 0, 2.5)]),
    "one_row": lambda: _tiny(1, 50, [(0, j, j + 1.0) for j in range(0, 50, 3)]),
    "one_col": lambda: _tiny(40, 1, [(i, 0, i - 3.0) for i in range(0, 40, 2)]),
    "all_empty": lambda: CSR(33, 17, np.zeros(34, np.int32), np.zeros(0, np.int32), np.zeros(0), "all_empty"),
}


def make(A: CSR, dtype="f64"):
    vals, vals64 = stored_values(A, dtype)
    if dtype == "bf16":
        vals = vals.view(np.int16)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)
    return M, vals64


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    return request.param, CASES[request.param]()


def test_features_bit_exact(case):
    name, A = case
    M, _ = make(A)
    f = M.features()
    fo = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    for k in ("m", "n", "nnz", "max_rd", "min_rd", "empty_rows", "ndiags", "ntdiags", "s2", "r_valid"):
        assert f[k] == fo[k], (name, k, f[k], fo[k])
    for k in ("aver_rd", "var_rd", "er_dia", "er_ell", "ntdiags_ratio", "r"):
        assert np.float64(f[k]).view(np.uint64) == np.float64(fo[k]).view(np.uint64), (name, k, f[k], fo[k])
    M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_conversions_bit_exact(case, dtype):
    name, A = case
    M, _ = make(A, dtype)
    vals, _ = stored_values(A, dtype)
    adm = M.features()["admissible"]
    if (adm >> smat.SMAT_V_ELL) & 1 and A.nnz > 0:
        M.convert(smat.SMAT_FMT_ELL)
        col, val, K, P = M.export(smat.SMAT_FMT_ELL)
        ocol, oval, oK, oP = oracle.to_ell(A.m, A.rowptr, A.colidx, vals)
        assert (K, P) == (oK, oP)
        assert np.array_equal(col, ocol)
        assert np.array_equal(val.view(np.uint8), oval.view(np.uint8))
    if (adm >> smat.SMAT_V_DIA) & 1:
        M.convert(smat.SMAT_FMT_DIA)
        off, val, nd, P = M.export(smat.SMAT_FMT_DIA)
        ooff, oval, oP = oracle.to_dia(A.m, A.n, A.rowptr, A.colidx, vals)
        assert np.array_equal(off, ooff) and P == oP
        assert np.array_equal(val.view(np.uint8), oval.view(np.uint8))
    M.convert(smat.SMAT_FMT_COO)
    row, _, nnz, _ = M.export(smat.SMAT_FMT_COO)
    assert np.array_equal(row, oracle.to_coo(A.m, A.rowptr))
    M.close()


EXACT_F64 = {smat.SMAT_V_CSR_SCALAR_EXACT}


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (2.0, -1.0), (0.0, 0.5)])
def test_spmv_every_variant(case, dtype, ab):
    name, A = case
    alpha, beta = ab
    M, vals64 = make(A, dtype)
    x = vec(synth.uniform(0, 1, A.n), dtype)
    y0 = vec(synth.uniform(1, 1, A.m), dtype)
    ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
    adm = M.features()["admissible"]
    xd = torch.from_numpy(x).to(DEV)
    for v in range(smat.SMAT_NUM_VARIANTS + 1):
        if v < smat.SMAT_NUM_VARIANTS and not (adm >> v) & 1:
            continue
        y = torch.from_numpy(y0.copy()).to(DEV)
        if beta == 0:
            y.fill_(float("nan"))  # beta = 0: y must not be read
        M.spmv(xd, y, alpha, beta, variant=v)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.float64)
        what = f"{name} {dtype} {smat.VARIANT_NAMES[v]} alpha={alpha} beta={beta}"
        if dtype == "f64" and v in EXACT_F64:
            assert np.array_equal(got, ref), what + ": not bit-identical to the oracle"
        else:
            assert_close_rows(got, ref, scale, TOL[dtype], what)
    M.close()


def test_variant_runs_are_deterministic():
    A = synth.powerlaw(20000, 1.8, 3000, 5)
    M, _ = make(A)
    x = torch.from_numpy(synth.uniform(0, 1, A.n)).to(DEV)
    for v in range(smat.SMAT_NUM_VARIANTS):
        if not (M.features()["admissible"] >> v) & 1:
            continue
        a = M.spmv(x, variant=v).cpu().numpy()
        b = M.spmv(x, variant=v).cpu().numpy()
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), smat.VARIANT_NAMES[v]
    M.close()


def test_host_buffers_match_device():
    A = synth.uniform_random(3000, 9.0, 4)
    M, _ = make(A)
    M.tune("exhaustive", trial_reps=3)
    x = synth.uniform(0, 1, A.n)
    y0 = synth.uniform(1, 1, A.m)
    yd = M.spmv(torch.from_numpy(x).to(DEV), torch.from_numpy(y0.copy()).to(DEV), 1.5, 0.25).cpu().numpy()
    yh = y0.copy()
    M.spmv_host(x, yh, 1.5, 0.25)
    assert np.array_equal(yd, yh)
    M.close()


def test_casts_bit_exact():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(10000), rng.standard_normal(1000) * 1e-39,
                        rng.standard_normal(1000) * 1e38, [0.0, -0.0, 1e300, -1e300, 5e-324]])
    d = torch.from_numpy(v).to(DEV)
    o32 = torch.empty(len(v), dtype=torch.float32, device=DEV)
    ob = torch.empty(len(v), dtype=torch.int16, device=DEV)
    assert smat.smat_cast_f64_to_f32(d.data_ptr(), o32.data_ptr(), len(v), 0) == 0
    assert smat.smat_cast_f64_to_bf16(d.data_ptr(), ob.data_ptr(), len(v), 0) == 0
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):   # +-1e300 round to +-inf in FP32, as they must
        want32 = v.astype(np.float32)
    assert np.array_equal(o32.cpu().numpy().view(np.uint32), want32.view(np.uint32))
    assert np.array_equal(ob.cpu().numpy().view(np.uint16), oracle.round_bf16(v))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_misaligned_vectors_are_safe(dtype):
    # x and y one element into their buffers: ELL / DIA plans fall back to a
    # kernel without vector accesses; every variant still matches the oracle
    A = synth.stencil3d7(12)
    M, vals64 = make(A, dtype)
    npdt = np.float64 if dtype == "f64" else np.float32
    x = synth.uniform(0, 1, A.n).astype(npdt)
    y0 = synth.uniform(1, 1, A.m).astype(npdt)
    ref, scale = reference(A, vals64, x, 1.5, -0.5, y0)
    xb = torch.zeros(A.n + 1, dtype=torch.from_numpy(x).dtype, device=DEV)
    yb = torch.zeros(A.m + 1, dtype=torch.from_numpy(x).dtype, device=DEV)
    xb[1:] = torch.from_numpy(x).to(DEV)
    for v in range(smat.SMAT_NUM_VARIANTS):
        if not (M.features()["admissible"] >> v) & 1:
            continue
        yb[1:] = torch.from_numpy(y0).to(DEV)
        M.spmv(xb[1:], yb[1:], 1.5, -0.5, variant=v)
        torch.cuda.synchronize()
        assert_close_rows(yb[1:].cpu().numpy().astype(np.float64), ref, scale, TOL[dtype],
                          f"misaligned {dtype} {smat.VARIANT_NAMES[v]}")
    M.close()


def test_async_host_products_on_several_streams():
    mats = [synth.uniform_random(4000, 7.0, s) for s in range(4)]
    hs = [make(A)[0] for A in mats]
    xs = [torch.from_numpy(synth.uniform(i, 1, A.n)).pin_memory() for i, A in enumerate(mats)]
    ys = [torch.zeros(A.m, dtype=torch.float64).pin_memory() for A in mats]
    streams = [torch.cuda.Stream() for _ in range(2)]
    for rep in range(2):
        for i, M in enumerate(hs):
            M.spmv_host_async(xs[i], ys[i], 2.0, 0.0, stream=streams[i % 2])
        torch.cuda.synchronize()
        for i, A in enumerate(mats):
            ref, scale = reference(A, A.val, xs[i].numpy(), 2.0, 0.0, None)
            assert_close_rows(ys[i].numpy(), ref, scale, TOL["f64"], f"async host product {i}")
    for M in hs:
        M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_coo_full_and_partial_tiles(dtype):
    # COO over many full 2048-entry tiles and a partial last one (long rows
    # spanning tiles included): the oracle's product within the bars, and the
    # same bits run after run
    for A in (synth.powerlaw(60000, 1.8, 5000, 8), synth.uniform_random(20011, 7.0, 9), _long_row()):
        M, vals64 = make(A, dtype)
        x = vec(synth.uniform(0, 1, A.n), dtype)
        y0 = vec(synth.uniform(1, 1, A.m), dtype)
        ref, scale = reference(A, vals64, x, 1.25, -0.5, y0)
        xd = torch.from_numpy(x).to(DEV)
        outs = []
        for _ in range(2):
            y = torch.from_numpy(y0.copy()).to(DEV)
            M.spmv(xd, y, 1.25, -0.5, variant=smat.SMAT_V_COO)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy().astype(np.float64))
        assert_close_rows(outs[0], ref, scale, TOL[dtype], f"{A.name} {dtype} coo")
        assert np.array_equal(outs[0], outs[1]), A.name
        assert A.nnz % 2048 != 0   # a partial last tile is part of the case
        M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_alpha_zero_reads_neither_matrix_nor_x(dtype):
    # alpha = 0: y = beta*y (0 when beta = 0) in every variant, even with NaN
    # and Inf in x (the BLAS convention: A and x are not referenced)
    A = synth.powerlaw(20000, 1.8, 3000, 4)
    M, _ = make(A, dtype)
    npdt = np.float64 if dtype == "f64" else np.float32
    x = synth.uniform(0, 1, A.n).astype(npdt)
    x[::7] = np.nan
    x[3::11] = np.inf
    y0 = synth.uniform(1, 1, A.m).astype(npdt)
    xd = torch.from_numpy(x).to(DEV)
    for v in list(range(smat.SMAT_NUM_VARIANTS)) + [smat.SMAT_V_HYB, smat.SMAT_V_SPLIT]:
        for beta in (0.0, -0.75):
            y = torch.from_numpy(y0.copy()).to(DEV)
            try:
                M.spmv(xd, y, 0.0, beta, variant=v)
            except smat.SmatError:
                continue
            torch.cuda.synchronize()
            want = (np.float64(beta) * y0.astype(np.float64)).astype(npdt) if beta else np.zeros_like(y0)
            assert np.array_equal(y.cpu().numpy(), want), (smat.VARIANT_NAMES[v], beta)
    M.close()
