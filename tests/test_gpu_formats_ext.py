"""GPU parity of the further formats (HYB, SELL-32-sigma, BCSR, SPLIT; future work in
Sec. 8): conversions bit for bit against the oracle's, products within the
per-row bars, admissibility by the stated limits, and their place in the
execute-and-measure search."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import TOL, assert_close_rows, reference, stored_values, vec
from test_gpu_parity import CASES, make

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ESZ = {"f64": 8, "f32": 4, "bf16": 2}
EXT = {smat.SMAT_V_HYB: smat.SMAT_FMT_HYB, smat.SMAT_V_SELL: smat.SMAT_FMT_SELL, smat.SMAT_V_BCSR: smat.SMAT_FMT_BCSR,
       smat.SMAT_V_SPLIT: smat.SMAT_FMT_SPLIT}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    return request.param, CASES[request.param]()


def _convert(M, fmt):
    try:
        M.convert(fmt)
        return True
    except smat.SmatError as e:
        assert e.status == smat.SMAT_ERR_UNSUPPORTED, e
        return False


def _same_bytes(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


def _expected_admissible(A, dtype, slots, byts, extra_ok=True):
    # the limits ELL and DIA obey: slots <= 20 NNZ, bytes <= 4 x CSR bytes
    csr = (ESZ[dtype] + 4) * A.nnz + 4 * (A.m + 1)
    return A.nnz > 0 and A.m > 0 and extra_ok and slots <= 20 * A.nnz and byts <= 4 * max(csr, 1)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_ext_conversions_bit_exact(case, dtype):
    name, A = case
    M, _ = make(A, dtype)
    vals, _ = stored_values(A, dtype)
    esz = ESZ[dtype]
    P = oracle.pitch(A.m)
    # HYB
    ecol, ev, crow, ccol, cv, K, _ = oracle.to_hyb(A.m, A.rowptr, A.colidx, vals)
    want = _expected_admissible(A, dtype, K * A.m + len(crow), (esz + 4) * K * P + (esz + 8) * len(crow), K >= 1)
    assert _convert(M, smat.SMAT_FMT_HYB) == want, name
    if want:
        p = M.export_parts(smat.SMAT_FMT_HYB)
        assert p["K"] == K
        assert np.array_equal(p["ell_col"], ecol) and _same_bytes(p["ell_val"], ev)
        assert np.array_equal(p["coo_row"], crow) and np.array_equal(p["coo_col"], ccol)
        assert _same_bytes(p["coo_val"], cv)
    # SELL, the default window of 256 rows
    perm, width, sptr, scol, sval = oracle.to_sell(A.m, A.rowptr, A.colidx, vals, 256)
    ns = len(width)
    want = _expected_admissible(A, dtype, int(sptr[-1]), (esz + 4) * int(sptr[-1]) + 4 * 32 * ns + 12 * ns + 8)
    assert _convert(M, smat.SMAT_FMT_SELL) == want, name
    if want:
        p = M.export_parts(smat.SMAT_FMT_SELL)
        assert np.array_equal(p["perm"], perm) and np.array_equal(p["width"], width)
        assert np.array_equal(p["col"], scol) and _same_bytes(p["val"], sval)
    # BCSR, block size by bytes
    b, nb = oracle.bcsr_choose(A.m, A.n, A.rowptr, A.colidx, esz)
    want = _expected_admissible(A, dtype, nb * b * b, nb * (b * b * esz + 4) + 4 * (-(-A.m // b) + 1))
    assert _convert(M, smat.SMAT_FMT_BCSR) == want, name
    if want:
        p = M.export_parts(smat.SMAT_FMT_BCSR)
        brp, bcol, bval = oracle.to_bcsr(A.m, A.n, A.rowptr, A.colidx, vals, b)
        assert p["b"] == b and np.array_equal(p["browptr"], brp) and np.array_equal(p["bcol"], bcol)
        assert _same_bytes(p["val"], bval)
    # SPLIT: rows of >= 1024 entries in chunks of <= 4096, the rest as COO
    sp = oracle.split_rows(A.m, A.rowptr, A.colidx, vals, L=1024, CK=4096)
    nl, nc, ns, ne = len(sp["lrows"]), len(sp["crow"]), len(sp["srow"]), len(sp["empty"])
    byts = (esz + 4) * (A.nnz - ns) + 12 * nc + 4 * (2 * nl + 1) + (esz + 8) * ns + 4 * ne
    want = _expected_admissible(A, dtype, A.nnz, byts, nl >= 1)
    assert _convert(M, smat.SMAT_FMT_SPLIT) == want, name
    if want:
        p = M.export_parts(smat.SMAT_FMT_SPLIT)
        for k in ("crow", "cstart", "cend", "srow", "scol"):
            assert np.array_equal(p[k], sp[k]), (name, k)
        assert _same_bytes(p["sval"], sp["sval"])
    adm = M.features()["admissible"]
    for v, fmt in EXT.items():
        assert bool((adm >> v) & 1) == (smat.smat_format_dims(M.h, fmt)[0] == smat.SMAT_OK), (name, v)
    M.close()


def test_sell_window_follows_the_tuning_option():
    A = synth.powerlaw(3000, 1.8, 400, 4)
    M, _ = make(A)
    for sigma in (32, 256, 4096):
        M.tune("fixed", variant=smat.SMAT_V_SELL, sell_sigma=sigma, bytes_cap=100.0, fill_ratio_max=1000,
               keep_formats=1)
        perm, width, sptr, scol, sval = oracle.to_sell(A.m, A.rowptr, A.colidx, A.val, sigma)
        p = M.export_parts(smat.SMAT_FMT_SELL)
        assert np.array_equal(p["perm"], perm) and np.array_equal(p["col"], scol), sigma
        assert _same_bytes(p["val"], sval)
    with pytest.raises(smat.SmatError):
        M.tune("fixed", variant=smat.SMAT_V_SELL, sell_sigma=48)   # not a multiple of 32
    M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (2.0, -1.0), (0.0, 0.5)])
def test_ext_spmv(case, dtype, ab):
    name, A = case
    alpha, beta = ab
    M, vals64 = make(A, dtype)
    x = vec(synth.uniform(0, 1, A.n), dtype)
    y0 = vec(synth.uniform(1, 1, A.m), dtype)
    ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
    xd = torch.from_numpy(x).to(DEV)
    ran = 0
    for v in EXT:
        y = torch.from_numpy(y0.copy()).to(DEV)
        if beta == 0:
            y.fill_(float("nan"))  # beta = 0: y must not be read
        try:
            M.spmv(xd, y, alpha, beta, variant=v)
        except smat.SmatError as e:
            assert e.status == smat.SMAT_ERR_UNSUPPORTED
            assert not (M.features()["admissible"] >> v) & 1
            continue
        torch.cuda.synchronize()
        assert_close_rows(y.cpu().numpy().astype(np.float64), ref, scale, TOL[dtype],
                          f"{name} {dtype} {smat.VARIANT_NAMES[v]} alpha={alpha} beta={beta}")
        ran += 1
    if A.nnz > 0 and name not in ("one_row", "one_col", "one_by_one", "long_row", "powerlaw_20000"):
        assert ran >= 2, name
    if name in ("long_row", "powerlaw_20000"):   # rows of 1024 or more entries: SPLIT runs
        assert (M.features()["admissible"] >> smat.SMAT_V_SPLIT) & 1, name
    M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mk", [lambda: synth.blockdiag(999, 8, 2), lambda: synth.powerlaw(3000, 1.8, 2000, 6)])
def test_ext_misaligned_vectors_are_safe(dtype, mk):
    A = mk()
    M, vals64 = make(A, dtype)
    npdt = np.float64 if dtype == "f64" else np.float32
    x = synth.uniform(0, 1, A.n).astype(npdt)
    y0 = synth.uniform(1, 1, A.m).astype(npdt)
    ref, scale = reference(A, vals64, x, 1.5, -0.5, y0)
    xb = torch.zeros(A.n + 1, dtype=torch.from_numpy(x).dtype, device=DEV)
    yb = torch.zeros(A.m + 1, dtype=torch.from_numpy(x).dtype, device=DEV)
    xb[1:] = torch.from_numpy(x).to(DEV)
    for v in EXT:
        yb[1:] = torch.from_numpy(y0).to(DEV)
        try:
            M.spmv(xb[1:], yb[1:], 1.5, -0.5, variant=v)
        except smat.SmatError as e:   # not admissible on this matrix
            assert e.status == smat.SMAT_ERR_UNSUPPORTED
            continue
        torch.cuda.synchronize()
        assert_close_rows(yb[1:].cpu().numpy().astype(np.float64), ref, scale, TOL[dtype],
                          f"misaligned {dtype} {smat.VARIANT_NAMES[v]}")
    M.close()


def _csr_from_coo(m, n, rows, cols, seed, name):
    from paper_1210_2536_gb300.synth import CSR
    order = np.lexsort((cols, rows))
    rows, cols = np.asarray(rows)[order], np.asarray(cols)[order]
    rowptr = np.zeros(m + 1, np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    val = np.random.default_rng(seed).standard_normal(len(cols))
    return CSR(m, n, rowptr, cols.astype(np.int32), val, name=name)


def _uneven_blocks(m, b, seed):
    # even block rows hold two dense b x b blocks (their own and one far away),
    # odd block rows none: as many blocks as block rows, but not one per row
    rows, cols = [], []
    mb = (m + b - 1) // b
    for I in range(0, mb, 2):
        J2 = (I + mb // 2) % mb
        for J in (I, J2):
            for r in range(I * b, min(m, I * b + b)):
                for c in range(J * b, min(m, J * b + b)):
                    rows.append(r)
                    cols.append(c)
    return _csr_from_coo(m, m, rows, cols, seed, f"uneven_blocks_{m}")


def _blockdiag_plus_one(m, b, seed):
    A = synth.blockdiag(m, b, seed)
    rows = np.repeat(np.arange(m), np.diff(A.rowptr))
    return _csr_from_coo(m, m, np.append(rows, 5), np.append(A.colidx, m - 1), seed, f"blockdiag_plus_one_{m}")


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("mk", [lambda: synth.blockdiag(20000, 8, 4), lambda: synth.blockdiag(999, 8, 2),
                                lambda: _uneven_blocks(4000, 8, 5), lambda: _blockdiag_plus_one(4000, 8, 6)],
                         ids=["uniform", "uniform_ragged", "uneven_same_count", "one_extra_block"])
def test_bcsr_uniform_and_uneven_block_rows(dtype, mk):
    # block rows that all hold the same number of blocks skip the block-row
    # pointers; a layout whose block count divides evenly among the block
    # rows without every row holding that count, and one that does not
    # divide, read them; all match the oracle
    A = mk()
    M, vals64 = make(A, dtype)
    x = vec(synth.uniform(3, 1, A.n), dtype)
    y0 = vec(synth.uniform(3, 2, A.m), dtype)
    assert _convert(M, smat.SMAT_FMT_BCSR), A.name
    for alpha, beta in [(1.0, 0.0), (-2.0, 0.5)]:
        ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
        y = torch.from_numpy(y0.copy()).to(DEV)
        M.spmv(torch.from_numpy(x).to(DEV), y, alpha, beta, variant=smat.SMAT_V_BCSR)
        torch.cuda.synchronize()
        assert_close_rows(y.cpu().numpy().astype(np.float64), ref, scale, TOL[dtype], f"{A.name} {dtype} a={alpha} b={beta}")
    M.close()


def test_ext_formats_in_the_search():
    # exhaustive mode times every admissible variant, the further formats too
    A = synth.blockdiag(200000, 8, 1)
    M, _ = make(A)
    M.tune("exhaustive", trial_reps=5)
    t = M.timings()
    adm = M.features()["admissible"]
    assert (adm >> smat.SMAT_V_BCSR) & 1 and (adm >> smat.SMAT_V_HYB) & 1
    for v in range(smat.SMAT_NUM_ALL_VARIANTS):
        if v != smat.SMAT_V_CSR_SCALAR_EXACT and (adm >> v) & 1:
            assert t[v] > 0, smat.VARIANT_NAMES[v]
    tried = [v for v in range(smat.SMAT_NUM_ALL_VARIANTS) if t[v] > 0]
    assert t[M.plan()["variant"]] <= 1.02 * min(t[v] for v in tried)   # within the near-tie tolerance
    # without them in `allowed`, none is timed
    M.tune("exhaustive", trial_reps=3, allowed=0xFF)
    assert np.all(M.timings()[8:] < 0)
    # fixed mode accepts them; the CSR-exact kernel is not a plan
    M.tune("fixed", variant=smat.SMAT_V_BCSR)
    assert M.plan()["variant"] == smat.SMAT_V_BCSR and M.launches() == 1
    with pytest.raises(smat.SmatError):
        M.tune("fixed", variant=smat.SMAT_V_CSR_SCALAR_EXACT)
    M.close()


def test_learned_mode_times_cheaper_further_formats():
    # a model that always answers ELL: on a block-diagonal matrix BCSR (8x8
    # blocks) moves fewer bytes than ELL, HYB as many and SELL a few more, all
    # within 1.25x, so all are timed beside the pick
    W = np.zeros(smat.SMAT_MLP_PARAMS, np.float32)
    W[-8 + smat.SMAT_V_ELL] = 10.0          # output bias of the ELL class
    assert smat.smat_set_model(W, np.zeros(12), np.ones(12)) == 0
    try:
        A = synth.blockdiag(100000, 8, 2)
        M, _ = make(A)
        M.tune("learned", conf_threshold=0.5)
        t = M.timings()
        ext = (smat.SMAT_V_HYB, smat.SMAT_V_SELL, smat.SMAT_V_BCSR)
        assert t[smat.SMAT_V_ELL] > 0 and all(t[v] > 0 for v in ext) and M.plan()["trialled"] == 1
        assert M.plan()["variant"] in (smat.SMAT_V_ELL,) + ext
        assert t[M.plan()["variant"]] <= 1.02 * min(t[v] for v in (smat.SMAT_V_ELL,) + ext)
        M.tune("learned", conf_threshold=0.5, trial_extended=0)
        assert M.plan()["variant"] == smat.SMAT_V_ELL and M.plan()["trialled"] == 0
        M.close()
    finally:
        smat.smat_set_model(None, None, None)


def test_ext_allocation_failures_leak_nothing():
    A = synth.blockdiag(50000, 8, 1)
    torch.cuda.synchronize()
    assert smat.lib().smat_release_cached_memory() == smat.SMAT_OK
    free0 = torch.cuda.mem_get_info()[0]
    seen = set()
    for k in range(1, 14):
        M, _ = make(A)
        smat.lib().smat_test_fail_alloc_after(k)
        try:
            st = smat.smat_convert(M.h, smat.SMAT_FMT_BCSR, 0)
            st2 = smat.smat_convert(M.h, smat.SMAT_FMT_SELL, 0)
            st3 = smat.smat_convert(M.h, smat.SMAT_FMT_HYB, 0)
        finally:
            smat.lib().smat_test_fail_alloc_after(0)
        seen |= {st, st2, st3}
        assert {st, st2, st3} <= {smat.SMAT_OK, smat.SMAT_ERR_ALLOC}
        M.close()
    assert smat.SMAT_ERR_ALLOC in seen
    torch.cuda.synchronize()
    assert smat.lib().smat_release_cached_memory() == smat.SMAT_OK   # the pool's cached blocks are not leaks
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_split_long_short_and_empty_rows_in_one_product(dtype):
    # every part of a SPLIT product at once: chunks of long rows and COO tiles
    # of short rows in one grid, then the long rows' sums, the tiles' carries
    # and the empty rows in one closing pass
    from paper_1210_2536_gb300.synth import CSR
    P = synth.powerlaw(30000, 1.8, 6000, 7)
    rl = np.diff(P.rowptr).astype(np.int64)
    keep = np.ones(P.m, bool)
    keep[::97] = False                                        # empty rows
    mask = np.repeat(keep, rl)
    rp = np.concatenate([[0], np.cumsum(rl * keep)]).astype(np.int32)
    A = CSR(P.m, P.n, rp, P.colidx[mask], P.val[mask], "powerlaw_with_empty_rows")
    M, vals64 = make(A, dtype)
    M.convert(smat.SMAT_FMT_SPLIT)
    f = M.features()
    assert f["split_nc"] > 1 and f["empty_rows"] > 0
    assert f["split_ns"] > 4 * 2048                           # several COO tiles, so carries
    x = vec(synth.uniform(5, 1, A.n), dtype)
    xd = torch.from_numpy(x).to(DEV)
    for alpha, beta in ((1.0, 0.0), (2.0, -0.5), (-1.5, 1.0), (0.0, 0.75)):
        y0 = vec(synth.uniform(6, 1, A.m), dtype)
        y = torch.from_numpy(y0.copy()).to(DEV)
        if beta == 0:
            y.fill_(float("nan"))
        M.spmv(xd, y, alpha, beta, variant=smat.SMAT_V_SPLIT)
        torch.cuda.synchronize()
        ref, scale = reference(A, vals64, x, alpha, beta, y0 if beta != 0 else None)
        assert_close_rows(y.cpu().numpy().astype(np.float64), ref, scale, TOL[dtype],
                          f"SPLIT {dtype} alpha={alpha} beta={beta}")
    M.close()


def test_split_launch_count():
    # SPLIT is two launches: the grid of chunks and COO tiles, then the
    # closing pass (long rows' sums, carries, empty rows) when it has work
    from test_gpu_parity import _long_row
    for A, want in ((synth.powerlaw(30000, 1.8, 6000, 7), 2), (_long_row(), 2)):
        M, _ = make(A, "f64")
        M.tune("fixed", variant=smat.SMAT_V_SPLIT)
        assert M.launches() == want, A.name
        M.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_every_variant_gives_the_same_bits_twice(dtype):
    # every kernel combines its partial sums in a fixed order (no atomics on
    # values), so a product repeated on the same inputs gives identical bits:
    # the carries of COO / merge-path / HYB / SPLIT tiles and SPLIT's chunk
    # sums included
    A = synth.powerlaw(40000, 1.8, 5000, 11)
    M, _ = make(A, dtype)
    x = torch.from_numpy(vec(synth.uniform(2, 1, A.n), dtype)).to(DEV)
    y0 = vec(synth.uniform(3, 1, A.m), dtype)
    ran = 0
    for v in range(smat.SMAT_NUM_ALL_VARIANTS):
        outs = []
        for _ in range(2):
            y = torch.from_numpy(y0.copy()).to(DEV)
            try:
                M.spmv(x, y, 1.5, 0.25, variant=v)
            except smat.SmatError as e:
                assert e.status == smat.SMAT_ERR_UNSUPPORTED
                break
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
        if len(outs) == 2:
            assert np.array_equal(outs[0].view(np.uint8), outs[1].view(np.uint8)), smat.VARIANT_NAMES[v]
            ran += 1
    assert ran >= 8
    M.close()
