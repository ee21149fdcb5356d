"""The C ABI's behaviour on the GPU: CSR validation through the device flag,
allocation failures without leaks, the tuning modes, and parity at the full
size of the bench workload."""
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


def _create(m, n, rp, ci, v, dtype=smat.SMAT_F64):
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci, np.int32)
    v = np.ascontiguousarray(v, np.float64)
    st, h = smat.smat_create(m, n, len(ci), rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                             v.ctypes.data if len(v) else None, dtype)
    return st, h


BAD = {
    "unsorted columns": (3, 4, [0, 2, 3, 4], [2, 1, 0, 3], [1, 1, 1, 1]),
    "duplicate column": (2, 4, [0, 2, 3], [1, 1, 0], [1, 1, 1]),
    "column out of range": (2, 4, [0, 1, 2], [0, 4], [1, 1]),
    "negative column": (2, 4, [0, 1, 2], [-1, 0], [1, 1]),
    "rowptr decreasing": (3, 3, [0, 2, 1, 3], [0, 1, 2], [1, 1, 1]),
    "rowptr end mismatch": (2, 3, [0, 1, 3], [0, 1], [1, 1]),
    "rowptr start nonzero": (2, 3, [1, 1, 2], [0, 1], [1, 1]),
}


@pytest.mark.parametrize("case", sorted(BAD))
def test_invalid_csr_is_rejected(case):
    m, n, rp, ci, v = BAD[case]
    st, h = _create(m, n, rp, ci, v)
    assert st == smat.SMAT_ERR_INVALID_CSR and not h


def test_valid_edge_cases_are_accepted():
    for m, n, rp, ci in [(0, 0, [0], []), (3, 0, [0, 0, 0, 0], []), (1, 1, [0, 1], [0])]:
        st, h = _create(m, n, rp, ci, np.ones(len(ci)))
        assert st == smat.SMAT_OK
        smat.smat_destroy(h)


def test_allocation_failure_returns_alloc_and_leaks_nothing():
    A = synth.powerlaw(50000, 1.8, 2000, 1)
    torch.cuda.synchronize()
    assert smat.lib().smat_release_cached_memory() == smat.SMAT_OK
    free0 = torch.cuda.mem_get_info()[0]
    seen = set()
    for k in range(1, 12):
        smat.lib().smat_test_fail_alloc_after(k)
        try:
            st, h = _create(A.m, A.n, A.rowptr, A.colidx, A.val)
            if st == smat.SMAT_OK:
                M = h
                o = smat.smat_tune_opts_default()
                o.mode = smat.SMAT_TUNE_EXHAUSTIVE
                o.trial_reps = 2
                st = smat.smat_tune(M, o, 0)
                smat.smat_destroy(M)
        finally:
            smat.lib().smat_test_fail_alloc_after(0)
        seen.add(st)
        assert st in (smat.SMAT_OK, smat.SMAT_ERR_ALLOC), smat.smat_status_string(st)
    assert smat.SMAT_ERR_ALLOC in seen
    torch.cuda.synchronize()
    assert smat.lib().smat_release_cached_memory() == smat.SMAT_OK   # the pool's cached blocks are not leaks
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)   # nothing left allocated


def test_tuning_modes():
    A = synth.stencil3d7(24)
    M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, "f64")
    adm = M.features()["admissible"]
    assert (adm >> smat.SMAT_V_DIA) & 1 and (adm >> smat.SMAT_V_ELL) & 1
    M.tune("rules")                                  # the paper's thresholds: few, full diagonals -> DIA
    assert M.plan()["variant"] == smat.SMAT_V_DIA and M.plan()["trialled"] == 0
    M.tune("fixed", variant=smat.SMAT_V_CSR_MERGE)
    assert M.plan()["variant"] == smat.SMAT_V_CSR_MERGE
    M.tune("exhaustive", trial_reps=5, allowed=0b11100001)
    t = M.timings()
    tried = [v for v in range(8) if t[v] > 0]
    assert set(tried) == {0, 5, 6, 7}
    # the fastest, or a lower variant id within the 2 % near-tie tolerance
    assert t[M.plan()["variant"]] <= 1.02 * min(t[v] for v in tried)
    smat.smat_set_model(None, None, None)
    with pytest.raises(smat.SmatError):
        M.tune("learned")                             # no model installed
    P = synth.powerlaw(5000, 1.8, 1000, 3)
    Q = smat.SpMatrix(P.m, P.n, P.rowptr, P.colidx, P.val, "f64")
    assert not (Q.features()["admissible"] >> smat.SMAT_V_DIA) & 1   # 20x fill rule
    with pytest.raises(smat.SmatError):
        Q.tune("fixed", variant=smat.SMAT_V_DIA)
    M.close(), Q.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_bench_workload_parity(dtype):
    # the bench's matrices at full size, tuned as the bench tunes them, all rows
    if smat.smat_load_model(smat.MODEL_PATH) != 0:
        pytest.skip("no selector model")
    for A in synth.structures_suite(1.0):
        vals, v64 = stored_values(A, dtype)
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                          torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)
        M.tune("learned")
        x = synth.uniform(0, 1, A.n).astype(np.float64 if dtype == "f64" else np.float32)
        y = M.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy().astype(np.float64)
        ref, scale = reference(A, v64, x, 1.0, 0.0, None)
        assert_close_rows(y, ref, scale, TOL[dtype], f"{A.name} {dtype} {M.plan()['name']}")
        f, fo = M.features(), oracle.features(A.m, A.n, A.rowptr, A.colidx)
        for k in ("nnz", "max_rd", "min_rd", "ndiags", "ntdiags", "var_rd", "er_dia", "er_ell", "r"):
            assert f[k] == fo[k], (A.name, k)
        M.close()
    smat.smat_set_model(None, None, None)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_every_variant_parity(dtype):
    # every variant the tuner can pick for the bench's matrices, at full size
    # (the pick itself depends on timings), and every kernel behind DIA and
    # ELL, all rows against the oracle
    timeouts0 = smat.smat_get_wait_timeouts()
    for A in synth.structures_suite(1.0):
        vals, v64 = stored_values(A, dtype)
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                          torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)
        x = synth.uniform(0, 1, A.n).astype(np.float64 if dtype == "f64" else np.float32)
        xd = torch.from_numpy(x).to(DEV)
        ref, scale = reference(A, v64, x, 1.0, 0.0, None)
        ran = []
        for v in range(smat.SMAT_NUM_ALL_VARIANTS):
            try:
                M.spmv(xd, variant=v)                 # builds the format when admissible
            except smat.SmatError:
                continue
            kernels = {smat.SMAT_V_DIA: (0, 1, 2), smat.SMAT_V_ELL: (0, 1)}.get(v, (None,))
            for k in kernels:
                if k is not None:
                    try:
                        M.set_kernel(v, k)
                    except smat.SmatError:            # a staged shape this matrix does not fit
                        continue
                y = M.spmv(xd, variant=v).cpu().numpy().astype(np.float64)
                assert_close_rows(y, ref, scale, TOL[dtype], f"{A.name} {dtype} {smat.VARIANT_NAMES[v]} kernel {k}")
                ran.append((v, k))
        assert len({v for v, _ in ran}) >= 6, (A.name, ran)
        M.close()
    assert smat.smat_get_wait_timeouts() == timeouts0


def test_concurrent_products_on_one_handle():
    # products on one handle from two streams at once: the plans that carry
    # partial sums between CTAs (merge-path, COO, HYB, SPLIT) give each stream
    # scratch of its own, so every product is the oracle's
    A = synth.powerlaw(150000, 1.8, 5000, 3)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(A.val).to(DEV), "f64")
    xs = [synth.uniform(70 + k, 1, A.n) for k in range(2)]
    refs = [reference(A, A.val, x, 1.0, 0.0, None) for x in xs]
    xd = [torch.from_numpy(x).to(DEV) for x in xs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for v in (smat.SMAT_V_COO, smat.SMAT_V_CSR_MERGE, smat.SMAT_V_HYB, smat.SMAT_V_SPLIT):
        M.spmv(xd[0], variant=v)          # builds the format
        torch.cuda.synchronize()
        ys = [[torch.empty(A.m, dtype=torch.float64, device=DEV) for _ in range(6)] for _ in range(2)]
        for r in range(6):
            for k in range(2):
                M.spmv(xd[k], ys[k][r], variant=v, stream=streams[k])
        torch.cuda.synchronize()
        for k in range(2):
            ref, scale = refs[k]
            for r in range(6):
                assert_close_rows(ys[k][r].cpu().numpy(), ref, scale, TOL["f64"], f"{smat.VARIANT_NAMES[v]} s{k} r{r}")
    M.close()


def test_exhaustive_near_ties_take_the_fewest_bytes():
    # trial_tie: medians within that fraction of the fastest count as equal;
    # among them the pick moves the fewest matrix bytes, then has the lowest
    # variant id
    A = synth.stencil2d5(64)    # every variant within a few us of the others
    M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, "f64")

    def expected(t, tie):
        tried = [v for v in range(smat.SMAT_NUM_ALL_VARIANTS) if t[v] > 0]
        best = min(t[v] for v in tried)
        return min((M.variant_bytes(v), v) for v in tried if t[v] <= (1.0 + tie) * best)[1]

    M.tune("exhaustive", trial_reps=5, trial_race=0.0, trial_tie=100.0)
    t = M.timings()
    assert M.plan()["variant"] == expected(t, 100.0)
    for tie in (0.0, 0.02, 0.25):
        M.tune("exhaustive", trial_reps=5, trial_race=0.0, trial_tie=tie)
        t = M.timings()
        best = min(t[v] for v in range(smat.SMAT_NUM_ALL_VARIANTS) if t[v] > 0)
        pick = M.plan()["variant"]
        assert t[pick] <= (1.0 + tie) * best
        assert pick == expected(t, tie), (tie, pick, t)
        y = M.spmv(torch.from_numpy(synth.uniform(0, 1, A.n)).to(DEV))   # the pick's format is in place
        assert y.shape[0] == A.m
    # bytes agree with the formats' sizes
    assert M.variant_bytes(smat.SMAT_V_CSR_SCALAR) == 12 * A.nnz + 4 * (A.m + 1)
    assert M.variant_bytes(smat.SMAT_V_COO) == 16 * A.nnz
    M.close()


def test_exhaustive_pick_is_stable_when_retimed():
    # the exhaustive search checks itself: a second, independent search
    # finds the first search's pick within 15 % of its own fastest variant (timing noise of
    # ~20 us launches included)
    for A in (synth.stencil3d7(96), synth.powerlaw(300000, 1.8, 5000, 2), synth.uniform_random(300000, 16.0, 3)):
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                          torch.from_numpy(A.val).to(DEV), "f64")
        M.tune("exhaustive", trial_reps=10, keep_formats=1)
        first = M.plan()["variant"]
        M.tune("exhaustive", trial_reps=10, keep_formats=1)
        t = M.timings()
        best = min(v for v in t if v > 0)
        assert t[first] <= 1.15 * best, (A.name, smat.VARIANT_NAMES[first], t[first], best)
        M.close()


def test_gather_rate_measurement():
    # the gather ceiling: positive, and no faster for FP64 than for FP32 x
    r64 = smat.smat_measure_gather_rate(2_000_000, 4_000_000, "f64", 5)
    r32 = smat.smat_measure_gather_rate(2_000_000, 4_000_000, "f32", 5)
    assert 1e9 < r64 < 1e13 and 1e9 < r32 < 1e13
    assert r64 <= 1.5 * r32
    with pytest.raises(smat.SmatError):
        smat.smat_measure_gather_rate(0, 100, "f64", 5)


def test_fp64_rate_measurement():
    # the FP64 roof: a GB300 runs a few hundred G fused multiply-adds per
    # second (about 2 per clock per SM), far below its FP32 rate
    r = smat.smat_measure_fp64_rate(5)
    assert 1e11 < r < 3e12, r
    with pytest.raises(smat.SmatError):
        smat.smat_measure_fp64_rate(0)


def test_trial_racing_keeps_the_pick_and_saves_time():
    # racing stops timing a candidate after 3 products when it is already
    # 1.3x the best so far; on a power-law matrix, where CSR-scalar and the
    # long-row kernels are several times slower than the best, the exhaustive
    # search then finds an equally fast plan in less time
    A = synth.powerlaw(300000, 1.8, 5000, 4)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(A.val).to(DEV), "f64")
    M.tune("exhaustive", trial_race=0.0)          # warm: formats and kernels loaded once
    M.tune("exhaustive", trial_race=0.0)
    full, t_full = M.timings(), M.plan()["tune_ms"]
    pick_full = M.plan()["variant"]
    M.tune("exhaustive")                          # default: racing at 1.3
    raced, t_raced = M.timings(), M.plan()["tune_ms"]
    pick_raced = M.plan()["variant"]
    assert raced[pick_raced] <= 1.15 * full[pick_full], (smat.VARIANT_NAMES[pick_raced], smat.VARIANT_NAMES[pick_full])
    assert t_raced < t_full, (t_raced, t_full)
    # every candidate still has a timing, and the stopped ones are the slow ones
    ran = full > 0
    assert np.array_equal(raced > 0, ran)
    assert raced[pick_raced] <= 1.02 * raced[ran].min()
    M.close()


def _random_rows(m, n, lens, seed):
    rng = np.random.default_rng(seed)
    rp = np.zeros(m + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate([np.sort(rng.choice(n, size=int(k), replace=False)) for k in lens]).astype(np.int32)
    return rp, ci


def test_validation_at_chunk_and_word_boundaries():
    # validation reads the columns 4 at a time and marks row starts in a
    # bitmap of 32-entry words: an order violation placed exactly at those
    # boundaries (and inside a long row, and at the last entries) is caught,
    # and rows starting at them, whose first column is below the previous
    # row's last, are accepted
    m, n = 3000, 5000
    rng = np.random.default_rng(21)
    lens = rng.integers(0, 12, size=m)
    lens[1500] = 2500                      # one long row
    rp, ci = _random_rows(m, n, lens, 22)
    nnz = len(ci)
    st, h = _create(m, n, rp, ci, np.ones(nnz))
    assert st == smat.SMAT_OK
    smat.smat_destroy(h)
    row_of = np.repeat(np.arange(m), np.diff(rp))
    picks = [3, 4, 7, 31, 32, 63, 64, 127, 128, int(rp[1500]) + 1000, int(rp[1500]) + 2047, nnz - 2]
    tried = 0
    for k0 in picks:
        # the nearest k >= k0 whose next entry is in the same row
        k = next((j for j in range(k0, nnz - 1) if row_of[j] == row_of[j + 1]), None)
        if k is None:
            continue
        bad = ci.copy()
        bad[k], bad[k + 1] = bad[k + 1], bad[k]
        st, h = _create(m, n, rp, bad, np.ones(nnz))
        assert st == smat.SMAT_ERR_INVALID_CSR and not h, (k0, k)
        tried += 1
    assert tried >= len(picks) - 1
    # rows that start on word boundaries with a smaller first column
    lens2 = np.full(64, 32, np.int64)
    rp2 = np.zeros(65, np.int32)
    rp2[1:] = np.cumsum(lens2)
    ci2 = np.concatenate([np.arange(2600 - 40 * r, 2632 - 40 * r) for r in range(64)]).astype(np.int32)
    st, h = _create(64, 5000, rp2, ci2, np.ones(len(ci2)))
    assert st == smat.SMAT_OK
    smat.smat_destroy(h)
