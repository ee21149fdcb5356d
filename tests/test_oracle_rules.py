"""Pins of the oracle's admissibility filter (Sec. 2.3) and of the paper's
observations as an ordered rule set (Sec. 4, order of Sec. 6): matrices whose
features follow in closed form, the paper's own consequence of the 20x rule
(at least 5 % of the stored slots are entries), and each rule's boundary."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth
from helpers import csr_from_degrees as from_degrees

C = {name: i for i, name in enumerate(oracle.CLASSES)}
ALWAYS = sum(1 << C[c] for c in ("csr_scalar", "csr_vec4", "csr_vec8", "csr_vec32", "csr_merge", "coo"))
ALL8 = (1 << 8) - 1


@pytest.fixture(params=[8, 4, 2], ids=["f64", "f32", "bf16"])
def vb(request):
    """Value bytes of the storage type: the byte cap, and so the mask, depend on it."""
    return request.param


def pick(A, value_bytes=8):
    f = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    mask = oracle.admissible(A.m, A.nnz, f["max_rd"], f["ndiags"], value_bytes)
    return oracle.rules_select(f, mask), mask, f


# --- matrices whose choice the paper states ---------------------------------

@pytest.mark.parametrize("make", [lambda: synth.stencil2d5(64), lambda: synth.stencil3d7(12),
                                  lambda: synth.stencil3d27(16), lambda: synth.blockdiag(4096, 8, 0)])
def test_banded_matrices_take_dia(make, vb):
    # 5, 7 and 15 diagonals are fewer than 25; the 27-point operator has 27
    # but 88 % of its DIA slots hold entries ((46/48)^3 for 16^3), above 60 %
    A = make()
    v, mask, f = pick(A, vb)
    assert mask == ALL8
    assert v == C["dia"], (A.name, f["ndiags"], f["er_dia"])


def test_27_point_needs_the_fill_observation():
    A = synth.stencil3d27(16)
    f = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    assert f["ndiags"] == 27 and f["er_dia"] == float(Fraction(46 ** 3, 27 * 16 ** 3))
    g = dict(f, er_dia=0.5, ntdiags_ratio=0.3)   # neither fill observation holds: no DIA
    assert oracle.rules_select(g, ALL8) != C["dia"]


def test_constant_short_rows_take_ell(vb):
    # three random columns per row: far more than 20 x 3 diagonals (no DIA),
    # max_RD 3 < 5 and var_RD 0 (ELL)
    A = from_degrees([3] * 5000, 5000, 1)
    v, mask, f = pick(A, vb)
    assert not (mask >> C["dia"]) & 1 and (mask >> C["ell"]) & 1
    assert (f["max_rd"], f["var_rd"], f["er_ell"]) == (3, 0.0, 1.0)
    assert v == C["ell"]


def test_constant_long_rows_take_ell_by_fill(vb):
    # 12 per row: max_RD >= 5 but ER_ELL = 100 % > 90 % and var_RD = 0
    A = from_degrees([12] * 3000, 3000, 2)
    assert pick(A, vb)[0] == C["ell"]


@pytest.mark.parametrize("degs,lanes", [((2, 6), "csr_vec4"), ((10, 14), "csr_vec8"), ((30, 34), "csr_vec32")])
def test_two_row_lengths_take_csr_by_mean(degs, lanes, vb):
    # rows alternate between two lengths: var_RD = 4 (no ELL), and the two
    # histogram points have equal counts, so the fitted R is 0 (no COO)
    A = from_degrees([degs[i % 2] for i in range(4000)], 4000, 3)
    v, mask, f = pick(A, vb)
    assert f["var_rd"] == 4.0 and f["r_valid"] == 1 and abs(f["r"]) < 1e-9
    assert v == C[lanes]


def _power_histogram_matrix(h, n, seed):
    deg = [k for k, cnt in sorted(h.items()) for _ in range(cnt)]
    order = np.random.default_rng(seed).permutation(len(deg))
    return from_degrees(np.asarray(deg)[order], n, seed)


@pytest.mark.parametrize("h,R,want", [
    ({1: 640, 2: 160, 4: 40, 8: 10}, 2.0, "coo"),       # h[k] = 640 k^-2: small world
    ({1: 512, 4: 64, 16: 8}, 1.5, "coo"),              # 8x fewer rows per 4x length
    ({2: 512, 4: 64, 8: 8}, 3.0, "coo"),                # 8x fewer rows per 2x length
    ({2: 1024 * 3, 4: 32 * 3, 8: 3}, 5.0, None),        # R = 5: not small world -> CSR
    ({1: 400, 4: 200, 16: 100}, 0.5, None),             # R = 1/2: not small world -> CSR
])
def test_power_law_degree_histogram(h, R, want, vb):
    # an exact power law h[k] ~ k^-R: the fit returns R up to rounding; the
    # mixed lengths defeat ELL (max_RD >= 5 and ER_ELL < 90 %, or var_RD > 0.5)
    A = _power_histogram_matrix(h, 6000, 4)
    v, mask, f = pick(A, vb)
    assert abs(f["r"] - R) < 1e-12 and f["r_valid"] == 1
    assert not (mask >> C["dia"]) & 1
    if want:
        assert v == C[want]
    else:
        assert v in (C["csr_vec4"], C["csr_vec8"], C["csr_vec32"])


def test_power_law_network_is_small_world(vb):
    # the generator's truncated Zipf(1.8) rows up to 1000 entries: neither
    # zero-filling format is admissible, and the fitted R lands in [1, 4)
    A = synth.powerlaw(20000, 1.8, 1000, 3)
    v, mask, f = pick(A, vb)
    assert mask == ALWAYS
    assert 1.0 <= f["r"] < 4.0
    assert v == C["coo"]


# --- the admissibility filter ------------------------------------------------

def test_fill_rule_keeps_five_percent_entries():
    # Sec. 2.3: the 20x limit means at least 5 % of the stored slots are entries
    rng = np.random.default_rng(7)
    seen = {"ell": 0, "dia": 0}
    dropped = {"ell": 0, "dia": 0}
    for t in range(60):
        m = int(rng.integers(50, 400))
        band = int(rng.integers(1, 60))
        busy = (1.0, 0.3, 0.05, 0.01)[t % 4]   # share of rows that hold entries
        deg, cols = [], []
        for i in range(m):
            lo, hi = max(0, i - band), min(m, i + band + 1)
            k = int(rng.integers(1, hi - lo + 1)) if rng.random() < busy else 0
            deg.append(k)
            cols.append(np.sort(rng.choice(np.arange(lo, hi), size=k, replace=False)))
        rowptr = np.zeros(m + 1, np.int32)
        rowptr[1:] = np.cumsum(deg)
        colidx = np.concatenate(cols).astype(np.int32)
        f = oracle.features(m, m, rowptr, colidx)
        mask = oracle.admissible(m, int(rowptr[-1]), f["max_rd"], f["ndiags"], 8, bytes_cap=1e18)
        if (mask >> C["ell"]) & 1:
            seen["ell"] += 1
            assert f["er_ell"] >= 0.05
        else:
            dropped["ell"] += 1
            assert f["nnz"] == 0 or f["er_ell"] < 0.05
        if (mask >> C["dia"]) & 1:
            seen["dia"] += 1
            assert f["er_dia"] >= 0.05
        else:
            dropped["dia"] += 1
            assert f["nnz"] == 0 or f["er_dia"] < 0.05
    assert min(seen.values()) >= 5 and min(dropped.values()) >= 5, (seen, dropped)


@pytest.mark.parametrize("vb", [8, 4, 2])
def test_fill_rule_boundary_in_integers(vb):
    # max_RD * M = 20 NNZ is admissible, one more slot is not
    m, nnz = 100, 500
    big = 1e18
    assert (oracle.admissible(m, nnz, 100, 1, vb, bytes_cap=big) >> C["ell"]) & 1
    assert not (oracle.admissible(m, nnz, 101, 1, vb, bytes_cap=big) >> C["ell"]) & 1
    assert (oracle.admissible(m, nnz, 1, 100, vb, bytes_cap=big) >> C["dia"]) & 1
    assert not (oracle.admissible(m, nnz, 1, 101, vb, bytes_cap=big) >> C["dia"]) & 1


def _comb(m, k, stride=20):
    # row i stores the columns i + d, d = i (mod stride), 0 <= d < k: every
    # offset 0..k-1 occurs, so Ndiags = k, and with m a multiple of stride the
    # rows hold k entries in all per residue class: NNZ = (m / stride) k
    rows, cols = [], []
    for i in range(m):
        c = [i + d for d in range(i % stride, k, stride)]
        rows.append(len(c))
        cols.extend(c)
    rowptr = np.zeros(m + 1, np.int32)
    rowptr[1:] = np.cumsum(rows)
    return rowptr, np.asarray(cols, np.int32)


@pytest.mark.parametrize("vb", [8, 4, 2])
def test_dia_offset_cap_on_the_fill_boundary(vb):
    # 100 rows, 8192 and 8193 diagonals: NNZ = 5 k, so Ndiags * M = 20 NNZ
    # exactly and the fill rule admits both; the 8192-offset reading drops the
    # second.  The byte cap is lifted so that only those two rules act.
    m, big = 100, 1e18
    for k, admitted in ((8192, True), (8193, False)):
        rowptr, colidx = _comb(m, k)
        f = oracle.features(m, m + k, rowptr, colidx)
        nnz = int(rowptr[-1])
        assert (f["ndiags"], nnz) == (k, 5 * k) and f["ndiags"] * m == 20 * nnz
        got = (oracle.admissible(m, nnz, f["max_rd"], f["ndiags"], vb, bytes_cap=big) >> C["dia"]) & 1
        assert got == admitted, k
        assert (oracle.admissible(m, nnz, f["max_rd"], f["ndiags"], vb, bytes_cap=big,
                                  dia_max_offsets=10 ** 9) >> C["dia"]) & 1


@pytest.mark.parametrize("vb,ell_from,dia_from", [(8, 208, 129), (4, 192, 73), (2, 176, 48)])
def test_default_byte_cap_thresholds_per_storage_type(vb, ell_from, dia_from):
    # M = P = 96 rows, max_RD = Ndiags = 10, default cap 4x the CSR bytes
    # (vb + 4) NNZ + 388.  Worked by hand: ELL moves (vb + 4) 960 bytes, so it
    # enters at NNZ 208 / 192 / 176 (FP64 / FP32 / BF16); DIA moves
    # 960 vb + 40 bytes and enters at 129 / 73 by the cap, while for BF16 the
    # fill rule (960 <= 20 NNZ) binds first, at 48
    m = 96
    for nnz in range(40, 260):
        mask = oracle.admissible(m, nnz, 10, 10, vb)
        assert ((mask >> C["ell"]) & 1) == (nnz >= ell_from), (vb, nnz)
        assert ((mask >> C["dia"]) & 1) == (nnz >= dia_from), (vb, nnz)


def test_byte_cap_binds_inside_the_fill_rule():
    # one row in ten holds ten times the mean: the fill rule admits ELL
    # (max_RD * M = 10 NNZ) but the padded arrays move ~10x the CSR bytes
    deg = [50 if i % 10 == 0 else 5 for i in range(2000)]   # mean 9.5, max 50
    A = from_degrees(deg, 2000, 5)
    f = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    assert f["max_rd"] * A.m <= 20 * A.nnz
    assert (oracle.admissible(A.m, A.nnz, f["max_rd"], f["ndiags"], 8, bytes_cap=1e18) >> C["ell"]) & 1
    for vb in (8, 4, 2):
        assert not (oracle.admissible(A.m, A.nnz, f["max_rd"], f["ndiags"], vb) >> C["ell"]) & 1


def test_byte_caps_count_the_padded_pitch():
    # 7-point stencil on 10^3 (M = 1000, pitch P = 1024) against (s + 4) NNZ
    # + 4 (M + 1) CSR bytes: DIA moves 7 P values and 7 offsets, ELL 7 P
    # values and columns; with a cap just below either ratio the format drops
    A = synth.stencil3d7(10)
    P = oracle.pitch(A.m)
    assert P == 1024 != A.m
    for vb in (8, 4, 2):
        csr = (vb + 4) * A.nnz + 4 * (A.m + 1)
        for name, byts in (("dia", vb * 7 * P + 4 * 7), ("ell", (vb + 4) * 7 * P)):
            ratio = byts / csr
            assert (oracle.admissible(A.m, A.nnz, 7, 7, vb, bytes_cap=ratio) >> C[name]) & 1
            assert not (oracle.admissible(A.m, A.nnz, 7, 7, vb, bytes_cap=ratio * (1 - 1e-9)) >> C[name]) & 1


def test_empty_and_degenerate_matrices(vb):
    assert oracle.admissible(0, 0, 0, 0, 8) == ALWAYS
    assert oracle.admissible(10, 0, 0, 0, 8) == ALWAYS
    A = from_degrees([0] * 10, 10, 0)
    v, mask, f = pick(A, vb)
    assert mask == ALWAYS and v == C["csr_vec4"]


# --- rule order and boundaries -------------------------------------------------

def _f(**kw):
    base = dict(aver_rd=12.0, max_rd=40, var_rd=9.0, ndiags=900, er_dia=0.1, er_ell=0.3,
                ntdiags_ratio=0.1, r=0.2, r_valid=1)
    base.update(kw)
    return base


def test_rule_boundaries():
    assert oracle.rules_select(_f(ndiags=24), ALL8) == C["dia"]
    assert oracle.rules_select(_f(ndiags=25), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(ndiags=500, er_dia=0.61), ALL8) == C["dia"]
    assert oracle.rules_select(_f(ndiags=501, er_dia=1.0, ntdiags_ratio=1.0), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(ndiags=100, er_dia=0.6), ALL8) == C["csr_vec8"]          # strictly above 60 %
    assert oracle.rules_select(_f(ndiags=100, ntdiags_ratio=0.41), ALL8) == C["dia"]
    assert oracle.rules_select(_f(ndiags=100, ntdiags_ratio=0.4), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(max_rd=4, var_rd=0.49), ALL8) == C["ell"]
    assert oracle.rules_select(_f(max_rd=4, var_rd=0.5), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(max_rd=5, var_rd=0.0), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(er_ell=0.91, var_rd=0.1), ALL8) == C["ell"]
    assert oracle.rules_select(_f(er_ell=0.9, var_rd=0.1), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(r=1.0), ALL8) == C["coo"]
    assert oracle.rules_select(_f(r=3.999), ALL8) == C["coo"]
    assert oracle.rules_select(_f(r=4.0), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(r=2.0, r_valid=0), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(aver_rd=7.99), ALL8) == C["csr_vec4"]
    assert oracle.rules_select(_f(aver_rd=8.0), ALL8) == C["csr_vec8"]
    assert oracle.rules_select(_f(aver_rd=24.0), ALL8) == C["csr_vec32"]


def test_rule_order_and_inadmissible_formats():
    both = _f(ndiags=10, max_rd=3, var_rd=0.0, r=2.0)
    assert oracle.rules_select(both, ALL8) == C["dia"]                     # DIA is tried first
    assert oracle.rules_select(both, ALL8 & ~(1 << C["dia"])) == C["ell"]  # then ELL
    assert oracle.rules_select(both, ALWAYS) == C["coo"]                   # then COO before CSR
    only_scalar = 1 << C["csr_scalar"]
    assert oracle.rules_select(_f(), only_scalar) == C["csr_scalar"]


def test_no_admissible_class_is_an_error():
    with pytest.raises(ValueError):
        oracle.rules_select(_f(), 0)
