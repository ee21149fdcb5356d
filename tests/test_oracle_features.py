"""Pins of the oracle's feature parameters (Sec. 4, Table "Feature parameters
of a sparse matrix") to closed forms, brute force and exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR


def feats(A, tau=(3, 5)):
    return oracle.features(A.m, A.n, A.rowptr, A.colidx, tau)


def rn(num, den):
    """Correctly rounded double of the exact rational num/den."""
    return float(Fraction(num, den)) if den else 0.0


@pytest.mark.parametrize("mx,my", [(64, 64), (7, 3), (2, 9), (1, 5)])
def test_5pt_closed_form(mx, my):
    A = synth.stencil2d5(mx, my)
    f = feats(A)
    M = mx * my
    nnz = 5 * M - 2 * mx - 2 * my
    assert (f["m"], f["n"], f["nnz"]) == (M, M, nnz)
    # degrees: 5 inside, minus one per missing neighbour
    deg = np.full((my, mx), 5)
    deg[0, :] -= 1; deg[-1, :] -= 1; deg[:, 0] -= 1; deg[:, -1] -= 1
    assert f["max_rd"] == deg.max() and f["min_rd"] == deg.min()
    s2 = int((deg.astype(np.int64) ** 2).sum())
    assert f["s2"] == s2
    assert f["aver_rd"] == rn(nnz, M)
    assert f["var_rd"] == rn(M * s2 - nnz * nnz, M * M)
    offs = {0}
    if mx > 1: offs |= {-1, 1}
    if my > 1: offs |= {-mx, mx}
    assert f["ndiags"] == len(offs)
    assert f["er_dia"] == rn(nnz, len(offs) * M)
    assert f["er_ell"] == rn(nnz, int(deg.max()) * M)


def test_5pt_64_values():
    f = feats(synth.poisson_2d_64())
    assert f["nnz"] == 20224 and f["aver_rd"] == 4.9375
    assert list(f["hist"]) == [0, 0, 0, 4, 248, 3844]
    assert f["var_rd"] == 0.060546875            # exactly 248/4096
    assert f["ndiags"] == 5 and f["ntdiags"] == 5 and f["ntdiags_ratio"] == 1.0
    assert f["er_dia"] == 0.9875 and f["er_ell"] == 0.9875


@pytest.mark.parametrize("m", [3, 6, 11])
def test_3d7_closed_form(m):
    f = feats(synth.stencil3d7(m))
    i = m - 2
    assert f["nnz"] == 7 * m ** 3 - 6 * m ** 2
    assert list(f["hist"][4:]) == [8, 12 * i, 6 * i * i, i ** 3]
    assert (f["max_rd"], f["min_rd"], f["ndiags"]) == (7, 4, 7)


@pytest.mark.parametrize("m", [3, 5, 8])
def test_3d27_closed_form(m):
    f = feats(synth.stencil3d27(m))
    assert f["nnz"] == (3 * m - 2) ** 3
    assert (f["max_rd"], f["min_rd"], f["ndiags"]) == (27, 8, 27)


def test_blockdiag_closed_form():
    n = 8000
    f = feats(synth.blockdiag(n, 8, 0))
    assert (f["max_rd"], f["min_rd"], f["var_rd"], f["er_ell"]) == (8, 8, 0.0, 1.0)
    assert f["ndiags"] == 15 and f["er_dia"] == rn(8 * n, 15 * n)
    # diagonal d holds (8-|d|) n/8 of its n-|d| positions: "true" at 3/5 iff |d| <= 3
    assert f["ntdiags"] == 7
    assert f["r_valid"] == 0 and f["r"] == 0.0


def _brute(d, tau):
    """Features by a dense scan, written independently of the oracle."""
    m, n = d.shape
    nz = d != 0
    rd = nz.sum(axis=1).astype(np.int64)
    nnz = int(rd.sum())
    cnt = {}
    for i in range(m):
        for j in range(n):
            if nz[i, j]:
                cnt[j - i] = cnt.get(j - i, 0) + 1
    def dlen(dd):
        return sum(1 for i in range(m) if 0 <= i + dd < n)
    true = sum(1 for dd, c in cnt.items() if tau[1] * c > tau[0] * dlen(dd))
    s2 = int((rd * rd).sum())
    return dict(nnz=nnz, max_rd=int(rd.max()), min_rd=int(rd.min()), ndiags=len(cnt), ntdiags=true,
                s2=s2, hist=np.bincount(rd), aver_rd=rn(nnz, m), var_rd=rn(m * s2 - nnz * nnz, m * m),
                er_dia=rn(nnz, len(cnt) * m), er_ell=rn(nnz, int(rd.max()) * m),
                ntdiags_ratio=rn(true, len(cnt)))


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    m, n = rng.integers(1, 40, size=2)
    d = rng.standard_normal((m, n)) * (rng.random((m, n)) < rng.uniform(0.05, 0.9))
    rows, cols = np.nonzero(d)
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    A = CSR(m, n, np.cumsum(rp).astype(np.int32), cols.astype(np.int32), d[rows, cols])
    tau = [(3, 5), (1, 2), (1, 10)][seed % 3]
    f, b = feats(A, tau), _brute(d, tau)
    for k, v in b.items():
        if k == "hist":
            assert np.array_equal(f["hist"], v)
        else:
            assert f[k] == v, k


def test_true_diagonal_is_strict():
    # 10x10 with diagonal 0 holding 6 of 10 entries: 5*6 = 3*10, not "true" at 3/5
    d = np.zeros((10, 10))
    d[np.arange(6), np.arange(6)] = 1.0
    rows, cols = np.nonzero(d)
    rp = np.zeros(11, np.int64)
    np.add.at(rp, rows + 1, 1)
    A = CSR(10, 10, np.cumsum(rp).astype(np.int32), cols.astype(np.int32), d[rows, cols])
    assert feats(A)["ntdiags"] == 0
    d[6, 6] = 1.0
    rows, cols = np.nonzero(d)
    rp = np.zeros(11, np.int64)
    np.add.at(rp, rows + 1, 1)
    A = CSR(10, 10, np.cumsum(rp).astype(np.int32), cols.astype(np.int32), d[rows, cols])
    assert feats(A)["ntdiags"] == 1


def test_power_law_fit_against_polyfit():
    A = synth.powerlaw(50000, 1.8, 2000, 3)
    f = feats(A)
    h = f["hist"]
    k = np.nonzero(h)[0]
    k = k[k >= 1]
    slope = np.polyfit(np.log(k), np.log(h[k].astype(float)), 1)[0]
    assert f["r_valid"] == 1
    assert abs(f["r"] + slope) <= 1e-9 * abs(slope)
    assert 1.0 <= f["r"] < 4.0 or f["r"] > 0  # a heavy tail gives a positive exponent


def test_power_law_two_points_closed_form():
    # rows of degree 2 (x12) and degree 6 (x3): R = -(ln 3 - ln 12)/(ln 6 - ln 2)
    rl = [2] * 12 + [6] * 3
    rp = np.concatenate([[0], np.cumsum(rl)]).astype(np.int32)
    col = np.concatenate([np.arange(r) for r in rl]).astype(np.int32)
    A = CSR(15, 10, rp, col, np.ones(len(col)))
    f = feats(A)
    want = -(np.log(3.0) - np.log(12.0)) / (np.log(6.0) - np.log(2.0))
    assert f["r_valid"] == 1 and abs(f["r"] - want) <= 8 * np.finfo(float).eps * abs(want)


def test_degenerate_matrices():
    A = CSR(4, 6, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    f = feats(A)
    assert (f["nnz"], f["max_rd"], f["min_rd"], f["ndiags"], f["empty_rows"]) == (0, 0, 0, 0, 4)
    assert (f["aver_rd"], f["var_rd"], f["er_dia"], f["er_ell"], f["r_valid"]) == (0.0, 0.0, 0.0, 0.0, 0)
    # one dense row among empty ones
    rp = np.array([0, 0, 7, 7], np.int32)
    B = CSR(3, 7, rp, np.arange(7, dtype=np.int32), np.ones(7))
    g = feats(B)
    assert (g["max_rd"], g["min_rd"], g["empty_rows"], g["ndiags"]) == (7, 0, 2, 7)
    assert g["var_rd"] == rn(3 * 49 - 49, 9)
