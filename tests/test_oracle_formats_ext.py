"""Pins of the oracle's further GPU formats (left to future work in Sec. 8):
HYB (Bell & Garland's ELL + COO split), SELL-C-sigma (Kreutzer et al.), BCSR
with b x b blocks, and SPLIT (long rows in chunks, short rows as COO).  Closed
forms are derived by hand in the comments; the rest is brute force on small
dense matrices."""
import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR

MAKERS = [lambda: synth.stencil2d5(9, 7), lambda: synth.uniform_random(150, 4.0, 1),
          lambda: synth.powerlaw(200, 1.8, 60, 2), lambda: synth.blockdiag(53, 4, 3),
          lambda: synth.stencil3d27(4), lambda: synth.uniform_random(77, 9.0, 5)]


def _from_lengths(lengths, n=None):
    """A CSR matrix whose row i holds lengths[i] entries in columns 0..len-1."""
    lengths = np.asarray(lengths, dtype=np.int64)
    n = int(lengths.max(initial=0)) if n is None else n
    rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    ci = np.concatenate([np.arange(k) for k in lengths]).astype(np.int32) if lengths.sum() else \
        np.zeros(0, np.int32)
    v = np.arange(1, len(ci) + 1, dtype=np.float64)
    return CSR(len(lengths), n, rp, ci, v, "lengths")


# ---------------------------------------------------------------------------
# HYB
# ---------------------------------------------------------------------------

def test_hyb_width_closed_forms():
    # 5-point 64x64: 3844 rows of 5 entries, and 3 * 3844 >= 4096, so K = 5
    # and the COO part is empty
    A = synth.poisson_2d_64()
    assert oracle.hyb_width(A.m, A.rowptr) == 5
    assert len(oracle.to_hyb(A.m, A.rowptr, A.colidx, A.val)[2]) == 0
    # lengths 0,1,1,2,3,10: rows with >= 3 entries: 2, 3*2 >= 6; with >= 4: 1,
    # 3*1 < 6; so K = 3 and the COO part holds the last row's 7 entries past 3
    B = _from_lengths([0, 1, 1, 2, 3, 10])
    ecol, ev, crow, ccol, cv, K, P = oracle.to_hyb(B.m, B.rowptr, B.colidx, B.val)
    assert K == 3 and list(crow) == [5] * 7 and list(ccol) == list(range(3, 10))
    # every row has 8 entries: K = 8
    C = synth.blockdiag(64, 8, 0)
    assert oracle.hyb_width(C.m, C.rowptr) == 8
    # one long row among 99 empty ones: 3 * 1 < 100 for every k >= 1, so K = 0
    assert oracle.hyb_width(100, _from_lengths([0] * 99 + [40]).rowptr) == 0
    assert oracle.hyb_width(0, np.zeros(1, np.int32)) == 0


@pytest.mark.parametrize("mk", MAKERS)
def test_hyb_reconstructs_dense(mk):
    A = mk()
    ecol, ev, crow, ccol, cv, K, P = oracle.to_hyb(A.m, A.rowptr, A.colidx, A.val)
    rl = np.diff(A.rowptr)
    assert len(crow) == int(np.maximum(rl - K, 0).sum())
    ecol, ev = ecol.reshape(K, P), ev.reshape(K, P)
    d = np.zeros((A.m, A.n))
    for s in range(K):
        for i in range(P):
            if ecol[s, i] >= 0:
                d[i, ecol[s, i]] += ev[s, i]
            else:
                assert ev[s, i].view(np.uint64) == 0
    for i in range(A.m):
        assert np.all(ecol[:min(rl[i], K), i] >= 0) and np.all(ecol[min(rl[i], K):, i] == -1)
    for r, c, v in zip(crow, ccol, cv):
        assert d[r, c] == 0  # each entry in exactly one part
        d[r, c] = v
    assert np.all(np.diff(crow) >= 0)
    assert np.array_equal(d, A.todense())


# ---------------------------------------------------------------------------
# SELL-C-sigma
# ---------------------------------------------------------------------------

def test_sell_closed_forms():
    A = synth.poisson_2d_64()
    # sigma = C = 32: slices are half grid rows; the 4 halves of grid rows 0
    # and 63 are 4 wide, the other 124 halves 5 wide: 32 * (4*4 + 124*5)
    assert oracle.sell_layout(A.m, A.rowptr, 32)[2][-1] == 32 * (4 * 4 + 124 * 5) == 20352
    # sigma = 64 sorts inside a grid row: the two corners (3) move to the end
    # but both halves still hold a row of 4 (or 5): the same total
    assert oracle.sell_layout(A.m, A.rowptr, 64)[2][-1] == 20352
    # sigma = 4096 sorts the whole matrix: 3844 rows of 5, 248 of 4, 4 of 3.
    # Positions 0..3871 lie in slices 0..120, all 5 wide (slice 120 starts
    # with the last 4 rows of 5); slices 121..127 are 4 wide.
    perm, width, sptr = oracle.sell_layout(A.m, A.rowptr, 4096)
    assert sptr[-1] == 32 * (121 * 5 + 7 * 4) == 20256
    assert list(width[119:123]) == [5, 5, 4, 4]
    rl = np.diff(A.rowptr)
    assert list(rl[perm[-4:]]) == [3, 3, 3, 3] and list(perm[-4:]) == [0, 63, 4032, 4095]


@pytest.mark.parametrize("mk", MAKERS)
@pytest.mark.parametrize("sigma", [32, 64, 1024])
def test_sell_reconstructs_dense(mk, sigma):
    A = mk()
    C = oracle.SELL_C
    perm, width, sptr, col, val = oracle.to_sell(A.m, A.rowptr, A.colidx, A.val, sigma)
    mp = (A.m + C - 1) // C * C
    rl = np.diff(A.rowptr)
    # perm: inside every window a permutation of the window's rows, longest first
    for w0 in range(0, A.m, sigma):
        w1 = min(w0 + sigma, A.m)
        seg = perm[w0:w1]
        assert sorted(seg) == list(range(w0, w1))
        lens = rl[seg]
        assert np.all(np.diff(lens) <= 0)
        for a, b in zip(seg[:-1], seg[1:]):  # equal lengths keep row order
            if rl[a] == rl[b]:
                assert a < b
    assert np.all(perm[A.m:] == -1) and len(perm) == mp
    ln = np.where(perm >= 0, rl[np.maximum(perm, 0)], 0)
    assert np.array_equal(width, ln.reshape(-1, C).max(axis=1))
    assert np.array_equal(np.diff(sptr), C * width.astype(np.int64))
    d = np.zeros((A.m, A.n))
    for s in range(mp // C):
        for j in range(width[s]):
            for l in range(C):
                slot = sptr[s] + j * C + l
                r = perm[s * C + l]
                if col[slot] >= 0:
                    assert r >= 0 and j < rl[r]
                    d[r, col[slot]] = val[slot]
                else:
                    assert r < 0 or j >= rl[r]
                    assert val[slot].view(np.uint64) == 0
    assert np.array_equal(d, A.todense())


# ---------------------------------------------------------------------------
# BCSR
# ---------------------------------------------------------------------------

def test_bcsr_closed_forms():
    # 5-point 64x64, b = 2: block row I holds rows 2I, 2I+1 of one grid row.
    # Its blocks: I (diagonal) always; I-1 unless the pair starts the grid row
    # (31 of 32 pairs); I+1 unless it ends it (31 of 32); I-32 and I+32
    # unless the grid row is the first / last (63 of 64 grid rows each):
    # 2048 + 2*(64*31) + 2*(63*32)
    A = synth.poisson_2d_64()
    brp, bcol, bval = oracle.to_bcsr(A.m, A.n, A.rowptr, A.colidx, A.val, 2)
    assert len(bcol) == 2048 + 2 * 64 * 31 + 2 * 63 * 32 == 10048
    # 8x8 block diagonal, n = 800: b = 8 -> 100 full blocks; b = 4 -> 2 blocks
    # per 4-row block row (400); b = 2 -> 4 per 2-row block row (1600).
    # Bytes (FP64): 100*516 + 4*101 = 52004; 400*132 + 4*201 = 53604;
    # 1600*36 + 4*401 = 59204 -> b = 8
    B = synth.blockdiag(800, 8, 0)
    for b, nb in ((8, 100), (4, 400), (2, 1600)):
        assert len(oracle.to_bcsr(B.m, B.n, B.rowptr, B.colidx, B.val, b)[1]) == nb
    assert oracle.bcsr_choose(B.m, B.n, B.rowptr, B.colidx, 8) == (8, 100)
    # an empty matrix has no blocks
    brp, bcol, bval = oracle.to_bcsr(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), 4)
    assert len(brp) == 1 and brp[0] == 0 and len(bcol) == 0


def _bcsr_blocks_brute(dense_mask, b):
    m, n = dense_mask.shape
    mb, nbc = -(-m // b), -(-n // b)
    pad = np.zeros((mb * b, nbc * b), dtype=bool)
    pad[:m, :n] = dense_mask
    return pad.reshape(mb, b, nbc, b).any(axis=(1, 3))


@pytest.mark.parametrize("mk", MAKERS + [lambda: synth.uniform_random(13, 3.0, 7)])
@pytest.mark.parametrize("b", [2, 4, 8])
def test_bcsr_reconstructs_dense(mk, b):
    A = mk()
    dense = A.todense()
    brp, bcol, bval = oracle.to_bcsr(A.m, A.n, A.rowptr, A.colidx, A.val, b)
    mask = np.zeros((A.m, A.n), dtype=bool)
    mask[A.row_of_nnz(), A.colidx] = True
    blocks = _bcsr_blocks_brute(mask, b)
    assert np.array_equal(np.diff(brp), blocks.sum(axis=1))
    rec = np.zeros((len(brp) * b, (A.n + b - 1) // b * b + b))
    for I in range(len(brp) - 1):
        js = bcol[brp[I]:brp[I + 1]]
        assert np.all(np.diff(js) > 0) and np.array_equal(js, np.nonzero(blocks[I])[0])
        for k in range(brp[I], brp[I + 1]):
            blk = bval[k * b * b:(k + 1) * b * b].reshape(b, b)
            rec[I * b:I * b + b, bcol[k] * b:bcol[k] * b + b] = blk
    assert np.array_equal(rec[:A.m, :A.n], dense)
    assert not rec[A.m:].any() and not rec[:, A.n:].any()   # +0 past the edges


def test_bcsr_choose_is_the_byte_minimum():
    for mk in MAKERS:
        A = mk()
        for esz in (8, 4, 2):
            b, nb = oracle.bcsr_choose(A.m, A.n, A.rowptr, A.colidx, esz)
            mask = np.zeros((A.m, A.n), dtype=bool)
            mask[A.row_of_nnz(), A.colidx] = True
            cost = {c: int(_bcsr_blocks_brute(mask, c).sum()) * (c * c * esz + 4) + 4 * (-(-A.m // c) + 1)
                    for c in (2, 4, 8)}
            best = min(cost.values())
            assert cost[b] == best and b == min(c for c in cost if cost[c] == best)
            assert nb == int(_bcsr_blocks_brute(mask, b).sum())


# ---------------------------------------------------------------------------
# SPLIT (long rows in chunks + a COO of the short rows)
# ---------------------------------------------------------------------------

def test_split_closed_form():
    # lengths 0, 3, 10, 0, 1, 7 with L = 4, CK = 4: long rows 2 (10 entries ->
    # chunks of 4, 4, 2) and 5 (7 -> 4, 3); short rows 1 and 4 (3 + 1 entries);
    # empty rows 0 and 3
    B = _from_lengths([0, 3, 10, 0, 1, 7])
    s = oracle.split_rows(B.m, B.rowptr, B.colidx, B.val, L=4, CK=4)
    assert list(s["lrows"]) == [2, 5] and list(s["empty"]) == [0, 3]
    assert list(s["crow"]) == [2, 2, 2, 5, 5]
    rp = B.rowptr
    assert list(s["cstart"]) == [rp[2], rp[2] + 4, rp[2] + 8, rp[5], rp[5] + 4]
    assert list(s["cend"]) == [rp[2] + 4, rp[2] + 8, rp[3], rp[5] + 4, rp[6]]
    assert list(s["srow"]) == [1, 1, 1, 4] and list(s["scol"]) == [0, 1, 2, 0]


@pytest.mark.parametrize("mk", MAKERS)
@pytest.mark.parametrize("L", [1, 3, 16, 10 ** 6])
def test_split_reconstructs_dense(mk, L):
    A = mk()
    s = oracle.split_rows(A.m, A.rowptr, A.colidx, A.val, L=L, CK=5)
    rl = np.diff(A.rowptr)
    assert list(s["lrows"]) == list(np.nonzero(rl >= L)[0]) and list(s["empty"]) == list(np.nonzero(rl == 0)[0])
    d = np.zeros((A.m, A.n))
    for r, a, b in zip(s["crow"], s["cstart"], s["cend"]):
        assert 0 < b - a <= 5 and A.rowptr[r] <= a < b <= A.rowptr[r + 1]
        d[r, A.colidx[a:b]] += A.val[a:b]
    for r, c, v in zip(s["srow"], s["scol"], s["sval"]):
        assert rl[r] < L
        d[r, c] += v
    assert np.array_equal(d, A.todense())
    # chunks tile each long row exactly, in order
    for r in s["lrows"]:
        ch = [(a, b) for rr, a, b in zip(s["crow"], s["cstart"], s["cend"]) if rr == r]
        assert ch[0][0] == A.rowptr[r] and ch[-1][1] == A.rowptr[r + 1]
        assert all(ch[k][1] == ch[k + 1][0] for k in range(len(ch) - 1))


def _csr_from_mask(mask):
    rows, cols = np.nonzero(mask)
    rowptr = np.zeros(mask.shape[0] + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    return CSR(mask.shape[0], mask.shape[1], np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32),
               np.ones(len(cols)))


def test_bcsr_choose_breaks_ties_and_counts_row_pointers():
    # a 7 x 11 pattern with 20 blocks of 2x2, 6 of 4x4 and 2 of 8x8: at 4-byte
    # values both 2 and 4 cost 420 bytes (20*20 + 4*5 = 6*68 + 4*3), 8 costs
    # 528: the tie goes to the smaller block
    tie = np.array([[0, 0, 0, 1, 0, 0, 0, 0, 0, 1, 1], [0, 1, 0, 0, 0, 1, 1, 0, 1, 0, 0],
                    [1, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0], [0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 1],
                    [0, 1, 1, 1, 1, 0, 1, 0, 1, 1, 0], [0] * 11, [0, 1, 1, 0, 1, 0, 0, 1, 1, 1, 0]], bool)
    A = _csr_from_mask(tie)
    assert [int(_bcsr_blocks_brute(tie, c).sum()) for c in (2, 4, 8)] == [20, 6, 2]
    assert oracle.bcsr_choose(A.m, A.n, A.rowptr, A.colidx, 4) == (2, 20)
    # an 11 x 4 pattern with 11 / 3 / 2 blocks: at 8-byte values the blocks
    # alone cost 396 for both 2 and 4, and the row pointers (4 * 7 against
    # 4 * 4 bytes) make 4 the smaller: 424 against 412
    rp = np.array([[0, 0, 1, 0], [1, 0, 0, 0], [0, 1, 1, 0], [1, 0, 0, 1], [0, 0, 1, 1], [0, 0, 1, 1],
                   [0, 0, 0, 1], [1, 1, 0, 1], [0, 1, 0, 1], [1, 0, 0, 0], [1, 1, 0, 1]], bool)
    A = _csr_from_mask(rp)
    assert [int(_bcsr_blocks_brute(rp, c).sum()) for c in (2, 4, 8)] == [11, 3, 2]
    assert oracle.bcsr_choose(A.m, A.n, A.rowptr, A.colidx, 8) == (4, 3)
