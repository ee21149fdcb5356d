"""Pins of the Galerkin AMG hierarchy generator (input generation for the
batched path; the AMG setting is the paper's motivation, Sec. 1): the coarse
operators against a dense brute-force P^T A P, symmetry, stencil widths and
the vanishing row sums away from the boundary."""
import numpy as np
import pytest

pytest.importorskip("scipy")
from paper_1210_2536_gb300 import synth


def _dense(A):
    return A.todense()


def _dense_prolongator(m, A, omega):
    # written out from the definition: point (x, y, z) -> box aggregate
    # (x//2, y//2, z//2); then one damped-Jacobi smoothing step
    mc = (m + 1) // 2
    P0 = np.zeros((m ** 3, mc ** 3))
    for z in range(m):
        for y in range(m):
            for x in range(m):
                P0[x + m * y + m * m * z, x // 2 + mc * (y // 2) + mc * mc * (z // 2)] = 1.0
    D = _dense(A)
    return P0 - omega * (D / np.diag(D)[:, None]) @ P0


@pytest.mark.parametrize("m", [4, 5, 7])
def test_coarse_operator_is_dense_ptap(m):
    H = synth.galerkin_hierarchy(m, 3)
    A0, A1 = H[0], H[1]
    P = _dense_prolongator(m, A0, 2.0 / 3.0)
    ref = P.T @ _dense(A0) @ P
    got = _dense(A1)
    assert got.shape == ref.shape == (((m + 1) // 2) ** 3,) * 2
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-12 * np.abs(ref).max())
    # the stored pattern is exactly the structural product's (no entry lost)
    assert np.all((np.abs(ref) > 1e-12 * np.abs(ref).max()) <= (got != 0) | (np.abs(ref) <= 1e-12))
    if len(H) > 2:
        mc = (m + 1) // 2
        P1 = _dense_prolongator(mc, A1, 2.0 / 3.0)
        assert np.allclose(_dense(H[2]), P1.T @ got @ P1, rtol=1e-12, atol=1e-11 * np.abs(got).max())


def test_levels_are_symmetric_canonical_and_widen():
    import scipy.sparse as sp
    H = synth.galerkin_hierarchy(12, 5)
    assert [A.m for A in H] == [12 ** 3, 6 ** 3, 3 ** 3, 2 ** 3, 1]
    widths = []
    for A in H:
        rl = np.diff(A.rowptr)
        for i in range(A.m):  # canonical CSR: strictly increasing columns
            assert np.all(np.diff(A.colidx[A.rowptr[i]:A.rowptr[i + 1]]) > 0)
        S = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.m, A.n))
        assert abs(S - S.T).max() <= 1e-12 * abs(S).max()
        widths.append(int(rl.max()))
    # 27-point fine stencil; a 2x2x2 aggregate smoothed once covers 4 fine
    # points per direction, so coarse points couple within distance 2: 5^3 =
    # 125 on level 1 (6^3, whose middle points are 2 from every face); the
    # 3^3 and 2^3 levels are coupled all to all
    assert widths == [27, 125, 27, 8, 1]


def test_interior_coarse_row_sums_vanish():
    # A 1 = 0 at fine points away from the boundary (26 - 26 neighbours), so
    # P 1 = 1 there and (P^T A P 1)_c = 0 for coarse points whose support
    # (the aggregate widened by 2 fine points and its neighbours') avoids it
    m = 24
    H = synth.galerkin_hierarchy(m, 2)
    A1 = H[1]
    mc = m // 2
    s = A1.todense().sum(axis=1)
    scale = np.abs(A1.todense()).sum(axis=1)
    for c in range(A1.m):
        x, y, z = c % mc, (c // mc) % mc, c // (mc * mc)
        if min(x, y, z) >= 2 and max(x, y, z) <= mc - 3:
            assert abs(s[c]) <= 1e-13 * scale[c], c
    assert np.max(np.abs(s)) > 1e-3   # boundary rows keep a positive sum
