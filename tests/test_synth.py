"""The seeded input generators: Philox known answers, structure, determinism."""
import os

import numpy as np
import pytest

from paper_1210_2536_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert synth.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def _check_canonical(A):
    rp = A.rowptr.astype(np.int64)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(A.colidx)
    for i in range(A.m):
        c = A.colidx[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0)
        if len(c):
            assert c[0] >= 0 and c[-1] < A.n


@pytest.mark.parametrize("maker", [
    lambda: synth.stencil2d5(7, 5), lambda: synth.stencil3d7(5), lambda: synth.stencil3d27(4),
    lambda: synth.uniform_random(300, 6.0, 3), lambda: synth.powerlaw(400, 1.8, 100, 4),
    lambda: synth.blockdiag(37, 8, 5), lambda: synth.uniform_random(50, 40.0, 1),
    lambda: synth.box3d(6, 2), lambda: synth.box3d(5, 4),
])
def test_canonical_csr(maker):
    _check_canonical(maker())


def test_thread_count_does_not_change_output():
    for kind, p in [(synth.POWERLAW, [20000, 1.8, 1000]), (synth.UNIFORM, [20000, 9.0])]:
        a = synth.generate(kind, p, 11, nthreads=1)
        b = synth.generate(kind, p, 11, nthreads=5)
        assert np.array_equal(a.rowptr, b.rowptr)
        assert np.array_equal(a.colidx, b.colidx)
        assert np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))


def test_stencil_values_and_sizes():
    A = synth.stencil2d5(64, 64)
    assert (A.m, A.nnz) == (4096, 20224)
    d = A.todense()
    assert np.all(np.diag(d) == 4.0)
    assert set(np.unique(d[d != 0])) == {-1.0, 4.0}
    assert np.array_equal(d, d.T)
    B = synth.stencil3d27(6)
    assert B.nnz == (3 * 6 - 2) ** 3


def test_distributions_close_to_their_means():
    A = synth.uniform_random(200000, 16.0, 0)
    assert abs(A.nnz / A.m - 16.0) < 0.05
    # truncated Zipf(1.8) on [1, 1e4]: mean from the definition
    k = np.arange(1, 10001, dtype=np.float64)
    w = k ** -1.8
    mean = float((w * k).sum() / w.sum())
    assert abs(synth.zipf_mean(1.8, 10000) - mean) < 1e-9 * mean
    P = synth.powerlaw(400000, 1.8, 10000, 0)
    assert abs(P.nnz / P.m - mean) / mean < 0.05
    v = P.val
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01
    x = synth.uniform(0, 1, 100001)
    assert x.min() >= -1.0 and x.max() < 1.0 and abs(x.mean()) < 0.01


def test_dataset_specs_cover_all_kinds():
    kinds = {synth.dataset_spec(i)[0] for i in range(200)}
    assert kinds == set(range(6))
    assert synth.dataset_spec(synth.DATASET_PRIMARY)[0] == synth.BOX3D


def test_box_stencil_closed_forms():
    # radius 1 is the 27-point stencil, bit for bit
    a, b = synth.box3d(7, 1), synth.stencil3d27(7)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.colidx, b.colidx)
    assert np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))
    for m, r in [(9, 2), (6, 3), (4, 5)]:
        A = synth.box3d(m, r)
        # points within r of c on a line of m points, cubed over the three axes
        line = sum(min(c + r, m - 1) - max(c - r, 0) + 1 for c in range(m))
        assert (A.m, A.nnz) == (m ** 3, line ** 3)
        d = A.todense()
        assert np.array_equal(d, d.T)
        w = (2 * r + 1) ** 3
        assert np.all(np.diag(d) == w - 1.0)
        # every off-diagonal entry is -1, and the pattern is |di|,|dj|,|dk| <= r
        g = np.indices((m, m, m)).reshape(3, -1)[::-1].T       # (x, y, z) of each row, x fastest
        near = np.all(np.abs(g[:, None, :] - g[None, :, :]) <= r, axis=2)
        assert np.array_equal(d != 0, near)
        off = d[near & ~np.eye(m ** 3, dtype=bool)]
        assert np.all(off == -1.0)
        # rows with the whole box inside the grid sum to zero
        full = np.diff(A.rowptr) == w
        assert np.all(d[full].sum(axis=1) == 0.0)


def test_galerkin_levels_have_box_stencil_patterns():
    # the widened labelled set stands in for coarse multigrid operators: their
    # sparsity patterns are box stencils whose radius grows level by level
    H = synth.galerkin_hierarchy(32, 4)
    for A, (m, r) in zip(H, [(32, 1), (16, 2), (8, 3), (4, 3)]):
        B = synth.box3d(m, r)
        assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.colidx, B.colidx)


def test_widened_dataset_specs():
    from collections import Counter
    specs = [synth.dataset_spec(i) for i in range(synth.DATASET_PRIMARY, synth.DATASET_SIZE)]
    assert {k for k, _, _ in specs} == {synth.BOX3D}
    radii = Counter(int(p[1]) for _, p, _ in specs)
    assert set(radii) == {2, 3, 4, 5, 6} and min(radii.values()) >= 50
    for _, (m, r), seed in specs:
        assert m >= 8 and m ** 3 * (2 * r + 1) ** 3 <= 5e7 * 1.05   # nnz bound (before boundary truncation)
