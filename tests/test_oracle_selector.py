"""Pins of the oracle's learned-selector decision: its 12 inputs on a matrix
whose features are known in closed form, the clamp of R, and the pick through
networks whose logits are known (output bias only; a network whose logits are
its standardised inputs)."""
import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth

C = {name: i for i, name in enumerate(oracle.CLASSES)}
ALL8 = (1 << 8) - 1
NP = oracle.mlp_param_count()


def test_inputs_of_the_5_point_64x64():
    A = synth.poisson_2d_64()
    f = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    x = oracle.selector_inputs(f)
    # degrees: 4 corners of 3, 248 edge rows of 4, 3844 interior rows of 5
    k, h = np.array([3.0, 4.0, 5.0]), np.array([4.0, 248.0, 3844.0])
    R = -np.polyfit(np.log(k), np.log(h), 1)[0]
    want = [np.log(4097.0), np.log(4097.0), np.log(20225.0), np.log(5.9375), np.log(6.0), np.log(4.0),
            np.log1p(248.0 / 4096.0), np.log(6.0), 1.0, 0.9875, 0.9875, R]
    assert np.allclose(x, want, rtol=1e-14, atol=1e-13)
    assert x[8:11].tolist() == [1.0, 0.9875, 0.9875]


def test_inputs_of_a_small_rectangular_matrix():
    # rows {0, 4}, {1, 2, 3}, {2, 4} of a 3 x 5 matrix: NNZ 7, degrees 2, 3, 2
    # (var_RD = (3 * 17 - 49) / 9), diagonals j - i in {0, 1, 2, 4} of which
    # 0, 2 and 4 hold more than 3/5 of their positions, histogram h[2] = 2,
    # h[3] = 1 (R = ln 2 / ln 1.5)
    rowptr = np.array([0, 2, 5, 7], np.int32)
    colidx = np.array([0, 4, 1, 2, 3, 2, 4], np.int32)
    f = oracle.features(3, 5, rowptr, colidx)
    x = oracle.selector_inputs(f)
    want = [np.log1p(3), np.log1p(5), np.log1p(7), np.log1p(7 / 3), np.log1p(3), np.log1p(2), np.log1p(2 / 9),
            np.log1p(4), 0.75, 7 / 12, 7 / 9, np.log(2) / np.log(1.5)]
    assert np.allclose(x, want, rtol=1e-14, atol=0)


def test_r_input_is_clamped_and_zero_when_undefined():
    A = synth.poisson_2d_64()
    f = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    assert oracle.selector_inputs(dict(f, r=1e6))[11] == 100.0
    assert oracle.selector_inputs(dict(f, r=-1e6))[11] == -100.0
    assert oracle.selector_inputs(dict(f, r=3.5, r_valid=0))[11] == 0.0
    # an empty matrix: every count 0 and log(1 + 0) = 0
    E = oracle.features(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert np.array_equal(oracle.selector_inputs(E), np.zeros(12))


def _bias_net(b):
    p = np.zeros(NP)
    p[-8:] = b
    return p


def test_output_bias_gives_softmax_over_admissible():
    f = oracle.features(10, 10, np.arange(11, dtype=np.int32), np.arange(10, dtype=np.int32))
    b = np.array([0.0, 1.0, 2.0, 0.5, -1.0, 3.0, 2.5, 0.0])
    v, p = oracle.learned_select(f, ALL8, _bias_net(b), np.zeros(12), np.ones(12))
    e = np.exp(b - b.max())
    assert v == C["ell"] and np.allclose(p, e / e.sum(), rtol=1e-15)
    mask = ALL8 & ~(1 << C["ell"])
    v, p = oracle.learned_select(f, mask, _bias_net(b), np.zeros(12), np.ones(12))
    live = np.array([(mask >> c) & 1 for c in range(8)], bool)
    e = np.where(live, np.exp(b - b[live].max()), 0.0)
    assert v == C["dia"] and p[C["ell"]] == 0.0 and np.allclose(p, e / e.sum(), rtol=1e-15)
    # equal logits: the lowest id wins, each admissible class has 1/k
    v, p = oracle.learned_select(f, 0b10100100, _bias_net(np.zeros(8)), np.zeros(12), np.ones(12))
    assert v == 2 and np.allclose(p[[2, 5, 7]], 1 / 3) and p.sum() == pytest.approx(1.0)


def _identity_net():
    """Logit c = standardised input c (c < 8): ReLU(x) - ReLU(-x) through both
    hidden layers, which is x for any sign."""
    W1 = np.zeros((64, 12)); W2 = np.zeros((64, 64)); W3 = np.zeros((8, 64))
    for c in range(8):
        W1[c, c], W1[8 + c, c] = 1.0, -1.0
        W2[c, c], W2[8 + c, 8 + c] = 1.0, 1.0
        W3[c, c], W3[c, 8 + c] = 1.0, -1.0
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(8)])


def test_network_sees_the_standardised_inputs_in_order():
    A = synth.stencil3d7(9)
    f = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    x = oracle.selector_inputs(f)
    rng = np.random.default_rng(11)
    mean = rng.standard_normal(12)
    std = rng.random(12) + 0.5
    std[3] = 0.0                              # a constant input during training: left unscaled
    p = _identity_net()
    z = oracle.mlp_forward(p, ((x - mean) / np.where(std > 0, std, 1.0)).reshape(1, -1))[0]
    want = (x[:8] - mean[:8]) / np.where(std[:8] > 0, std[:8], 1.0)
    assert np.allclose(z, want, rtol=1e-15, atol=1e-15)
    v, prob = oracle.learned_select(f, ALL8, p, mean, std)
    assert v == int(np.argmax(want))
    e = np.exp(want - want.max())
    assert np.allclose(prob, e / e.sum(), rtol=1e-13)
    # moving one class's mean far down makes it the pick
    mean2 = mean.copy()
    mean2[C["coo"]] -= 1e3
    assert oracle.learned_select(f, ALL8, p, mean2, std)[0] == C["coo"]
    rest = [c for c in range(8) if c != C["coo"]]
    assert oracle.learned_select(f, ALL8 & ~(1 << C["coo"]), p, mean2, std)[0] == rest[int(np.argmax(want[rest]))]


def test_no_admissible_class():
    f = oracle.features(10, 10, np.arange(11, dtype=np.int32), np.arange(10, dtype=np.int32))
    v, p = oracle.learned_select(f, 0, _bias_net(np.arange(8.0)), np.zeros(12), np.ones(12))
    assert v == 0 and not p.any()
