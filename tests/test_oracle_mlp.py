"""Pins of the oracle MLP (12 -> 64 -> 64 -> 8, softmax cross-entropy) and Adam
to an independent autograd implementation, finite differences and special cases."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def _torch_forward(p, X):
    o = 0
    def take(shape):
        nonlocal o
        n = int(np.prod(shape))
        t = p[o:o + n].reshape(shape)
        o += n
        return t
    W1, b1, W2, b2, W3, b3 = take((64, 12)), take((64,)), take((64, 64)), take((64,)), take((8, 64)), take((8,))
    h = torch.relu(X @ W1.T + b1)
    h = torch.relu(h @ W2.T + b2)
    return h @ W3.T + b3


def _init(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(oracle.mlp_param_count()) * 0.3


def test_param_count():
    assert oracle.mlp_param_count() == 64 * 12 + 64 + 64 * 64 + 64 + 8 * 64 + 8


def test_forward_against_torch():
    p = _init(0)
    X = np.random.default_rng(1).standard_normal((17, 12))
    ref = _torch_forward(torch.tensor(p), torch.tensor(X)).numpy()
    assert np.max(np.abs(oracle.mlp_forward(p, X) - ref)) < 1e-12


def test_zero_weights_give_output_bias():
    p = np.zeros(oracle.mlp_param_count())
    p[-8:] = np.arange(8)
    out = oracle.mlp_forward(p, np.ones((3, 12)))
    assert np.array_equal(out, np.tile(np.arange(8.0), (3, 1)))
    loss, g = oracle.mlp_loss_grad(np.zeros_like(p), np.ones((2, 12)), np.full((2, 8), 1 / 8))
    assert abs(loss - np.log(8.0)) < 1e-15  # uniform softmax against uniform target
    assert np.max(np.abs(g)) < 1e-15


def test_gradient_against_autograd():
    p = _init(2)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((9, 12))
    T = rng.random((9, 8))
    T /= T.sum(1, keepdims=True)
    loss, g = oracle.mlp_loss_grad(p, X, T)
    pt = torch.tensor(p, requires_grad=True)
    z = _torch_forward(pt, torch.tensor(X))
    L = -(torch.tensor(T) * torch.log_softmax(z, dim=1)).sum() / 9
    L.backward()
    assert abs(loss - L.item()) < 1e-12
    assert np.max(np.abs(g - pt.grad.numpy())) < 1e-12


def test_gradient_against_finite_differences():
    p = _init(4)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((4, 12))
    T = np.eye(8)[[1, 7, 3, 3]]
    _, g = oracle.mlp_loss_grad(p, X, T)
    idx = rng.choice(len(p), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (oracle.mlp_loss_grad(p + e, X, T)[0] - oracle.mlp_loss_grad(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_adam_against_torch():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    pt = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        oracle.adam(p, g, m, v, t, 1e-2, 0.9, 0.999, 1e-8)
        opt.zero_grad()
        pt.grad = torch.tensor(g)
        opt.step()
    assert np.max(np.abs(p - pt.detach().numpy())) < 1e-13
