"""smat_spmv_many: independent products run side by side on the library's
own streams, ordered after the work already queued on the caller's stream and
before the work queued after the call.  Every product is compared with the
oracle within the per-row bars; the x each one reads is written on the
caller's stream just before the call, and y is read on it just after."""
import numpy as np
import pytest

import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _mats():
    return [(synth.stencil3d7(40), "f64"), (synth.stencil3d7(40), "f32"), (synth.uniform_random(80000, 16.0, 1), "f64"),
            (synth.uniform_random(80000, 16.0, 1), "bf16"), (synth.powerlaw(100000, 1.8, 5000, 2), "f64"),
            (synth.powerlaw(100000, 1.8, 5000, 2), "f32"), (synth.blockdiag(64000, 8, 3), "f64"),
            (synth.blockdiag(64000, 8, 3), "f32"), (synth.stencil2d5(64), "bf16"), (synth.stencil3d27(20), "f64")]


@pytest.fixture(scope="module")
def handles():
    out = []
    for A, dt in _mats():
        vals, v64 = stored_values(A, dt)
        if dt == "bf16":
            vals = vals.view(np.int16)
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                          torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dt)
        M.tune("exhaustive", trial_reps=3)
        out.append((A, dt, M, v64))
    yield out
    for _, _, M, _ in out:
        M.close()


def _vectors(items, seed):
    xs, ys, y0s, xh = [], [], [], []
    for k, (A, dt, _, _) in enumerate(items):
        t = np.float64 if dt == "f64" else np.float32
        x = synth.uniform(seed + k, 1, A.n).astype(t)
        y0 = synth.uniform(seed + k, 2, A.m).astype(t)
        xh.append(x)
        y0s.append(y0)
        xs.append(torch.zeros(A.n, dtype=torch.from_numpy(x).dtype, device=DEV))
        ys.append(torch.from_numpy(y0.copy()).to(DEV))
    return xs, ys, y0s, xh


def _check(items, xh, y0s, got, alphas, betas, what):
    for k, (A, dt, M, v64) in enumerate(items):
        ref, scale = reference(A, v64, xh[k], alphas[k], betas[k], y0s[k] if betas[k] != 0 else None)
        assert_close_rows(got[k], ref, scale, TOL[dt], f"{what} {k} {A.name} {dt} {M.plan()['name']}")


def test_many_products_match_the_oracle_and_keep_stream_order(handles):
    items = handles
    xs, ys, y0s, xh = _vectors(items, 100)
    alphas = [1.0, -0.5, 2.0, 1.0, 0.75, 1.0, -1.0, 3.0, 1.0, 0.5]
    betas = [0.0, 2.0, 0.0, -1.0, 0.5, 0.0, 1.0, 0.0, 0.25, 0.0]
    stream = torch.cuda.Stream()
    src = [torch.from_numpy(x).pin_memory() for x in xh]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for x, h in zip(xs, src):
            x.copy_(h, non_blocking=True)          # written on the caller's stream just before
        smat.spmv_many([M for _, _, M, _ in items], xs, ys, alphas, betas, stream=stream)
        out = [y.clone() for y in ys]              # read on it just after
    stream.synchronize()
    _check(items, xh, y0s, [o.cpu().numpy().astype(np.float64) for o in out], alphas, betas, "many")


def test_more_products_than_streams(handles):
    # 20 products on 16 streams: a handle appears twice, each time with its own y
    items = handles + handles
    xs, ys, y0s, xh = _vectors(items, 200)
    for x, v in zip(xs, xh):
        x.copy_(torch.from_numpy(v))
    alphas, betas = [1.0] * len(items), [0.0] * len(items)
    smat.spmv_many([M for _, _, M, _ in items], xs, ys, alphas, betas)
    torch.cuda.synchronize()
    _check(items, xh, y0s, [y.cpu().numpy().astype(np.float64) for y in ys], alphas, betas, "twenty")


def test_many_inside_a_captured_graph(handles):
    items = handles
    xs, ys, y0s, xh = _vectors(items, 300)
    mats = [M for _, _, M, _ in items]
    alphas, betas = [1.0] * len(items), [0.0] * len(items)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        smat.spmv_many(mats, xs, ys, alphas, betas, stream=s)   # first call outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        smat.spmv_many(mats, xs, ys, alphas, betas, stream=s)
    for x, v in zip(xs, xh):
        x.copy_(torch.from_numpy(v))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    _check(items, xh, y0s, [y.cpu().numpy().astype(np.float64) for y in ys], alphas, betas, "graph")


def test_many_argument_errors(handles):
    M = handles[0][2]
    assert smat.lib().smat_spmv_many(None, -1, None, None, None, None, None) == smat.SMAT_ERR_INVALID_ARG
    assert smat.lib().smat_spmv_many(None, 2, None, None, None, None, None) == smat.SMAT_ERR_INVALID_ARG
    assert smat.lib().smat_spmv_many(None, 0, None, None, None, None, None) == smat.SMAT_OK
    assert smat.spmv_many([], [], []) == []
    x = torch.zeros(M.n, dtype=torch.float64, device=DEV)
    y = torch.zeros(M.m, dtype=torch.float64, device=DEV)
    smat.spmv_many([M], [x], [y])                  # one product: runs on the caller's stream
    torch.cuda.synchronize()
    assert torch.all(y == 0)
