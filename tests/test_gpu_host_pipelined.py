"""smat_spmv_host_pipelined: host-buffer products on the handle's own
streams with two staging sets used in turn (the unified CSR interface of
Sec. 3 with x and y in host memory).  Consecutive calls with different
inputs, each checked against the oracle once the caller's stream has
finished; beta != 0 (y read from the host too); two handles of different
storage types interleaved on one stream; refusal while the stream captures
a graph; argument errors."""
import numpy as np
import pytest

import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _handle(A, dt, mode="exhaustive"):
    vals, v64 = stored_values(A, dt)
    if dt == "bf16":
        vals = vals.view(np.int16)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dt)
    M.tune(mode, trial_reps=3)
    return M, v64


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("mk", [lambda: synth.powerlaw(60000, 1.8, 3000, 3), lambda: synth.stencil3d7(30),
                                lambda: synth.uniform_random(40001, 9.0, 4)], ids=["powerlaw", "stencil", "uniform"])
def test_consecutive_calls_match_the_oracle(dt, mk):
    A = mk()
    M, v64 = _handle(A, dt)
    t = np.float64 if dt == "f64" else np.float32
    s = torch.cuda.Stream()
    calls = []
    for k in range(5):   # sets 0, 1, 0, 1, 0: each reused while the other is busy
        x = synth.uniform(50 + k, 1, A.n).astype(t)
        y0 = synth.uniform(50 + k, 2, A.m).astype(t)
        alpha, beta = [(1.0, 0.0), (-0.5, 2.0), (2.0, 0.0), (1.0, -1.0), (0.75, 0.5)][k]
        xh, yh = _pinned(x), _pinned(y0.copy())
        M.spmv_host_pipelined(xh, yh, alpha, beta, stream=s)
        calls.append((x, y0, alpha, beta, yh))
    s.synchronize()
    for k, (x, y0, alpha, beta, yh) in enumerate(calls):
        ref, scale = reference(A, v64, x, alpha, beta, y0 if beta != 0 else None)
        assert_close_rows(yh.numpy().astype(np.float64), ref, scale, TOL[dt], f"{A.name} {dt} call {k}")
    M.close()


def test_two_handles_interleaved_on_one_stream():
    A, B = synth.powerlaw(50000, 1.8, 2000, 5), synth.stencil3d7(24)
    MA, vA = _handle(A, "f64")
    MB, vB = _handle(B, "f32")
    s = torch.cuda.Stream()
    out = []
    for k in range(4):
        xa = synth.uniform(70 + k, 1, A.n)
        xb = synth.uniform(80 + k, 1, B.n).astype(np.float32)
        ya, yb = _pinned(np.zeros(A.m)), _pinned(np.zeros(B.m, np.float32))
        MA.spmv_host_pipelined(_pinned(xa), ya, stream=s)
        MB.spmv_host_pipelined(_pinned(xb), yb, stream=s)
        out.append((xa, ya, xb, yb))
    s.synchronize()
    for k, (xa, ya, xb, yb) in enumerate(out):
        ref, scale = reference(A, vA, xa, 1.0, 0.0, None)
        assert_close_rows(ya.numpy(), ref, scale, TOL["f64"], f"A call {k}")
        ref, scale = reference(B, vB, xb, 1.0, 0.0, None)
        assert_close_rows(yb.numpy().astype(np.float64), ref, scale, TOL["f32"], f"B call {k}")
    MA.close()
    MB.close()


def test_matches_the_synchronous_host_call_bit_for_bit():
    A = synth.powerlaw(30000, 1.8, 2000, 8)
    M, _ = _handle(A, "f64")
    x = _pinned(synth.uniform(9, 1, A.n))
    y1, y2 = _pinned(np.zeros(A.m)), _pinned(np.zeros(A.m))
    M.spmv_host(x, y1)
    s = torch.cuda.Stream()
    M.spmv_host_pipelined(x, y2, stream=s)
    s.synchronize()
    assert np.array_equal(y1.numpy().view(np.int64), y2.numpy().view(np.int64))
    M.close()


def test_refused_while_capturing_and_argument_errors():
    A = synth.stencil2d5(32)
    M, _ = _handle(A, "f64")
    x, y = _pinned(synth.uniform(1, 1, A.n)), _pinned(np.zeros(A.m))
    s = torch.cuda.Stream()
    M.spmv_host_pipelined(x, y, stream=s)      # streams and staging exist before the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    refused = []
    with torch.cuda.graph(g, stream=s):
        try:
            M.spmv_host_pipelined(x, y, stream=s)
        except smat.SmatError as e:            # refused before any work is enqueued
            refused.append(e.status)
    assert refused == [smat.SMAT_ERR_UNSUPPORTED]
    a = np.array([1.0])
    assert smat.smat_spmv_host_pipelined(M.h, a.ctypes.data, None, a.ctypes.data, y.data_ptr(), 0) == smat.SMAT_ERR_INVALID_ARG
    assert smat.smat_spmv_host_pipelined(None, a.ctypes.data, x.data_ptr(), a.ctypes.data, y.data_ptr(), 0) != smat.SMAT_OK
    # the handle still works afterwards
    M.spmv_host_pipelined(x, y, stream=s)
    s.synchronize()
    ref = M.spmv(torch.from_numpy(x.numpy()).to(DEV)).cpu().numpy()
    assert np.allclose(y.numpy(), ref, rtol=1e-12, atol=0)
    M.close()


@pytest.mark.parametrize("shape", [(3, 0), (0, 5), (50, 40)], ids=["no_columns", "no_rows", "all_rows_empty"])
def test_degenerate_matrices_pipelined_and_side_by_side(shape):
    # nnz = 0: y = beta*y through the pipelined host call and through
    # smat_spmv_many beside a regular product
    m, n = shape
    A = synth.CSR(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32), np.zeros(0), name=f"empty_{m}x{n}")
    M, _ = _handle(A, "f64")
    x = _pinned(np.ones(n))
    ys_h = [_pinned(np.full(m, 3.0 + k)) for k in range(3)]
    s = torch.cuda.Stream()
    for y in ys_h:                        # both staging sets, then the first again
        M.spmv_host_pipelined(x, y, 1.0, 0.5, stream=s)
    s.synchronize()
    for k, y in enumerate(ys_h):
        assert np.array_equal(y.numpy(), np.full(m, 0.5 * (3.0 + k)))
    B = synth.stencil2d5(16)
    MB, vB = _handle(B, "f64")
    xb = synth.uniform(4, 1, B.n)
    xs = [torch.ones(n, dtype=torch.float64, device=DEV), torch.from_numpy(xb).to(DEV)]
    ys = [torch.full((m,), 2.0, dtype=torch.float64, device=DEV), torch.zeros(B.m, dtype=torch.float64, device=DEV)]
    smat.spmv_many([M, MB], xs, ys, [1.0, 1.0], [-1.0, 0.0])
    torch.cuda.synchronize()
    assert torch.equal(ys[0].cpu(), torch.full((m,), -2.0, dtype=torch.float64))
    ref, scale = reference(B, vB, xb, 1.0, 0.0, None)
    assert_close_rows(ys[1].cpu().numpy(), ref, scale, TOL["f64"], "regular beside an empty one")
    M.close()
    MB.close()
