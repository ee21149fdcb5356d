"""GPU parity of the learned selector's kernels (forward, soft-target
cross-entropy gradient, Adam) against the CPU oracle, and the selector in use."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import learn, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _params(seed, scale=0.3):
    return (np.random.default_rng(seed).standard_normal(smat.SMAT_MLP_PARAMS) * scale).astype(np.float32)


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("B", [1, 31, 32, 100])
def test_forward_matches_oracle(B):
    p = _params(0)
    X = np.random.default_rng(1).standard_normal((B, 12)).astype(np.float32)
    z = torch.empty((B, 8), dtype=torch.float32, device=DEV)
    pd, xd = torch.from_numpy(p).to(DEV), torch.from_numpy(X).to(DEV)
    assert smat.smat_mlp_forward(pd.data_ptr(), xd.data_ptr(), B, z.data_ptr(), _stream()) == 0
    ref = oracle.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    got = z.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("B", [5, 77, 256])
def test_loss_and_gradient_match_oracle(B):
    p = _params(2)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((B, 12)).astype(np.float32)
    T = rng.random((B, 8)).astype(np.float32)
    T[:, 2] = 0.0
    T /= T.sum(1, keepdims=True)
    pd, xd, td = (torch.from_numpy(a).to(DEV) for a in (p, X, T))
    g = torch.empty_like(pd)
    loss = torch.empty(1, device=DEV)
    work = torch.empty(smat.smat_mlp_work_floats(B), device=DEV)
    assert smat.smat_mlp_loss_grad(pd.data_ptr(), xd.data_ptr(), td.data_ptr(), B, g.data_ptr(), loss.data_ptr(),
                                   work.data_ptr(), _stream()) == 0
    ref_loss, ref_g = oracle.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-4 * max(1.0, abs(ref_loss))
    got = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref_g)) <= 1e-3 * np.max(np.abs(ref_g)) + 1e-6
    # deterministic: a second evaluation is bitwise identical
    g2 = torch.empty_like(pd)
    assert smat.smat_mlp_loss_grad(pd.data_ptr(), xd.data_ptr(), td.data_ptr(), B, g2.data_ptr(), loss.data_ptr(),
                                   work.data_ptr(), _stream()) == 0
    assert torch.equal(g, g2)


def test_adam_matches_oracle():
    rng = np.random.default_rng(4)
    n = 5512
    p = rng.standard_normal(n)
    m, v = np.zeros(n), np.zeros(n)
    pd = torch.tensor(p, dtype=torch.float32, device=DEV)
    md, vd = torch.zeros_like(pd), torch.zeros_like(pd)
    for t in range(1, 4):
        g = rng.standard_normal(n)
        gd = torch.tensor(g, dtype=torch.float32, device=DEV)
        assert smat.smat_mlp_adam(pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), n, t, 1e-2, 0.9, 0.999,
                                  1e-8, _stream()) == 0
        oracle.adam(p, g.astype(np.float32).astype(np.float64), m, v, t, 1e-2, 0.9, 0.999, 1e-8)
    assert np.max(np.abs(pd.cpu().numpy() - p)) < 1e-5


def test_training_reduces_loss_on_a_learnable_task():
    # labels are a fixed function of the inputs: the GPU training loop must fit it
    rng = np.random.default_rng(5)
    recs = []
    for i in range(512):
        f = rng.standard_normal(12)
        best = int(np.argmax(f[:8]))
        t = np.full(8, 2.0)
        t[best] = 1.0
        recs.append({"id": i, "kind": "toy", "features": list(f), "admissible": 255, "timings_ms": list(t),
                     "rules": 0})
    params, mean, std, hist = learn.train(recs, epochs=60, batch=64, lr=3e-3, seed=0)
    assert hist[-1] < 0.5 * hist[0]
    P = learn.predict(params, mean, std, recs)
    assert learn.evaluate(P, recs)["mlp"]["accuracy"] > 0.9


def test_learned_mode_selects_an_admissible_variant():
    rng = np.random.default_rng(6)
    params = _params(7, 0.1)
    assert smat.smat_set_model(params, np.zeros(12), np.ones(12)) == 0
    try:
        A = synth.stencil3d7(30)
        M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, "f64")
        M.tune("learned", conf_threshold=0.0, trial_extended=0)   # trust the network: no trials
        plan = M.plan()
        adm = M.features()["admissible"]
        assert (adm >> plan["variant"]) & 1 and 0.0 < plan["confidence"] <= 1.0 and plan["trialled"] == 0
        M.tune("learned", conf_threshold=1.01, fallback_topk=2, trial_extended=0)  # always measure the top 2
        plan = M.plan()
        assert plan["trialled"] == 1 and (adm >> plan["variant"]) & 1
        assert int(np.sum(M.timings() > 0)) == 2
        x = torch.from_numpy(synth.uniform(0, 1, A.n)).to(DEV)
        y = M.spmv(x).cpu().numpy()
        ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x.cpu().numpy())
        assert np.max(np.abs(y - ref)) < 1e-12 * 8
        M.close()
    finally:
        smat.smat_set_model(None, None, None)


def test_model_reloads_while_other_threads_tune():
    # the selector model is process-wide; reloading it while other threads
    # tune their own handles is allowed (tuning predicts from a copy taken
    # under the model's lock)
    import threading
    assert smat.smat_load_model(smat.MODEL_PATH) == smat.SMAT_OK
    mats = [synth.stencil3d7(40), synth.powerlaw(60000, 1.8, 2000, 3)]
    hs = [smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, "f64") for A in mats]
    stop = threading.Event()
    errors = []

    def reload():
        while not stop.is_set():
            if smat.smat_load_model(smat.MODEL_PATH) != smat.SMAT_OK:
                errors.append("load")

    def tune(M, stream):
        try:
            for _ in range(20):
                M.tune("learned", stream=stream, trial_extended=0)
        except Exception as e:  # noqa: BLE001 -- reported below
            errors.append(repr(e))

    t0 = threading.Thread(target=reload)
    streams = [torch.cuda.Stream() for _ in hs]
    ts = [threading.Thread(target=tune, args=(M, st)) for M, st in zip(hs, streams)]
    t0.start()
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    stop.set()
    t0.join()
    assert not errors, errors
    for A, M in zip(mats, hs):   # every plan chosen under the reloads still computes the product
        x = synth.uniform(0, 1, A.n)
        y = M.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x, threads=8)
        scale = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(A.val), np.abs(x), threads=8)
        assert np.all(np.abs(y - ref) <= 1e-12 * scale + 1e-300), M.plan()["name"]
        M.close()
