"""The committed learned selector, evaluated on its held-out matrices: what
the trained network gains over the method without it (the paper's rules,
always CSR-scalar) measured as regret against the exhaustive search.
The CPU test runs the network through the oracle's FP64 forward pass; the GPU
test through libsmat's kernel, which must pick the same variants."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import learn, synth


def _heldout():
    recs = learn.load(smat.DATASET_PATH)
    train, held = learn.split(recs)
    return train, held


def test_dataset_and_split():
    train, held = _heldout()
    assert len(train) + len(held) == synth.DATASET_SIZE == 2400 and len(held) == 398 + 80
    assert {r["kind"] for r in held} == {r["kind"] for r in train} == set(synth.KIND_NAMES)
    # every record is the matrix its id names (the generators' contract)
    for r in train + held:
        kind, params, _ = synth.dataset_spec(r["id"])
        assert r["kind"] == synth.KIND_NAMES[kind]
        assert np.allclose(r["params"], [float(v) for v in params], rtol=1e-12)


def _oracle_forward(params, Xs):
    return oracle.mlp_forward(params.astype(np.float64), Xs.astype(np.float64))


def test_learned_selector_beats_rules_and_fixed_choices():
    params, mean, std = smat.read_model(smat.MODEL_PATH)
    _, held = _heldout()
    P = learn.predict(params, mean, std, held, forward=_oracle_forward)
    ev = learn.evaluate(P, held)
    assert ev["mlp"]["regret_mean"] <= 0.10           # at most 10 % mean slowdown vs exhaustive
    assert ev["mlp_with_fallback"]["regret_mean"] <= ev["mlp"]["regret_mean"] + 1e-12
    assert ev["mlp"]["regret_mean"] < 0.5 * ev["rules"]["regret_mean"]
    assert ev["mlp"]["accuracy"] > ev["rules"]["accuracy"] + 0.2
    assert ev["mlp"]["speedup_vs_csr_scalar_geomean"] > ev["rules"]["speedup_vs_csr_scalar_geomean"]


@pytest.mark.gpu
def test_gpu_forward_picks_like_the_oracle():
    params, mean, std = smat.read_model(smat.MODEL_PATH)
    _, held = _heldout()
    Pg = learn.predict(params, mean, std, held)                       # libsmat kernel
    Po = learn.predict(params, mean, std, held, forward=_oracle_forward)
    assert np.max(np.abs(Pg - Po)) < 1e-3
    agree = np.mean(Pg.argmax(1) == Po.argmax(1))
    assert agree >= 0.99
    assert learn.evaluate(Pg, held)["mlp"]["regret_mean"] <= 0.10
