"""Host-side logic of the selector's offline stage: split, labels, scoring."""
import numpy as np

from paper_1210_2536_gb300 import learn


def _rec(i, kind, t, adm=255, rules=0):
    return {"id": i, "kind": kind, "features": [0.0] * 12, "admissible": adm, "timings_ms": t, "rules": rules}


def test_split_is_stratified_and_deterministic():
    recs = [_rec(i, ["a", "b", "c"][i % 3], [1.0] * 8) for i in range(300)]
    tr, he = learn.split(recs)
    assert len(he) == 60 and len(tr) == 240
    for k in "abc":
        assert sum(r["kind"] == k for r in he) == 20
    assert [r["id"] for r in learn.split(recs)[1]] == [r["id"] for r in he]


def test_soft_targets_spread_over_ties_and_skip_inadmissible():
    t = np.array([[1.0, 1.01, 1.5, 2.0, np.inf, 1.0, 3.0, 4.0]])
    y = learn.soft_targets(t)
    assert np.allclose(y[0], [1 / 3, 1 / 3, 0, 0, 0, 1 / 3, 0, 0])


def test_evaluate_regret_and_fallback():
    recs = [_rec(0, "a", [2.0, 1.0, 4.0, 4.0, 4.0, 4.0, 4.0, 4.0], rules=0),
            _rec(1, "a", [1.0, 3.0, 4.0, 4.0, 4.0, 4.0, -1.0, 4.0], adm=0b10111111, rules=1)]
    P = np.zeros((2, 8))
    P[0, 2] = 0.55
    P[0, 1] = 0.45   # low confidence: the fallback times the top 3 and finds variant 1
    P[1, 0] = 0.9
    ev = learn.evaluate(P, recs, conf=0.6, topk=3)
    assert ev["mlp"]["regret_mean"] == (4.0 / 1.0 - 1 + 0.0) / 2
    assert ev["mlp_with_fallback"]["regret_mean"] == 0.0 and ev["fallback_rate"] == 0.5
    assert ev["rules"]["regret_mean"] == (1.0 + 2.0) / 2
    assert ev["exhaustive"]["regret_mean"] == 0.0
