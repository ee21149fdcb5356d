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


def _raw(ndiags=5, ntdiags=5, max_rd=5, er_dia=1.0, er_ell=1.0, var_rd=0.0, r=0.0, r_valid=0):
    return {"ndiags": ndiags, "ntdiags": ntdiags, "max_rd": max_rd, "min_rd": 0, "er_dia": er_dia,
            "er_ell": er_ell, "var_rd": var_rd, "r": r, "r_valid": r_valid}


def test_influence_bins_and_good_counts_by_hand():
    # DIA (variant 6) good when within 2 % of the fastest admissible class;
    # a matrix that does not admit DIA is not counted for DIA's parameters
    t_dia_best = [2.0, 2.0, 2.0, 2.0, 2.0, 1.5, 1.0, 3.0]
    t_dia_tie = [1.0, 2.0, 2.0, 2.0, 2.0, 1.5, 1.01, 3.0]
    t_dia_slow = [1.0, 2.0, 2.0, 2.0, 2.0, 1.5, 1.03, 3.0]
    recs = [
        dict(_rec(0, "a", t_dia_best), raw=_raw(ndiags=5, ntdiags=5, er_dia=0.95), nnz=10),
        dict(_rec(1, "a", t_dia_tie), raw=_raw(ndiags=30, ntdiags=12, er_dia=0.5), nnz=2_000_000),
        dict(_rec(2, "a", t_dia_slow), raw=_raw(ndiags=24, ntdiags=6, er_dia=0.7), nnz=2_000_000),
        dict(_rec(3, "a", [1.0] * 6 + [-1.0, 1.0], adm=0b10111111), raw=_raw(ndiags=3000), nnz=10),
        dict(_rec(4, "a", [1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 0.5]), raw=_raw(r=2.0, r_valid=1), nnz=10),
    ]
    rep = learn.influence(recs)
    by = {p["parameter"]: p for p in rep["parameters"]}
    nd = by["ndiags"]["bins"]                                 # [1,25) [25,100) [100,500) [500,inf)
    assert [(b["n"], b["good"]) for b in nd] == [(3, 1), (1, 1), (0, 0), (0, 0)]   # ids 0, 2, 4; id 1
    assert [(b["n_large"], b["good_large"]) for b in nd] == [(1, 0), (1, 1), (0, 0), (0, 0)]
    ed = by["er_dia"]["bins"]                                 # [0,.2) [.2,.4) [.4,.6) [.6,.8) [.8,inf)
    assert [b["n"] for b in ed] == [0, 0, 1, 1, 2] and [b["good"] for b in ed] == [0, 0, 1, 0, 1]
    nt = by["ntdiags_ratio"]["bins"]                          # 1.0, 0.4, 0.25, then ratio 5/5 for ids 3 and 4
    assert [b["n"] for b in nt] == [0, 1, 1, 0, 2]
    rr = by["r"]                                              # COO (7) admitted by all five
    assert sum(b["n"] for b in rr["bins"]) + rr["undefined"]["n"] == 5
    assert rr["bins"][1] == dict(rr["bins"][1], n=1, good=1)  # R = 2 in [1, 4), COO fastest
    assert rr["undefined"]["n"] == 4


def test_influence_report_is_reproducible_from_the_labelled_set():
    import json
    import os
    pkg = os.path.dirname(learn.__file__)
    recs = learn.load(os.path.join(pkg, "selector_dataset.jsonl"))
    rep = learn.influence(recs)
    assert rep == json.load(open(os.path.join(pkg, "influence_report.json")))
    for p in rep["parameters"]:
        v = learn.VARIANT_SHORT.index(p["format"])
        admitting = sum(1 for r in recs if (r["admissible"] >> v) & 1 and r["timings_ms"][v] > 0)
        counted = sum(b["n"] for b in p["bins"]) + (p["undefined"]["n"] if "undefined" in p else 0)
        assert counted == admitting, p["parameter"]
