"""Host-side logic of bench.py: the end-to-end issue order, the DRAM
traffic record lookup and the live selector-regret bookkeeping."""
import itertools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_e2e_issue_order_on_the_structures_suite_shape():
    # 8 products in no particular order, with their times alone
    times = [0.5, 0.3, 0.9, 0.1, 1.7, 0.2, 0.7, 1.3]
    order = bench.e2e_issue_order(times)
    by_time = sorted(range(8), key=lambda j: times[j])
    longest, second = by_time[-1], by_time[-2]
    assert order[1] == second and order[4] == longest       # second-longest second, longest halfway
    rest = [j for j in order if j not in (longest, second)]
    assert rest == by_time[:-2]                             # the others shortest first
    assert order[0] == by_time[0]


@pytest.mark.parametrize("n", range(0, 11))
def test_e2e_issue_order_is_a_permutation(n):
    times = [((7 * j) % 11) * 0.1 + j * 1e-3 for j in range(n)]
    order = bench.e2e_issue_order(times)
    assert sorted(order) == list(range(n))
    if n < 4:
        assert order == sorted(range(n), key=lambda j: times[j])


def test_traffic_record_needs_the_current_kernel_source(tmp_path, monkeypatch):
    # a recorded traffic figure counts only while spmv.cu hashes to the value
    # recorded beside it
    import hashlib
    src = open(os.path.join(ROOT, "paper_1210_2536_gb300", "csrc", "spmv.cu"), "rb").read()
    h = hashlib.sha256(src).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.md").write_text(
        "| kernel | alg | traffic | sha |\n|---|---|---|---|\n"
        f"| split:f64:m | 10 | 123 | {h} |\n| coo:f64:m | 10 | 456 | 0000000000000000 |\n")
    (tmp_path / "paper_1210_2536_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_1210_2536_gb300" / "csrc" / "spmv.cu").write_bytes(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic_record("split:f64:m") == 123.0
    assert bench.dram_traffic_record("coo:f64:m") is None     # recorded for another source
    assert bench.dram_traffic_record("sell:f64:m") is None    # not recorded


def test_break_even_reproduces_the_papers_count():
    # Sec. 7.3: tuning costs 19 CSR products and the tuned product takes a
    # third of CSR's time; it pays after n > 19 / (1 - 1/3) = 28.5 products,
    # the paper's 29
    n = bench.break_even_calls(19.0, 1.0, 1.0 / 3.0)
    assert abs(n - 28.5) < 1e-12 and int(n) + 1 == 29
    assert bench.break_even_calls(5.0, 1.0, 1.0) is None      # no gain, never pays
    assert bench.break_even_calls(5.0, 1.0, 2.0) is None
    assert bench.break_even_calls(0.0, 2.0, 1.0) == 0.0


def test_configuration_harness_loads_and_lists_its_workloads():
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "configs_bench.py"), "--help"],
                         capture_output=True, text=True, check=True).stdout
    for name in ("poisson64", "batched_hierarchy", "galerkin", "segments", "precision", "all"):
        assert name in out


def test_selector_regret_over_the_whole_plan_space():
    # the live regret loop with a fake timer: every admissible class and every
    # further format that builds is timed, the pick always (even outside the
    # classes' mask), each mode separately; regret = t(pick) / t(best) - 1
    import numpy as np
    import paper_1210_2536_gb300 as smat

    class _A:
        def __init__(self, name):
            self.name = name

    class _M:
        def timings(self):
            t = np.full(smat.SMAT_NUM_ALL_VARIANTS, -1.0, np.float32)
            t[smat.SMAT_V_CSR_VEC32] = 0.009
            return t

    V = smat
    warm_times = {  # product 0: CSR-vector-32 picked, COO faster; product 1: SPLIT picked and fastest
        0: {V.SMAT_V_CSR_SCALAR: 0.030, V.SMAT_V_CSR_VEC32: 0.010, V.SMAT_V_COO: 0.008, V.SMAT_V_SELL: 0.020},
        1: {V.SMAT_V_CSR_SCALAR: 0.200, V.SMAT_V_COO: 0.060, V.SMAT_V_SPLIT: 0.050},
    }
    cold_times = {0: dict(warm_times[0]), 1: dict(warm_times[1])}
    cold_times[0][V.SMAT_V_COO] = 0.012      # cold: the pick is the fastest after all
    cold_times[1][V.SMAT_V_COO] = 0.040      # cold: COO beats the pick by 25 %
    prods = [
        {"A": _A("m0"), "M": _M(), "f": {"admissible": (1 << V.SMAT_V_CSR_SCALAR) | (1 << V.SMAT_V_CSR_VEC32)
                                         | (1 << V.SMAT_V_COO)},
         "plan": {"variant": V.SMAT_V_CSR_VEC32, "name": "csr_vec32", "trialled": 1, "confidence": 0.61}},
        {"A": _A("m1"), "M": _M(), "f": {"admissible": (1 << V.SMAT_V_CSR_SCALAR) | (1 << V.SMAT_V_COO)},
         "plan": {"variant": V.SMAT_V_SPLIT, "name": "split", "trialled": 1, "confidence": 1.0}},
    ]
    calls = []

    def fake_time(p, v, cold=True):
        i = prods.index(p)
        calls.append((i, v, cold))
        table = (cold_times if cold else warm_times)[i]
        if v not in table:
            raise smat.SmatError(smat.SMAT_ERR_UNSUPPORTED, "build")
        return table[v]

    out = bench.selector_regret(prods, fake_time)
    w, c = out["warm"], out["cold_l2"]
    assert [r["regret"] for r in w["rows"]] == [0.25, 0.0]
    assert [r["best"] for r in w["rows"]] == ["coo", "split"]
    assert [r["hit"] for r in w["rows"]] == [False, True]
    assert [r["regret"] for r in c["rows"]] == [0.0, 0.25]
    assert w["mean_regret"] == 0.125 and w["max_regret"] == 0.25 and w["accuracy_within_2pct"] == 0.5
    assert w["rows"][0]["us"] == {"csr_scalar": 30.0, "csr_vec32": 10.0, "coo": 8.0, "sell": 20.0}
    assert w["rows"][0]["tuner_us"] == {"csr_vec32": 9.0}
    # the classes outside a matrix's mask are not timed, every further format is
    # tried, and the pick is timed even when it is a further format
    timed = {(i, v) for i, v, cold_ in calls if not cold_}
    assert (1, V.SMAT_V_CSR_VEC32) not in timed and (1, V.SMAT_V_SPLIT) in timed
    assert all((i, f) in timed for i in (0, 1) for f in (V.SMAT_V_HYB, V.SMAT_V_SELL, V.SMAT_V_BCSR, V.SMAT_V_SPLIT))


def test_reference_arm_prints_its_line_on_the_host():
    # the reference arm is the oracle on the host cores: it needs no GPU, and
    # its one JSON line carries the keys the bench contract asks of it
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--scale", "0.05"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1
    assert line["metric"] and line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
