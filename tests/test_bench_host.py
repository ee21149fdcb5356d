"""Host-side logic of bench.py: the end-to-end issue order and the DRAM
traffic record lookup."""
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
