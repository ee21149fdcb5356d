"""Plan cache, host side: the key's reference pinned to SplitMix64's
published outputs, and the cache file through the C library (no GPU)."""
import os

import numpy as np
import pytest

import paper_1210_2536_gb300 as smat
from plan_key_ref import GOLDEN, mix

KAT = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_kat.txt")


def test_mixer_matches_splitmix64_known_answers():
    rows = [l.split() for l in open(KAT) if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for seed, i, want in rows:
        with np.errstate(over="ignore"):
            z = np.uint64(int(seed)) + np.uint64(int(i) - 1) * GOLDEN
        assert int(mix(z)) == int(want)


def _lines(path):
    return sorted(l.strip() for l in open(path).read().splitlines()[1:] if l.strip())


def test_cache_file_round_trip(tmp_path):
    smat.plan_cache_clear()
    src = tmp_path / "a.txt"
    entries = ["00000000000000ff 0 10 10 28 6 256", "0123456789abcdef 1 5 7 12 10 64",
               "fedcba9876543210 2 1000 1000 5000 12 256"]
    src.write_text("smat-plan-cache 1\n" + "\n".join(entries) + "\n")
    smat.plan_cache_load(src)
    assert smat.plan_cache_size() == 3
    out = tmp_path / "b.txt"
    smat.plan_cache_save(out)
    assert open(out).readline() == "smat-plan-cache 1\n"
    assert _lines(out) == sorted(entries)
    # a loaded entry replaces the one with its key; others are kept
    upd = tmp_path / "c.txt"
    upd.write_text("smat-plan-cache 1\n00000000000000ff 0 10 10 28 0 256\n")
    smat.plan_cache_load(upd)
    assert smat.plan_cache_size() == 3
    smat.plan_cache_save(out)
    assert "00000000000000ff 0 10 10 28 0 256" in _lines(out)
    smat.plan_cache_clear()
    assert smat.plan_cache_size() == 0


@pytest.mark.parametrize("text", [
    "smat-plan-cache 2\n",                                          # unknown version
    "plan-cache 1\n",                                               # wrong header
    "smat-plan-cache 1\n00ff 0 10 10 28 6\n",                       # short line
    "smat-plan-cache 1\n00ff 3 10 10 28 6 256\n",                   # no such dtype
    "smat-plan-cache 1\n00ff 0 10 10 28 13 256\n",                  # no such variant
    "smat-plan-cache 1\n00ff 0 -1 10 28 6 256\n",                   # negative size
])
def test_malformed_cache_file_changes_nothing(tmp_path, text):
    smat.plan_cache_clear()
    good = tmp_path / "good.txt"
    good.write_text("smat-plan-cache 1\n0000000000000001 0 4 4 4 0 256\n")
    smat.plan_cache_load(good)
    bad = tmp_path / "bad.txt"
    bad.write_text(text + "0000000000000002 0 4 4 4 0 256\n")
    with pytest.raises(smat.SmatError):
        smat.plan_cache_load(bad)
    assert smat.plan_cache_size() == 1
    with pytest.raises(smat.SmatError):
        smat.plan_cache_load(tmp_path / "missing.txt")
    smat.plan_cache_clear()
