"""The roofline arithmetic the bench reports: algorithmic bytes per format,
L2 sector requests on random-column matrices, and the binding roof."""
import pytest

from paper_1210_2536_gb300 import roofline as R

F = {"m": 1000, "n": 800, "nnz": 5000, "max_rd": 9, "ndiags": 7, "empty_rows": 3,
     "hyb_K": 4, "hyb_ncoo": 1200, "sell_slots": 6400, "sell_ns": 32, "bcsr_b": 2, "bcsr_nb": 1800,
     "split_ns": 3000, "split_nc": 5}


@pytest.mark.parametrize("dt,sv,sx", [("f64", 8, 8), ("f32", 4, 4), ("bf16", 2, 4)])
def test_algorithmic_bytes_closed_forms(dt, sv, sx):
    xy = sx * F["n"] + sx * F["m"]
    assert R.algorithmic_bytes(F, 0, dt) == (sv + 4) * 5000 + 4 * 1001 + xy
    assert R.algorithmic_bytes(F, 0, dt, beta_nonzero=True) == (sv + 4) * 5000 + 4 * 1001 + xy + sx * F["m"]
    assert R.algorithmic_bytes(F, R.V_COO, dt) == (sv + 8) * 5000 + xy
    assert R.algorithmic_bytes(F, R.V_ELL, dt) == (sv + 4) * 9 * 1000 + xy
    assert R.algorithmic_bytes(F, R.V_DIA, dt) == sv * 7 * 1000 + 4 * 7 + xy
    assert R.algorithmic_bytes(F, R.V_HYB, dt) == (sv + 4) * 4 * 1000 + (sv + 8) * 1200 + xy
    assert R.algorithmic_bytes(F, R.V_BCSR, dt) == (sv * 4 + 4) * 1800 + 4 * 501 + xy
    assert R.algorithmic_bytes(F, R.V_SPLIT, dt) == (sv + 4) * 2000 + 20 * 5 + (sv + 8) * 3000 + 4 * 3 + xy
    # SELL: slots, a 4-byte row index per position (32 per slice), a width and
    # a slice pointer per slice, and the closing pointer
    assert R.algorithmic_bytes(F, R.V_SELL, dt) == (sv + 4) * 6400 + 4 * 32 * 32 + 12 * 32 + 8 + xy
    # every CSR kernel moves the same arrays
    for v in (1, 2, 3, 4, 8):
        assert R.algorithmic_bytes(F, v, dt) == R.algorithmic_bytes(F, 0, dt)
    with pytest.raises(ValueError):
        R.algorithmic_bytes(F, 13, dt)


def test_l2_sectors_on_random_columns():
    # COO in FP64: one sector per gather, 16 streamed bytes per entry, and a
    # whole sector per row written (rows are written one at a time)
    assert R.l2_sectors(F, R.V_COO, "f64") == 5000 + (16 * 5000) / 32 + 1000
    # FP32 COO also loads each thread's next row: one sector per 8 entries
    assert R.l2_sectors(F, R.V_COO, "f32") == 5000 + (12 * 5000) / 32 + 1000 + 5000 / 8
    # FP32 CSR: 8 bytes per entry, the row pointers, a coalesced 4-byte y
    assert R.l2_sectors(F, 0, "f32") == 5000 + (8 * 5000 + 4 * 1001 + 4 * 1000) / 32
    # SELL gathers once per slot, padding included, and writes y through its permutation
    assert R.l2_sectors(F, R.V_SELL, "f64") == 6400 + (R.algorithmic_bytes(F, R.V_SELL, "f64") - 8 * 800 - 8 * 1000) / 32 + 1000
    # SPLIT FP32: its short rows' tiles load next rows too
    split = (R.algorithmic_bytes(F, R.V_SPLIT, "f32") - 4 * 800 - 4 * 1000) / 32
    assert R.l2_sectors(F, R.V_SPLIT, "f32") == 5000 + split + 1000 + 3000 / 8


def test_bound_picks_the_slower_roof():
    # DIA in FP64 with 7 diagonals: 7000 FMAs; at 1 us the FP64 pipe needs
    # 2*7000 / 1.2586e12 s = 11.1 ns and HBM 56,028 + 14,400 bytes at 1000 GB/s
    # = 70.4 ns, so HBM binds
    b = R.bound(F, R.V_DIA, "f64", 1e-6, 1000.0)
    assert b["bound"] == "hbm" and b["frac"] == pytest.approx(b["hbm_frac"])
    assert b["fp64_frac"] == pytest.approx(2 * 7000 / (R.FP64_PEAK_TFLOPS * 1e12) / 1e-6)
    # at 100,000 GB/s the FP64 pipe binds
    b = R.bound(F, R.V_DIA, "f64", 1e-6, 100000.0)
    assert b["bound"] == "alu" and b["unit"] == "TFLOP/s" and b["frac"] == pytest.approx(b["fp64_frac"])
    assert R.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.07 / 1e3)
    # FP32 has no FP64 roof
    assert "fp64_frac" not in R.bound(F, R.V_COO, "f32", 1e-6, 1000.0)
