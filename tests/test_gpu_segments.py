"""Per-segment plans (Sec. 6): a matrix whose upper rows are a banded stencil
and whose lower rows are a power-law graph gets different formats per
segment; the product matches the oracle."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from helpers import TOL, assert_close_rows, reference, stored_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _stacked():
    return synth.stencil_over_powerlaw(24, 2000, 5)   # 13824 banded rows over 13824 irregular ones


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_segments_choose_per_part_and_match_oracle(dtype):
    A = _stacked()
    vals, v64 = stored_values(A, dtype)
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(DEV), torch.from_numpy(A.colidx).to(DEV),
                      torch.from_numpy(np.ascontiguousarray(vals)).to(DEV), dtype)
    # the paper's rules decide from the features alone, so the per-part
    # choice is deterministic: DIA for the banded rows, another format for
    # the power-law rows (timed picks on parts this small are within noise)
    R = smat.Segments(M, 4, "rules")
    assert R.info()["row_starts"] == oracle.segment_starts(A.m, A.rowptr, 4)
    vr = R.info()["variants"]
    assert vr[0] == "dia" and vr[-1] != "dia", vr
    R.close()
    S = smat.Segments(M, 4, "exhaustive", trial_reps=3)
    info = S.info()
    rs = info["row_starts"]
    assert rs == oracle.segment_starts(A.m, A.rowptr, 4)
    assert rs[0] == 0 and rs[-1] == A.m and all(r % 8 == 0 for r in rs[:-1]) and len(rs) >= 3
    npdt = np.float64 if dtype == "f64" else np.float32
    x = synth.uniform(0, 1, A.n).astype(npdt)
    y0 = synth.uniform(1, 1, A.m).astype(npdt)
    y = torch.from_numpy(y0.copy()).to(DEV)
    S.spmv(torch.from_numpy(x).to(DEV), y, 1.5, -0.25)
    torch.cuda.synchronize()
    ref, scale = reference(A, v64, x, 1.5, -0.25, y0)
    assert_close_rows(y.cpu().numpy().astype(np.float64), ref, scale, TOL[dtype], "segments")
    # misaligned y: falls back to the whole-matrix plan, still correct
    yb = torch.zeros(A.m + 1, dtype=y.dtype, device=DEV)
    yb[1:] = torch.from_numpy(y0).to(DEV)
    S.spmv(torch.from_numpy(x).to(DEV), yb[1:], 1.5, -0.25)
    torch.cuda.synchronize()
    assert_close_rows(yb[1:].cpu().numpy().astype(np.float64), ref, scale, TOL[dtype], "segments misaligned")
    S.close()
    M.close()
