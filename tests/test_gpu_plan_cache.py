"""Plan cache on the GPU: the structural key against its documented
definition, and smat_tune reusing, recording, saving and reloading plans."""
import numpy as np
import pytest

import oracle
import paper_1210_2536_gb300 as smat
from paper_1210_2536_gb300 import synth
from paper_1210_2536_gb300.synth import CSR
from helpers import TOL, assert_close_rows, reference, stored_values
from plan_key_ref import plan_key

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _model():
    assert smat.smat_load_model(smat.MODEL_PATH) == smat.SMAT_OK


def _handle(A, dtype="f64", vals=None):
    v = stored_values(A, dtype)[0] if vals is None else vals
    return smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, np.ascontiguousarray(v), dtype)


@pytest.mark.parametrize("mk", [lambda: synth.stencil3d7(9), lambda: synth.powerlaw(5000, 1.8, 500, 3),
                                lambda: CSR(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty"),
                                lambda: synth.uniform_random(3000, 6.0, 1)])
def test_key_matches_its_definition(mk):
    A = mk()
    for dt, code in (("f64", smat.SMAT_F64), ("f32", smat.SMAT_F32), ("bf16", smat.SMAT_BF16)):
        M = _handle(A, dt)
        assert M.plan_key() == plan_key(A.m, A.n, A.rowptr, A.colidx, code)
        M.close()


def test_key_depends_on_structure_only():
    A = synth.powerlaw(4000, 1.8, 400, 5)
    k = [_handle(A).plan_key(), _handle(A, vals=A.val * -3.0 + 1.0).plan_key()]
    assert k[0] == k[1]                                   # values do not enter
    # move the last column of one row one place right (the row stays sorted)
    col = A.colidx.copy()
    ends = A.rowptr[1:][np.diff(A.rowptr) > 0] - 1
    e = int(ends[np.argmax(col[ends] + 1 < A.n)])
    col[e] += 1
    B = CSR(A.m, A.n, A.rowptr, col, A.val)
    assert _handle(B).plan_key() != k[0]
    assert _handle(A, "f32").plan_key() != k[0]          # the storage dtype enters


def test_tune_reuses_records_saves_and_reloads(tmp_path):
    smat.plan_cache_clear()
    A = synth.powerlaw(20000, 1.8, 3000, 2)
    M1 = _handle(A)
    M1.tune("learned", plan_cache=1)
    p1 = M1.plan()
    assert p1["from_cache"] == 0 and smat.plan_cache_size() == 1
    # a second handle of the same structure (other values) takes the recorded plan
    vals2 = synth.normal(9, 3, A.nnz)
    M2 = _handle(A, vals=vals2)
    M2.tune("learned", plan_cache=1)
    p2 = M2.plan()
    assert p2["from_cache"] == 1 and p2["variant"] == p1["variant"] and p2["trialled"] == 0
    x = torch.from_numpy(synth.uniform(0, 1, A.n)).cuda()
    y = M2.spmv(x)
    ref, scale = reference(A, vals2, x.cpu().numpy(), 1.0, 0.0, None)
    assert_close_rows(y.cpu().numpy(), ref, scale, TOL["f64"], "cached plan")
    # the cache survives a file round trip
    path = tmp_path / "plans.txt"
    smat.plan_cache_save(path)
    smat.plan_cache_clear()
    M3 = _handle(A)
    M3.tune("rules", plan_cache=0)
    assert M3.plan()["from_cache"] == 0 and smat.plan_cache_size() == 0   # not recorded without plan_cache
    smat.plan_cache_load(path)
    M3.tune("rules", plan_cache=1)
    assert M3.plan()["from_cache"] == 1 and M3.plan()["variant"] == p1["variant"]
    # a recorded plan outside `allowed` is not used: the handle is tuned again
    allowed = ((1 << smat.SMAT_NUM_ALL_VARIANTS) - 1) & ~(1 << p1["variant"]) & ~(1 << smat.SMAT_V_CSR_SCALAR_EXACT)
    M3.tune("exhaustive", plan_cache=1, allowed=allowed, trial_reps=2)
    assert M3.plan()["from_cache"] == 0 and M3.plan()["variant"] != p1["variant"]
    # FIXED mode neither reads nor writes the cache
    M4 = _handle(A)
    M4.tune("fixed", variant=smat.SMAT_V_CSR_SCALAR, plan_cache=1)
    assert M4.plan()["from_cache"] == 0 and M4.plan()["variant"] == smat.SMAT_V_CSR_SCALAR
    for M in (M1, M2, M3, M4):
        M.close()
    smat.plan_cache_clear()


def test_cached_sell_plan_keeps_its_window():
    smat.plan_cache_clear()
    A = synth.uniform_random(6000, 9.0, 4)
    M1 = _handle(A)
    M1.tune("exhaustive", plan_cache=1, allowed=1 << smat.SMAT_V_SELL, sell_sigma=64, trial_reps=2)
    assert M1.plan()["variant"] == smat.SMAT_V_SELL
    M2 = _handle(A)
    M2.tune("learned", plan_cache=1)          # default window 256; the recorded plan used 64
    assert M2.plan()["from_cache"] == 1 and M2.plan()["variant"] == smat.SMAT_V_SELL
    parts = M2.export_parts(smat.SMAT_FMT_SELL)
    perm, width, _ = oracle.sell_layout(A.m, A.rowptr, 64)
    assert np.array_equal(parts["perm"], perm) and np.array_equal(parts["width"], width)
    x = torch.from_numpy(synth.uniform(1, 1, A.n)).cuda()
    ref, scale = reference(A, A.val, x.cpu().numpy(), 1.0, 0.0, None)
    assert_close_rows(M2.spmv(x).cpu().numpy(), ref, scale, TOL["f64"], "cached SELL plan")
    M1.close(), M2.close()
    smat.plan_cache_clear()


def test_alloc_hook_armed_from_the_environment():
    # SMAT_TEST_FAIL_ALLOC_AFTER=k makes the k-th allocation fail from the
    # moment the library loads (a child process, so this one stays clean)
    import os
    import subprocess
    import sys
    code = ("import numpy as np, paper_1210_2536_gb300 as smat\n"
            "from paper_1210_2536_gb300 import synth\n"
            "A = synth.stencil3d7(6)\n"
            "try:\n"
            "    smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, 'f64'); print('ok')\n"
            "except smat.SmatError as e:\n"
            "    print('status', e.status)\n")
    env = dict(os.environ, SMAT_TEST_FAIL_ALLOC_AFTER="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == f"status {smat.SMAT_ERR_ALLOC}"
