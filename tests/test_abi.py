"""The C ABI library builds, loads without a GPU, and exports every function
declared in include/*.h; host-only argument checks need no device."""
import ctypes
import glob
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1210_2536_gb300 import _build
    _build.build()
    import paper_1210_2536_gb300 as smat
    return smat.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(smat_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi(lib):
    import paper_1210_2536_gb300 as smat
    for n in declared_functions():
        if n in ("smat_test_fail_alloc_after",):
            continue
        assert n in smat._SIGS, n


def test_struct_layouts(lib):
    import paper_1210_2536_gb300 as smat
    assert ctypes.sizeof(smat.smat_features_t) == 8 * 9 + 8 * 6 + 8
    o = smat.smat_tune_opts_default()
    assert (o.mode, o.tau_num, o.tau_den, o.fill_ratio_max, o.trial_reps) == (smat.SMAT_TUNE_LEARNED, 3, 5, 20, 10)
    assert abs(o.conf_threshold - 0.6) < 1e-7 and o.bytes_cap == 4.0


def test_host_side_argument_checks(lib):
    import paper_1210_2536_gb300 as smat
    assert smat.smat_status_string(smat.SMAT_ERR_INVALID_CSR) == "invalid CSR structure"
    st, h = smat.smat_create(-1, 4, 0, None, None, None, smat.SMAT_F64)
    assert st == smat.SMAT_ERR_INVALID_ARG and not h
    st, h = smat.smat_create(4, 4, 0, None, None, None, smat.SMAT_F64)   # rowptr missing
    assert st == smat.SMAT_ERR_INVALID_ARG
    st, h = smat.smat_create(2**31, 4, 0, 1, None, None, smat.SMAT_F64)   # beyond int32 indexing
    assert st == smat.SMAT_ERR_UNSUPPORTED
    assert smat.smat_destroy(None) == smat.SMAT_OK
    assert smat.smat_spmv(None, None, None, None, None, 0) == smat.SMAT_ERR_INVALID_ARG
    assert smat.smat_load_model("/nonexistent/model.bin") == smat.SMAT_ERR_MODEL


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_1210_2536_gb300 as s; s.LIB_PATH = '/nonexistent/libsmat.so'\n"
            "try:\n    s.lib()\nexcept RuntimeError as e:\n    print('raised', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "raised" in r.stdout and "no fallback" in r.stdout


def test_model_file_roundtrip(lib, tmp_path):
    import numpy as np
    import paper_1210_2536_gb300 as smat
    p = str(tmp_path / "m.bin")
    smat.write_model(p, np.zeros(smat.SMAT_MLP_PARAMS, np.float32), np.zeros(12), np.ones(12))
    assert smat.smat_load_model(p) == smat.SMAT_OK
    with open(p, "r+b") as f:
        f.write(b"XXXX")
    assert smat.smat_load_model(p) == smat.SMAT_ERR_MODEL
    assert smat.smat_set_model(None, None, None) == smat.SMAT_OK


def test_model_path_from_the_environment(lib, tmp_path, monkeypatch):
    # smat_load_model(NULL) loads the file SMAT_MODEL_PATH names
    import numpy as np
    import paper_1210_2536_gb300 as smat
    p = str(tmp_path / "env.bin")
    smat.write_model(p, np.zeros(smat.SMAT_MLP_PARAMS, np.float32), np.zeros(12), np.ones(12))
    monkeypatch.delenv("SMAT_MODEL_PATH", raising=False)
    assert smat.smat_load_model(None) == smat.SMAT_ERR_INVALID_ARG
    monkeypatch.setenv("SMAT_MODEL_PATH", p)
    assert smat.smat_load_model(None) == smat.SMAT_OK
    monkeypatch.setenv("SMAT_MODEL_PATH", str(tmp_path / "missing.bin"))
    assert smat.smat_load_model(None) == smat.SMAT_ERR_MODEL
    assert smat.smat_set_model(None, None, None) == smat.SMAT_OK
