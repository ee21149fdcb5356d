"""The boundary from plain C: tests/c_abi_check.c includes include/smat.h,
links libsmat.so and runs a whole create / tune / multiply cycle."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1210_2536_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_check.c")


def _compile(out, link):
    cmd = ["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC, "-o", out]
    if link:
        from paper_1210_2536_gb300 import _build
        _build.build()
        libdir = os.path.dirname(_build.LIB)
        cmd += [os.path.join(libdir, "libsmat.so"), f"-Wl,-rpath,{libdir}"]
    else:
        cmd = cmd[:-2] + ["-fsyntax-only"]
    subprocess.check_call(cmd)


def test_header_is_plain_c(tmp_path):
    _compile(str(tmp_path / "x"), link=False)


@pytest.mark.gpu
def test_c_program_matches_oracle(tmp_path):
    exe = str(tmp_path / "c_abi_check")
    _compile(exe, link=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    assert lines[0].startswith("nnz 4992 ndiags 5")
    got = np.array([float(t) for t in lines[1].split()[1:]])
    A = synth.stencil2d5(32)
    x = (np.arange(A.n) % 7) - 3.0
    ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x, 2.0, -1.0, np.ones(A.m))
    assert np.array_equal(got, ref[[0, 1, 32, A.m - 1]])  # small integers: every order is exact
