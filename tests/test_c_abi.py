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


CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(out, link):
    cmd = ["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(CUDA, "include"), SRC, "-o", out]
    if link:
        from paper_1210_2536_gb300 import _build
        _build.build()
        libdir = os.path.dirname(_build.LIB)
        cudalib = next(d for d in (os.path.join(CUDA, "lib64"), os.path.join(CUDA, "lib"))
                       if os.path.exists(os.path.join(d, "libcudart.so")))
        cmd += [os.path.join(libdir, "libsmat.so"), f"-Wl,-rpath,{libdir}", "-L", cudalib, "-lcudart",
                f"-Wl,-rpath,{cudalib}"]
    else:
        cmd = cmd[:-2] + ["-fsyntax-only"]
    subprocess.check_call(cmd)


def test_header_is_plain_c(tmp_path):
    _compile(str(tmp_path / "x"), link=False)


@pytest.mark.gpu
def test_c_program_matches_oracle(tmp_path):
    exe = str(tmp_path / "c_abi_check")
    _compile(exe, link=True)
    out = str(tmp_path / "part2.bin")
    r = subprocess.run([exe, out], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr, r.stdout)
    lines = r.stdout.split("\n")
    assert lines[0].startswith("nnz 4992 ndiags 5")
    # part 4 (printed right after part 1's y): pipelined host-buffer calls
    # equal the synchronous host-buffer call bit for bit
    assert lines[2] == "part4 mismatches 0"
    del lines[2]
    got = np.array([float(t) for t in lines[1].split()[1:]])
    A = synth.stencil2d5(32)
    x = (np.arange(A.n) % 7) - 3.0
    ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x, 2.0, -1.0, np.ones(A.m))
    assert np.array_equal(got, ref[[0, 1, 32, A.m - 1]])  # small integers: every order is exact
    # part 2: device pointers through smat_create / smat_spmv, every row
    # against the oracle at the FP64 per-row bar
    raw = open(out, "rb").read()
    m, n, k = np.frombuffer(raw[:24], np.int64)
    off = 24
    def take(dt, cnt):
        nonlocal off
        a = np.frombuffer(raw[off:off + cnt * np.dtype(dt).itemsize], dt)
        off += cnt * np.dtype(dt).itemsize
        return a
    rowptr, col, val = take(np.int32, m + 1), take(np.int32, k), take(np.float64, k)
    x, y0, y = take(np.float64, n), take(np.float64, m), take(np.float64, m)
    assert off == len(raw) and int(rowptr[-1]) == k and np.any(np.diff(rowptr) == 0)
    assert np.any(val != np.round(val))
    ref = oracle.spmv_csr(int(m), rowptr, col, val, x, -0.75, 0.5, y0)
    scale = 0.75 * oracle.spmv_csr(int(m), rowptr, col, np.abs(val), np.abs(x)) + 0.5 * np.abs(y0)
    assert np.all(np.abs(y - ref) <= 1e-12 * scale), float(np.max(np.abs(y - ref) / np.maximum(scale, 1e-300)))
    assert lines[2].startswith("part2 nnz ")
    # part 3: the refused CSR
    assert lines[3] == f"part3 status {2} handle null"
