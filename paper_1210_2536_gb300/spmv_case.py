"""Run one synthetic matrix through chosen SpMV variants and report time,
GFLOP/s and the fraction of HBM bandwidth each reaches (algorithmic bytes,
see roofline.py).  Used for kernel studies and profiler captures:

  python -m paper_1210_2536_gb300.spmv_case --matrix stencil3d7:128 --dtype f64 --variant all
  python -m paper_1210_2536_gb300.spmv_case --matrix powerlaw:2000000 --variant coo --reps 3
  python -m paper_1210_2536_gb300.spmv_case --matrix stencil3d7:128 --variant dia --cold
  python -m paper_1210_2536_gb300.spmv_case --matrix stencil3d7:128 --variant dia --kernel all

Matrices: stencil2d5:<m>, stencil3d7:<m>, stencil3d27:<m>, uniform:<n>[:lambda],
powerlaw:<n>[:alpha], blockdiag:<n>[:b].
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time

import numpy as np


def make_matrix(spec: str):
    from . import synth
    kind, *args = spec.split(":")
    a = [float(v) for v in args]
    if kind == "stencil2d5":
        return synth.stencil2d5(int(a[0]))
    if kind == "stencil3d7":
        return synth.stencil3d7(int(a[0]))
    if kind == "stencil3d27":
        return synth.stencil3d27(int(a[0]))
    if kind == "uniform":
        return synth.uniform_random(int(a[0]), a[1] if len(a) > 1 else 16.0, 0)
    if kind == "powerlaw":
        return synth.powerlaw(int(a[0]), a[1] if len(a) > 1 else 1.8, 10000, 0)
    if kind == "blockdiag":
        return synth.blockdiag(int(a[0]), int(a[1]) if len(a) > 1 else 8, 0)
    raise ValueError(spec)


def main():
    import torch

    import paper_1210_2536_gb300 as smat
    from .roofline import algorithmic_bytes
    ap = argparse.ArgumentParser()
    ap.add_argument("--matrix", default="stencil3d7:128")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--variant", default="all")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--kernel", default="measured",
                    help="kernels behind DIA / ELL: 'measured' (the handle's choice), or 'all' to time each "
                         "(DIA: direct / staged; ELL: consecutive / lane-striped)")
    ap.add_argument("--cold", action="store_true",
                    help="read a buffer of twice the L2 size between timed repetitions (x and the matrix "
                         "start from HBM; L2 holds clean lines of other data)")
    a = ap.parse_args()
    A = make_matrix(a.matrix)
    from . import synth
    dev = torch.device("cuda:0")
    if a.dtype == "f64":
        vals = A.val
    elif a.dtype == "f32":
        vals = A.val.astype(np.float32)
    else:
        vals = torch.from_numpy(A.val).to(torch.bfloat16).view(torch.int16).numpy()
    M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                      torch.from_numpy(np.ascontiguousarray(vals)).to(dev), a.dtype)
    f = M.features()
    tdt = torch.float64 if a.dtype == "f64" else torch.float32
    x = torch.from_numpy(synth.uniform(0, 1, A.n)).to(dev).to(tdt)
    y = torch.zeros(A.m, dtype=tdt, device=dev)
    peak = 6800.0
    try:
        peak = float(json.load(open(os.path.join(os.path.dirname(os.path.dirname(__file__)),
                                                 "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    names = smat.VARIANT_NAMES
    vs = [v for v in range(8) if (f["admissible"] >> v) & 1] + [9, 10, 11, 12] if a.variant == "all" \
        else [names.index(a.variant)]
    out = {"matrix": A.name, "m": A.m, "nnz": A.nnz, "dtype": a.dtype, "cache": "cold" if a.cold else "warm-x",
           "variants": {}}
    flush = None
    if a.cold:
        l2 = torch.cuda.get_device_properties(dev).L2_cache_size
        flush = torch.ones(2 * l2 // 4, dtype=torch.int32, device=dev)
    kernel_names = {smat.SMAT_V_DIA: ("direct", "staged1", "staged2"),
                    smat.SMAT_V_ELL: ("rows", "lanes")}
    for v in vs:
        try:
            M.spmv(x, y, variant=v)   # builds the format; further formats may not be admissible
        except smat.SmatError:
            continue
        f = M.features()
        kernels = [None]
        if v in kernel_names:
            measured = M.kernel(v)
            kernels = list(range(len(kernel_names[v]))) if a.kernel == "all" else [measured]
        for k in kernels:
            label = names[v]
            if k is not None:
                try:
                    M.set_kernel(v, k)
                except smat.SmatError:
                    continue
                label = f"{names[v]}:{kernel_names[v][k]}" + ("*" if k == measured else "")
            # a device sleep lets the host queue the launches ahead of the GPU,
            # so that no host launch latency falls between two events
            w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda._sleep(2100 * (100 + 30 * max(a.warmup, 1)))
            w0.record()
            for _ in range(max(a.warmup, 1)):
                M.spmv(x, y, variant=v)
            w1.record()
            torch.cuda.synchronize()
            # warm: enough products per repetition (up to 32) to span about
            # 40 us, since the event-timed duration of a single short kernel
            # moves in steps of about 2 us
            group = 1 if a.cold else max(1, min(32, math.ceil(0.040 / max(w0.elapsed_time(w1) / max(a.warmup, 1),
                                                                           1e-4))))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(a.reps)]
            hold_us = 500 + a.reps * (30 * group + (70 if a.cold else 0))
            for _ in range(3):
                t0 = time.perf_counter()
                torch.cuda._sleep(int(2100 * hold_us))    # cycles at about 2.1 GHz
                for s, e in ev:
                    if flush is not None:
                        flush.sum()
                    s.record()
                    for _ in range(group):
                        M.spmv(x, y, variant=v)
                    e.record()
                host_us = (time.perf_counter() - t0) * 1e6
                torch.cuda.synchronize()
                if host_us < hold_us:     # the queue stayed ahead of the GPU
                    break
                hold_us = 1.5 * host_us + 500
            t = sorted(s.elapsed_time(e) / group for s, e in ev)
            q = len(t) // 4
            ms = statistics.mean(t[q:len(t) - q])   # mean of the middle half
            b = algorithmic_bytes(f, v, a.dtype)
            out["variants"][label] = {"ms": round(ms, 5), "gflops": round(2 * A.nnz / ms / 1e6, 1),
                                      "gbs": round(b / ms / 1e6, 1), "hbm_frac": round(b / ms / 1e6 / peak, 4)}
    print(json.dumps(out))
    M.close()


if __name__ == "__main__":
    main()
