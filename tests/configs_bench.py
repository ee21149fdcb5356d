"""Measurements of the parity/feature configurations beside the main bench:

  poisson64          2-D 5-point 64x64 FP64: features, exhaustive trial, every
                     variant's latency (the matrix lives in L2: a latency
                     case, not a roofline one)
  batched_hierarchy  27-point hierarchy 192^3..12^3 + 64 mixed matrices, FP64:
                     one batched graph launch vs per-matrix launches (plain
                     and graph-captured)
  galerkin           Galerkin AMG hierarchy (smoothed aggregation, P^T A P) of
                     the 27-point operator on 128^3, FP64 and FP32: each
                     level's own plan, one batched launch vs per-matrix
                     launches, every level checked against the oracle
  segments           per-segment plans (Sec. 6) on the 7-point 128^3 stencil
                     stacked over a 2e6-row power-law graph, FP64 and FP32:
                     the whole-matrix plan against 2, 4 and 8 nonzero-balanced
                     segments, each with its own format
  precision          power-law n = 8e6 with FP64 / FP32 / BF16 values (error
                     vs FP64), and mixed-precision CG on the 3-D 7-point 256^3
                     Laplacian

  python tests/configs_bench.py poisson64|batched_hierarchy|galerkin|segments|precision|all \
      [--out results.jsonl]

Each prints one JSON line.  The harness sits with the tests because it
checks every measured product against the oracle (the error columns); the
oracle is the CPU checker, never part of the measured path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time

import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def _time(fn, reps=20, warmup=3):
    """Milliseconds per call of fn, back to back: the mean of the middle half
    of `reps` repetitions, each timing enough calls (up to 32) to span about
    40 us, since the event-timed duration of a single short kernel on this
    GPU moves in steps of about 2 us;
    the repetitions are queued behind a device sleep that outlasts their host
    enqueue (re-queued behind a longer one if it did not), so that no host
    launch latency falls between a pair of events."""
    import torch
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(2100 * (100 + 50 * max(warmup, 1)))
    w0.record()
    for _ in range(max(warmup, 1)):
        fn()
    w1.record()
    torch.cuda.synchronize()
    group = max(1, min(32, math.ceil(0.040 / max(w0.elapsed_time(w1) / max(warmup, 1), 1e-4))))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    hold_us = 500 + 50 * reps * group
    for _ in range(3):
        t0 = time.perf_counter()
        torch.cuda._sleep(int(2100 * min(hold_us, 200000)))     # cycles at about 2.1 GHz
        for s, e in ev:
            s.record()
            for _ in range(group):
                fn()
            e.record()
        host_us = (time.perf_counter() - t0) * 1e6
        torch.cuda.synchronize()
        if host_us < hold_us:
            break
        hold_us = 1.5 * host_us + 500
    t = sorted(s.elapsed_time(e) / group for s, e in ev)
    q = len(t) // 4
    return statistics.mean(t[q:len(t) - q])


def _select():
    import paper_1210_2536_gb300 as smat
    if os.path.exists(smat.MODEL_PATH) and smat.smat_load_model(smat.MODEL_PATH) == 0:
        return "learned"
    return "exhaustive"


def poisson64():
    import torch

    import oracle
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    A = synth.poisson_2d_64()
    dev = torch.device("cuda:0")
    M = smat.SpMatrix(A.m, A.n, A.rowptr, A.colidx, A.val, "f64")
    t0 = time.perf_counter()
    M.tune("exhaustive", keep_formats=1)
    tune_wall = (time.perf_counter() - t0) * 1e3
    f = M.features()
    x = torch.from_numpy(synth.uniform(0, 1, A.n)).to(dev)
    ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x.cpu().numpy())
    scale = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(A.val), np.abs(x.cpu().numpy()))
    lat = {}
    err = {}
    for v in list(range(8)) + [smat.SMAT_V_HYB, smat.SMAT_V_SELL, smat.SMAT_V_BCSR, smat.SMAT_V_SPLIT]:
        if v < 8 and not (f["admissible"] >> v) & 1:
            continue
        y = torch.empty(A.m, dtype=torch.float64, device=dev)
        try:
            M.spmv(x, y, variant=v)   # builds a further format if it is admissible
        except smat.SmatError:
            continue
        lat[smat.VARIANT_NAMES[v]] = round(_time(lambda: M.spmv(x, y, variant=v), 50) * 1e3, 2)
        err[smat.VARIANT_NAMES[v]] = float(np.max(np.abs(y.cpu().numpy() - ref) / scale))
    fo = oracle.features(A.m, A.n, A.rowptr, A.colidx)
    same = all(f[k] == fo[k] for k in ("nnz", "max_rd", "min_rd", "ndiags", "ntdiags", "aver_rd", "var_rd",
                                         "er_dia", "er_ell", "ntdiags_ratio", "r"))
    out = {"config": "poisson2d_64 f64", "features_bit_exact": same, "pick": M.plan()["name"],
           "tune_ms": round(M.plan()["tune_ms"], 3), "tune_wall_ms": round(tune_wall, 3),
           "latency_us": lat, "max_err_normalized": err, "hbm": "n/a (0.3 MB, L2-resident)"}
    M.close()
    return out


def batched_hierarchy():
    import torch

    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    from paper_1210_2536_gb300.roofline import algorithmic_bytes
    dev = torch.device("cuda:0")
    select = _select()
    mats = synth.amg_like_hierarchy(192) + synth.mixed_batch(64)
    hs, xs, ys = [], [], []
    for A in mats:
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                          torch.from_numpy(A.val).to(dev), "f64")
        M.tune(select)
        hs.append(M)
        xs.append(torch.from_numpy(synth.uniform(0, 1, A.n)).to(dev))
        ys.append(torch.zeros(A.m, dtype=torch.float64, device=dev))
    nnz = sum(A.nnz for A in mats)
    byts = sum(algorithmic_bytes(M.features(), M.plan()["variant"], "f64") for M in hs)
    B = smat.Batch(hs)
    t0 = time.perf_counter()
    B.tune()
    tune_s = time.perf_counter() - t0
    info = B.info()

    def per_matrix():
        for M, x, y in zip(hs, xs, ys):
            M.spmv(x, y)

    t_loop = _time(per_matrix, 20)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        per_matrix()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            per_matrix()
    t_graph = _time(lambda: g.replay(), 20)
    t_batch = _time(lambda: B.spmv(xs, ys), 20)
    small = [i for i, A in enumerate(mats) if i >= 5]
    t_small_loop = _time(lambda: [hs[i].spmv(xs[i], ys[i]) for i in small], 20)
    Bs = smat.Batch([hs[i] for i in small]).tune()
    t_small_batch = _time(lambda: Bs.spmv([xs[i] for i in small], [ys[i] for i in small]), 20)
    peak = _peak()
    out = {"config": "27-pt hierarchy 192^3..12^3 + 64 mixed, f64", "matrices": len(mats), "nnz": nnz,
           "selector": select, "alg_bytes": byts,
           "per_matrix_launches_ms": round(t_loop, 4), "per_matrix_graph_ms": round(t_graph, 4),
           "batched_graph_ms": round(t_batch, 4),
           "batched_gflops": round(2 * nnz / t_batch / 1e6, 1), "batched_hbm_frac": round(byts / t_batch / 1e6 / peak, 4),
           "per_matrix_gflops": round(2 * nnz / t_loop / 1e6, 1),
           "small_64_only": {"per_matrix_launches_ms": round(t_small_loop, 4), "batched_ms": round(t_small_batch, 4),
                             "info": Bs.info()},
           "batch_info": info, "batch_tune_s": round(tune_s, 2),
           "picks": {smat.VARIANT_NAMES[v]: sum(1 for M in hs if M.plan()["variant"] == v)
                     for v in range(smat.SMAT_NUM_ALL_VARIANTS)}}
    Bs.close()
    B.close()
    for M in hs:
        M.close()
    return out


def galerkin(m_fine=128):
    import torch

    import oracle
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    from paper_1210_2536_gb300.roofline import algorithmic_bytes
    dev = torch.device("cuda:0")
    select = _select()
    t0 = time.perf_counter()
    mats = synth.galerkin_hierarchy(m_fine, 5)
    gen_s = time.perf_counter() - t0
    threads = os.cpu_count() or 1
    peak = _peak()
    out = {"config": f"Galerkin AMG hierarchy (smoothed aggregation) of the 27-point operator on {m_fine}^3",
           "selector": select, "generate_s": round(gen_s, 1),
           "levels": [{"name": A.name, "m": A.m, "nnz": A.nnz, "max_rd": int(np.diff(A.rowptr).max())} for A in mats]}
    for dt in ("f64", "f32"):
        npdt = np.float64 if dt == "f64" else np.float32
        hs, xs, ys, per_level = [], [], [], []
        for i, A in enumerate(mats):
            vals = A.val if dt == "f64" else A.val.astype(np.float32)
            M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                              torch.from_numpy(vals).to(dev), dt)
            M.tune(select)
            x = synth.uniform(60 + i, 1, A.n).astype(npdt)
            xd = torch.from_numpy(x).to(dev)
            y = M.spmv(xd)
            ms = _time(lambda: M.spmv(xd, y), 20)
            v64 = np.asarray(vals, dtype=np.float64)
            ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, v64, x.astype(np.float64), threads=threads)
            sc = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(v64), np.abs(x.astype(np.float64)), threads=threads)
            err = float(np.max(np.abs(y.double().cpu().numpy() - ref) / np.maximum(sc, 1e-300)))
            b = algorithmic_bytes(M.features(), M.plan()["variant"], dt)
            per_level.append({"level": i, "pick": M.plan()["name"], "ms": round(ms, 4),
                              "gflops": round(2 * A.nnz / ms / 1e6, 1), "hbm_frac": round(b / ms / 1e6 / peak, 4),
                              "max_err_normalized": err})
            hs.append(M)
            xs.append(xd)
            ys.append(torch.zeros(A.m, dtype=xd.dtype, device=dev))
        nnz = sum(A.nnz for A in mats)
        B = smat.Batch(hs).tune()

        def per_matrix():
            for M, x, y in zip(hs, xs, ys):
                M.spmv(x, y)

        t_loop = _time(per_matrix, 20)
        t_batch = _time(lambda: B.spmv(xs, ys), 20)
        info = B.info()
        B.close()
        # the selector on structures it was not trained on: regret of each
        # level's pick against the exhaustive search's fastest variant
        for lv, M, x, y in zip(per_level, hs, xs, ys):
            if select == "learned":
                M.tune("exhaustive", trial_reps=10)
                best = _time(lambda: M.spmv(x, y), 20)
                lv["exhaustive_pick"] = M.plan()["name"]
                lv["exhaustive_ms"] = round(best, 4)
                lv["regret"] = round(lv["ms"] / best - 1.0, 4)
        out[dt] = {"per_level": per_level, "per_matrix_launches_ms": round(t_loop, 4),
                   "batched_ms": round(t_batch, 4), "batched_gflops": round(2 * nnz / t_batch / 1e6, 1),
                   "per_matrix_gflops": round(2 * nnz / t_loop / 1e6, 1), "batch_info": info}
        for M in hs:
            M.close()
    return out


def segments(m=128):
    import torch

    import oracle
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    dev = torch.device("cuda:0")
    select = _select()
    A = synth.stencil_over_powerlaw(m)
    threads = os.cpu_count() or 1
    out = {"config": f"per-segment plans: {A.name}", "m": A.m, "nnz": A.nnz, "selector": select}
    for dt in ("f64", "f32"):
        npdt = np.float64 if dt == "f64" else np.float32
        vals = A.val if dt == "f64" else A.val.astype(np.float32)
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                          torch.from_numpy(vals).to(dev), dt)
        M.tune(select)
        x = synth.uniform(0, 1, A.n).astype(npdt)
        xd = torch.from_numpy(x).to(dev)
        y = torch.zeros(A.m, dtype=xd.dtype, device=dev)
        v64 = np.asarray(vals, dtype=np.float64)
        ref = oracle.spmv_csr(A.m, A.rowptr, A.colidx, v64, x.astype(np.float64), threads=threads)
        sc = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(v64), np.abs(x.astype(np.float64)), threads=threads)

        def err_of(yy):
            return float(np.max(np.abs(yy.double().cpu().numpy() - ref) / np.maximum(sc, 1e-300)))

        M.spmv(xd, y)
        whole = {"pick": M.plan()["name"], "ms": round(_time(lambda: M.spmv(xd, y), 20), 4), "max_err": err_of(y)}
        segs = {}
        for k in (2, 4, 8):
            t0 = time.perf_counter()
            S = smat.Segments(M, k, select)
            build_s = time.perf_counter() - t0
            S.spmv(xd, y)
            segs[str(k)] = {"picks": S.info()["variants"], "ms": round(_time(lambda: S.spmv(xd, y), 20), 4),
                            "max_err": err_of(y), "build_s": round(build_s, 2)}
            S.close()
        out[dt] = {"whole": whole, "segments": segs,
                   "gflops_whole": round(2 * A.nnz / whole["ms"] / 1e6, 1),
                   "gflops_best_segments": round(2 * A.nnz / min(v["ms"] for v in segs.values()) / 1e6, 1)}
        M.close()
    return out


def precision(cg_total=500, cg_cap=5000):
    import torch

    import oracle
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    from paper_1210_2536_gb300.roofline import algorithmic_bytes
    dev = torch.device("cuda:0")
    select = _select()
    A = synth.powerlaw(8_000_000, 1.8, 10000, 0)
    x64 = synth.uniform(0, 1, A.n)
    threads = os.cpu_count() or 1
    ref64 = oracle.spmv_csr(A.m, A.rowptr, A.colidx, A.val, x64, threads=threads)
    scale64 = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(A.val), np.abs(x64), threads=threads)
    peak = _peak()
    prec = {}
    for dt in ("f64", "f32", "bf16"):
        if dt == "f64":
            vals, v64, xx = A.val, A.val, x64
        elif dt == "f32":
            vals = A.val.astype(np.float32)
            v64, xx = vals.astype(np.float64), x64.astype(np.float32)
        else:
            vals = oracle.round_bf16(A.val)
            v64, xx = oracle.bf16_to_double(vals), x64.astype(np.float32)
            vals = vals.view(np.int16)
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                          torch.from_numpy(np.ascontiguousarray(vals)).to(dev), dt)
        M.tune(select)
        xd = torch.from_numpy(np.ascontiguousarray(xx)).to(dev)
        y = M.spmv(xd)
        ms = _time(lambda: M.spmv(xd, y), 20)
        csr_ms = _time(lambda: M.spmv(xd, y, variant=0), 5, 1)
        got = M.spmv(xd).double().cpu().numpy()
        xs64 = np.asarray(xx, dtype=np.float64)
        ref_s = oracle.spmv_csr(A.m, A.rowptr, A.colidx, v64, xs64, threads=threads)
        sc_s = oracle.spmv_csr(A.m, A.rowptr, A.colidx, np.abs(v64), np.abs(xs64), threads=threads)
        e_stored = np.abs(got - ref_s) / np.maximum(sc_s, 1e-300)
        e_fp64 = np.abs(got - ref64) / np.maximum(scale64, 1e-300)
        b = algorithmic_bytes(M.features(), M.plan()["variant"], dt)
        prec[dt] = {"pick": M.plan()["name"], "ms": round(ms, 4), "gflops": round(2 * A.nnz / ms / 1e6, 1),
                    "hbm_frac": round(b / ms / 1e6 / peak, 4), "csr_scalar_ms": round(csr_ms, 4),
                    "err_vs_stored_max": float(e_stored.max()), "err_vs_stored_median": float(np.median(e_stored)),
                    "err_vs_fp64_max": float(e_fp64.max()), "err_vs_fp64_median": float(np.median(e_fp64))}
        M.close()
    # mixed-precision CG on the 7-point 256^3 Laplacian
    L = synth.stencil3d7(256)
    xt = synth.uniform(0, 5, L.n)
    b = oracle.spmv_csr(L.m, L.rowptr, L.colidx, L.val, xt, threads=threads)
    H64 = smat.SpMatrix(L.m, L.n, torch.from_numpy(L.rowptr).to(dev), torch.from_numpy(L.colidx).to(dev),
                        torch.from_numpy(L.val).to(dev), "f64").tune(select)
    H32 = smat.SpMatrix(L.m, L.n, torch.from_numpy(L.rowptr).to(dev), torch.from_numpy(L.colidx).to(dev),
                        torch.from_numpy(L.val.astype(np.float32)).to(dev), "f32").tune(select)
    bd = torch.from_numpy(b).to(dev)
    cg = {}
    for name, kw in (("500_inner_iterations", dict(max_total_inner=cg_total, rtol=1e-10, max_inner=cg_total)),
                     ("to_1e-10", dict(max_total_inner=cg_cap, rtol=1e-10, max_inner=2000))):
        xd = torch.zeros(L.n, dtype=torch.float64, device=dev)
        info = smat.cg_mixed(H64, H32, bd, xd, **kw)
        xs = xd.cpu().numpy()
        r = b - oracle.spmv_csr(L.m, L.rowptr, L.colidx, L.val, xs, threads=threads)
        info["relres_oracle"] = float(np.linalg.norm(r) / np.linalg.norm(b))
        cg[name] = info
    out = {"config": "precision: powerlaw 8e6 f64/f32/bf16; mixed CG stencil3d7 256^3", "nnz": A.nnz,
           "selector": select, "precision": prec, "cg": cg,
           "cg_plans": {"f64": H64.plan()["name"], "f32": H32.plan()["name"]}}
    H64.close()
    H32.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["poisson64", "batched_hierarchy", "galerkin", "segments", "precision", "all"])
    ap.add_argument("--out")
    a = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    todo = ["poisson64", "batched_hierarchy", "galerkin", "segments", "precision"] if a.which == "all" else [a.which]
    for w in todo:
        res = {"poisson64": poisson64, "batched_hierarchy": batched_hierarchy, "galerkin": galerkin,
               "segments": segments, "precision": precision}[w]()
        line = json.dumps(res)
        print(line, flush=True)
        if a.out:
            with open(a.out, "a") as f:
                f.write(line + "\n")


if __name__ == "__main__":
    main()
