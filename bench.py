#!/usr/bin/env python
"""SpMV benchmark: GFLOP/s and HBM % of peak of the tuned pick vs plain CSR.

Workload (the paper's structure classes at full size, synthetic, seeded):
3-D 7-point Laplacian 128^3; uniform random n = 1e6 with Poisson(16) rows;
power-law n = 2e6 with Zipf(1.8) rows capped at 1e4; 8x8 block diagonal
n = 1e6.  Each matrix is stored in FP64 and in FP32 (FP32 accumulation), so a
step is eight products y = A x through each handle's tuned plan.  Tuning
(feature extraction, selection, conversion) happens once per handle before the
timed region and is reported as overhead in units of one CSR-scalar product.

python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]
Under torchrun every rank runs its own replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line.

--workload picks the configuration (default: structures, the suite above):
  precision  power-law n = 8e6 (Zipf 1.8, cap 1e4) with values stored in FP64,
             FP32 and BF16 (FP32 accumulation): three products per step
  batched    the 27-point hierarchy 192^3 .. 12^3 plus 64 mixed matrices
             (n 1e3 .. 1e6), FP64: one batched launch per step
  cg         mixed-precision CG on the 3-D 7-point 256^3 Laplacian: FP32 inner
             products, FP64 residual and update; one step = 500 inner
             iterations from x = 0
  selector   the learned selector on held-out matrices of its labelled set
             (FP64): one product per matrix per step, each through its
             learned plan, with the regret against an exhaustive timing of
             the eight classes measured in the same run
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GFLOP/s, HBM % of peak: tuned/learned pick vs plain CSR at stated error"
UNIT = "GFLOP/s"
WORKLOADS = {
    "structures": "structures_suite: stencil3d7 128^3, uniform 1e6 Poisson(16), powerlaw 2e6 Zipf(1.8) cap 1e4, "
                  "blockdiag 1e6 b=8; FP64 and FP32 storage",
    "precision": "precision: powerlaw 8e6 Zipf(1.8) cap 1e4, values FP64 / FP32 / BF16 (FP32 accumulate)",
    "batched": "batched: 27-point stencils 192^3, 96^3, 48^3, 24^3, 12^3 + 64 mixed matrices n 1e3..1e6, FP64, "
               "one batched launch",
    "cg": "cg: mixed-precision CG, 3-D 7-point 256^3 (n 16.8e6), FP32 inner / FP64 outer, 500 inner iterations "
          "per step",
    "selector": "selector: learned picks on held-out matrices of the labelled set (FP64)",
}
WORKLOAD = WORKLOADS["structures"]
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5}
# every row of these products, tuned as here, against the oracle
PARITY_TESTS = {
    "structures": "tests/test_gpu_api.py::test_full_size_bench_workload_parity",
    "precision": "tests/test_gpu_full_size.py::test_powerlaw_8m_full_size",
    "batched": "tests/test_gpu_full_size.py::test_batched_hierarchy_full_size",
    "cg": "tests/test_gpu_full_size.py::test_mixed_cg_256_full_size",
    "selector": "tests/test_gpu_selection.py",
}
PARITY_TEST = PARITY_TESTS["structures"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=float, default=1.0, help="row-count scale of the workload (1 = full size)")
    p.add_argument("--select", default="auto", choices=["auto", "learned", "exhaustive", "rules"])
    p.add_argument("--dtypes", default="f64,f32")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--concurrent", type=int, default=1,
                   help="1: steps without per-product events run the products on a stream each")
    p.add_argument("--workload", default="structures", choices=sorted(WORKLOADS))
    p.add_argument("--selector-sample", type=int, default=48,
                   help="held-out matrices in the selector workload")
    return p.parse_args()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(scale):
    from paper_1210_2536_gb300 import synth
    mats = synth.structures_suite(scale)
    xs = [synth.uniform(0, 1, A.n) for A in mats]
    return mats, xs


def selector_sample(count):
    """Held-out matrices of the selector's labelled set (the split it was
    trained with), every k-th of those with at most 6e6 entries."""
    from paper_1210_2536_gb300 import learn, synth
    recs = learn.load(os.path.join(ROOT, "paper_1210_2536_gb300", "selector_dataset.jsonl"))
    _, held = learn.split(recs)
    held = [r for r in held if r["nnz"] <= 6e6]
    step = max(1, len(held) // max(1, count))
    return [synth.dataset_matrix(r["id"]) for r in held[::step][:count]]


def product_specs(args):
    """(matrix, storage type, x in FP64) for every product of a step."""
    from paper_1210_2536_gb300 import synth
    if args.workload == "structures":
        mats, xs = workload(args.scale)
        return [(A, dt, x) for A, x in zip(mats, xs) for dt in args.dtypes.split(",")]
    if args.workload == "precision":
        A = synth.powerlaw(int(round(8_000_000 * args.scale)), 1.8, 10000, 0)
        x = synth.uniform(0, 1, A.n)
        return [(A, dt, x) for dt in ("f64", "f32", "bf16")]
    if args.workload == "selector":
        return [(A, "f64", synth.uniform(0, 1, A.n)) for A in selector_sample(args.selector_sample)]
    raise ValueError(args.workload)


def stored(A, dtype):
    """Values as handed to the library (FP64 / FP32 host arrays; BF16 as the
    FP64 values, which device_values rounds) and their FP64 widening."""
    if dtype == "f64":
        return A.val, A.val
    v = A.val.astype(np.float32)
    return v, v.astype(np.float64)


def device_values(A, dtype, dev):
    """(values on the device as the library stores them, the same values
    widened to FP64 on the host).  BF16 rounding is the library's own cast."""
    import torch
    import paper_1210_2536_gb300 as smat
    if dtype != "bf16":
        vals, v64 = stored(A, dtype)
        return torch.from_numpy(np.ascontiguousarray(vals)).to(dev), v64
    d64 = torch.from_numpy(A.val).to(dev)
    out = torch.empty(A.nnz, dtype=torch.int16, device=dev)
    if smat.smat_cast_f64_to_bf16(d64.data_ptr(), out.data_ptr(), A.nnz, 0) != 0:
        raise RuntimeError("smat_cast_f64_to_bf16 failed")
    torch.cuda.synchronize()
    bits = out.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return out, bits.view(np.float32).astype(np.float64)


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_mhz_min": min(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def e2e_issue_order(times):
    """Issue order of the end-to-end step, from each product's time alone:
    shortest first, except that the second-longest goes second and the
    longest halfway.  The long kernels then start while later inputs are
    still arriving, do not hold the SMs at the same moment, and their
    outputs return while short kernels run (structures suite, one box, 5
    interleaved runs each: 389 GFLOP/s median against 357 shortest first)."""
    order = sorted(range(len(times)), key=lambda j: times[j])
    if len(order) >= 4:
        longest, second = order[-1], order[-2]
        rest = order[:-2]
        half = len(order) // 2 - 1
        order = rest[:1] + [second] + rest[1:half] + [longest] + rest[half:]
    return order


def break_even_calls(tune_ms, csr_ms, pick_ms):
    """Products after which tuning has paid for itself (Sec. 7.3, Eq.
    "num_iter"): n with tune + n * t_pick = n * t_CSR, i.e. tune / (t_CSR -
    t_pick); None when the pick is not faster than CSR-scalar."""
    if not csr_ms > pick_ms:
        return None
    return tune_ms / (csr_ms - pick_ms)


def dram_traffic_record(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source is unchanged since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if not os.path.exists(path):
        return None
    src = open(os.path.join(ROOT, "paper_1210_2536_gb300", "csrc", "spmv.cu"), "rb").read()
    h = hashlib.sha256(src).hexdigest()[:16]
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kernel_key and cells[3] == h:
            try:
                return float(cells[2])
            except ValueError:
                return None
    return None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(specs, seconds):
    """The oracle (threaded, nonzero-balanced rows, FP64 accumulation) timed
    on this host's cores over passes of the same products; specs are
    (matrix, stored values widened to FP64, x as the product reads it)."""
    import oracle
    threads = os.cpu_count() or 1
    prods = [(A, np.ascontiguousarray(v64), np.ascontiguousarray(np.asarray(x, dtype=np.float64)), np.zeros(A.m))
             for A, v64, x in specs]
    flops = sum(2.0 * A.nnz for A, _, _, _ in prods)
    t0 = time.perf_counter()
    passes = 0
    while True:
        for A, v, x, y in prods:
            oracle.spmv_csr_rows(A.rowptr, A.colidx, v, x, 0, A.m, 1.0, 0.0, y, threads)
        passes += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    # the serial oracle on one core: one full pass over the same products
    t1 = time.perf_counter()
    for A, v, x, y in prods:
        oracle.spmv_csr_rows(A.rowptr, A.colidx, v, x, 0, A.m, 1.0, 0.0, y, 1)
    st = time.perf_counter() - t1
    sflops = flops
    return {"value": round(flops * passes / dt / 1e9, 3), "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{passes} full passes over the {len(prods)} products (all rows), FP64 accumulation, "
                      f"{threads} threads, {dt:.1f} s",
            "serial_1core": {"value": round(sflops / st / 1e9, 3), "unit": UNIT,
                             "sample": f"one full pass over the {len(prods)} products, 1 thread, {st:.2f} s"}}


def batched_mats(scale):
    from paper_1210_2536_gb300 import synth
    top = max(12, int(round(192 * scale ** (1.0 / 3.0))) // 16 * 16)
    return synth.amg_like_hierarchy(top) + synth.mixed_batch(64)


def cg_matrix(scale):
    from paper_1210_2536_gb300 import synth
    return synth.stencil3d7(max(8, int(round(256 * scale ** (1.0 / 3.0)))))


def reference_specs(args):
    """(matrix, stored values widened to FP64, x) of every product a step of
    the workload runs, for the oracle arm."""
    import oracle
    from paper_1210_2536_gb300 import synth
    if args.workload == "batched":
        return [(A, A.val, synth.uniform(0, 1, A.n)) for A in batched_mats(args.scale)]
    if args.workload == "cg":
        L = cg_matrix(args.scale)
        x = synth.uniform(0, 5, L.n)
        return [(L, L.val, x), (L, L.val.astype(np.float32).astype(np.float64), x.astype(np.float32))]
    out = []
    for A, dt, x in product_specs(args):
        if dt == "bf16":
            v64 = oracle.bf16_to_double(oracle.round_bf16(A.val))
        else:
            v64 = stored(A, dt)[1]
        out.append((A, v64, x if dt == "f64" else x.astype(np.float32)))
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    prods = [[A, np.ascontiguousarray(v64), np.ascontiguousarray(np.asarray(x, dtype=np.float64)), np.zeros(A.m), 0]
             for A, v64, x in reference_specs(args)]
    budget_s = 120.0 / max(1, args.steps + args.warmup)
    t0 = time.perf_counter()
    for A, v, x, y, _ in prods:
        r1 = max(1, A.m // 64)
        oracle.spmv_csr_rows(A.rowptr, A.colidx, v, x, 0, r1, 1.0, 0.0, y, threads)
    probe = time.perf_counter() - t0
    frac = min(1.0, max(1e-6, budget_s / max(probe * 64, 1e-9)))

    def step():
        flops = 0.0
        for p in prods:
            A, v, x, y, off = p
            rows = max(1, int(A.m * frac))
            r0 = off if off + rows <= A.m else 0
            oracle.spmv_csr_rows(A.rowptr, A.colidx, v, x, r0, r0 + rows, 1.0, 0.0, y, threads)
            flops += 2.0 * (int(A.rowptr[r0 + rows]) - int(A.rowptr[r0]))
            p[4] = (r0 + rows) % A.m
        return flops

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    total = 0.0
    for _ in range(args.steps):
        total += step()
    dt = time.perf_counter() - t0
    value = total / dt / 1e9
    sample = f"{frac * 100:.3g}% of each product's rows per step ({len(prods)} products), {threads} threads"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / max(1, args.steps), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "scale": args.scale},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_1210_2536_gb300 as smat

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    select = args.select
    model_path = os.path.join(ROOT, "paper_1210_2536_gb300", "selector_mlp.bin")
    if select == "auto":
        select = "learned" if os.path.exists(model_path) else "exhaustive"
    if select == "learned":
        if smat.smat_load_model(model_path) != 0:
            raise RuntimeError("selector model did not load")
    ctx = dict(dev=dev, world=world, rank=rank, select=select)
    if args.workload == "batched":
        line = run_batched(args, ctx)
    elif args.workload == "cg":
        line = run_cg(args, ctx)
    else:
        line = run_products(args, ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def timed_region(K, W, step, world, dev, per_step_events=None):
    """W untimed steps, then K steps between CUDA events on the current
    stream, bracketed by a barrier (N > 1) and a device synchronisation,
    with nvidia-smi clock samples taken meanwhile; returns (max-over-ranks
    ms, clocks).  step(k) issues step k."""
    import torch
    import torch.distributed as dist
    from paper_1210_2536_gb300.dist import max_over_ranks
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = Clocks(vis.split(",")[torch.cuda.current_device()] if vis else str(torch.cuda.current_device()))
    clocks.start()
    time.sleep(0.3)
    # the warm-up runs after the sampler has started, so that the timed
    # region follows busy steps rather than the sampler's idle start-up
    for k in range(W):
        step(-1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    t_start.record()
    for k in range(K):
        step(k)
    t_end.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    return max_over_ranks(t_start.elapsed_time(t_end), dev), ck


def fp64_roof(smat):
    """Measured FP64 roof in TFLOP/s (2 flops per fused multiply-add)."""
    return 2.0 * smat.smat_measure_fp64_rate(10) / 1e12


def run_products(args, ctx):
    import torch
    import torch.distributed as dist
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300.roofline import algorithmic_bytes, l2_sectors
    from paper_1210_2536_gb300.roofline import bound as roof_bound
    from paper_1210_2536_gb300.dist import max_over_ranks, weak_scaling_throughput
    dev, world, rank, select = ctx["dev"], ctx["world"], ctx["rank"], ctx["select"]
    specs = product_specs(args)
    dtypes = sorted({dt for _, dt, _ in specs}, key=["f64", "f32", "bf16"].index)

    prods = []
    for A, dt, x in specs:
        vals, v64 = device_values(A, dt, dev)
        tdt = torch.float64 if dt == "f64" else torch.float32
        t0 = time.perf_counter()
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                          vals, dt)
        torch.cuda.synchronize()
        create_ms = (time.perf_counter() - t0) * 1e3
        del vals
        M.tune(select, keep_formats=0)
        plan = M.plan()
        xd = torch.from_numpy(x).to(dev).to(tdt)
        yd = torch.zeros(A.m, dtype=tdt, device=dev)
        prods.append(dict(A=A, dt=dt, M=M, x=xd, y=yd, v64=v64, plan=plan, create_ms=create_ms,
                          f=M.features(), launches=M.launches()))

    # plain CSR-scalar and tuned pick, each timed alone: the mean of the middle
    # half of 20 repetitions.  With cold=True L2 is flushed before every
    # repetition (a read of twice its size, outside the events, which leaves
    # it holding clean lines of other data, as the other products of the step
    # leave it), and a repetition is one product;
    # otherwise the repetitions run back to back, as the tuner's trials do,
    # each timing enough products (up to 32) to span about 40 us, since the
    # event-timed duration of a single short kernel on this GPU moves in steps
    # of about 2 us.  A device sleep
    # first lets the host queue the repetitions ahead of the GPU, so that no
    # host launch latency falls between a pair of events.
    flush = torch.ones(2 * torch.cuda.get_device_properties(dev).L2_cache_size // 4, dtype=torch.int32,
                       device=dev)

    def time_variant(p, v, reps=20, cold=True):
        M, x, y = p["M"], p["x"], p["y"]
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(2100 * 300)
        w0.record()
        for _ in range(3):
            M.spmv(x, y, variant=v)
        w1.record()
        torch.cuda.synchronize()
        group = 1 if cold else max(1, min(32, math.ceil(0.040 / max(w0.elapsed_time(w1) / 3, 1e-4))))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        hold_us = 500 + reps * (30 * group + (70 if cold else 0))
        for _ in range(3):
            t0 = time.perf_counter()
            torch.cuda._sleep(int(2100 * hold_us))    # cycles at about 2.1 GHz
            for s, e in ev:
                if cold:
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
        return statistics.mean(t[q:len(t) - q])

    for p in prods:
        p["csr_ms"] = time_variant(p, smat.SMAT_V_CSR_SCALAR)
        p["pick_ms"] = time_variant(p, p["plan"]["variant"])

    # ---- timed region: K steps of all products through their plans ----
    K, W = args.steps, args.warmup
    # per-product events on every 8th step (at most 50 steps): an event
    # between two kernels costs idle GPU time (the step's eight products ran
    # in 0.512 ms without events, 0.57 ms with a pair around each), and such
    # a step runs its products one after another (0.50 ms against 0.47 ms
    # side by side), which the steps without them do not pay
    stride = max(8, K // 50)
    sampled = list(range(stride // 2, K, stride)) or [0]
    # one event between consecutive products: product j runs between events
    # j and j + 1 of its step
    kev = {i: [torch.cuda.Event(enable_timing=True) for _ in range(len(prods) + 1)] for i in sampled}

    # The products of a step are independent.  Steps that carry per-product
    # events run them one after another on the current stream (those give
    # each product's own time); the others, with --concurrent, go through
    # smat_spmv_many, which runs them side by side on the library's streams,
    # ordered after and before the current stream's work, so that
    # gather-bound and bandwidth-bound products overlap.
    many = ([p["M"] for p in prods], [p["x"] for p in prods], [p["y"] for p in prods])

    def step(k):
        evs = kev.get(k)
        if args.concurrent and not evs:
            smat.spmv_many(*many)
            return
        if evs:
            evs[0].record()
        for j, p in enumerate(prods):
            p["M"].spmv(p["x"], p["y"])
            if evs:
                evs[j + 1].record()

    ms, ck = timed_region(K, W, step, world, dev)
    flops_step = sum(2.0 * p["A"].nnz for p in prods)
    value = weak_scaling_throughput(flops_step * K, ms / 1e3, world) / 1e9
    launches_per_step = sum(p["launches"] for p in prods)

    peak, peak_kind = measured_peak()
    fp64_tf = fp64_roof(smat)
    per = []
    for j, p in enumerate(prods):
        d = statistics.mean(kev[i][j].elapsed_time(kev[i][j + 1]) for i in sampled)
        byts = algorithmic_bytes(p["f"], p["plan"]["variant"], p["dt"])
        csr_bytes = algorithmic_bytes(p["f"], smat.SMAT_V_CSR_SCALAR, p["dt"])
        be = break_even_calls(p["plan"]["tune_ms"], p["csr_ms"], p["pick_ms"])
        per.append({"matrix": p["A"].name, "dtype": p["dt"], "nnz": p["A"].nnz, "variant": p["plan"]["name"],
                    "kernel": kernel_label(p["M"], p["plan"]["variant"]),
                    "confidence": round(p["plan"]["confidence"], 3), "trialled": p["plan"]["trialled"],
                    "ms_in_step": round(d, 5), "gflops": round(2 * p["A"].nnz / d / 1e6, 2),
                    "hbm_frac": round(byts / (d / 1e3) / 1e9 / peak, 4),
                    "bound": roof_bound(p["f"], p["plan"]["variant"], p["dt"], d / 1e3, peak, fp64_tf)["bound"],
                    "roof_frac": round(roof_bound(p["f"], p["plan"]["variant"], p["dt"], d / 1e3, peak, fp64_tf)["frac"], 4),
                    "pick_ms_alone": round(p["pick_ms"], 5), "csr_scalar_ms_alone": round(p["csr_ms"], 5),
                    "csr_scalar_gflops": round(2 * p["A"].nnz / p["csr_ms"] / 1e6, 2),
                    "csr_scalar_hbm_frac": round(csr_bytes / (p["csr_ms"] / 1e3) / 1e9 / peak, 4),
                    "speedup_vs_csr_scalar": round(p["csr_ms"] / p["pick_ms"], 3),
                    "tune_ms": round(p["plan"]["tune_ms"], 2),
                    "tune_overhead_csr_spmvs": round(p["plan"]["tune_ms"] / p["csr_ms"], 1),
                    "break_even_calls": None if be is None else round(be, 1),
                    "alg_bytes": byts, "_d": d})
    dom_i = max(range(len(per)), key=lambda j: per[j]["_d"])
    dom, dp = per[dom_i], prods[dom_i]
    dom_key = f"{dom['variant']}:{dom['dtype']}:{dom['matrix']}"
    rb = roof_bound(dp["f"], dp["plan"]["variant"], dp["dt"], dom["_d"] / 1e3, peak, fp64_tf)
    traffic = dram_traffic_record(dom_key)
    # random-column products are bound by x gathers before HBM: the measured
    # gather rate of this GPU over the dominant product's own x and count
    gather_peak = smat.smat_measure_gather_rate(dp["A"].n, dp["A"].nnz, dp["dt"], 20)
    gather_frac = dp["A"].nnz / (dom["_d"] / 1e3) / gather_peak
    # the same measurement as a rate of L2 sector requests (each gather one
    # sector, each streamed 4-byte index 1/8 of one), against the dominant
    # product's own requests: its gathers plus its streamed format bytes
    sector_peak = gather_peak * (1.0 + 4.0 / 32.0)
    sectors = l2_sectors(dp["f"], dp["plan"]["variant"], dp["dt"])
    sector_frac = sectors / (dom["_d"] / 1e3) / sector_peak
    for r in per:
        r.pop("_d")
        r.pop("alg_bytes")

    # ---- end to end: inputs from pinned host memory, results back to it ----
    # Beside the host-buffer calls below, the device-pointer calls with the
    # transfers arranged by the caller ("packed"): each storage type's x of all
    # products sit in one pinned host buffer and one device buffer, their y
    # likewise, so that each direction is one copy per storage type; two sets
    # of device buffers alternate between steps, and copies in, the products
    # (side by side through smat_spmv_many) and copies out run on three
    # streams, so that one set's transfers overlap the other set's products.
    # A step's copies in wait until the products two steps back have read
    # that set's x, its products until that set's previous copies out have
    # read y, its copies out until its products are done; the timed region
    # ends when every y is on the host.
    def packed(sizes):
        offs, o = [], 0
        for k in sizes:
            offs.append(o)
            o += (k + 31) // 32 * 32            # every vector 128-byte aligned or more
        return offs, o
    tdts = sorted({p["x"].dtype for p in prods}, key=str)
    grp = {t: [j for j, p in enumerate(prods) if p["x"].dtype == t] for t in tdts}
    xoff, yoff, xtot, ytot = {}, {}, {}, {}
    for t, js in grp.items():
        xo, xtot[t] = packed([prods[j]["A"].n for j in js])
        yo, ytot[t] = packed([prods[j]["A"].m for j in js])
        xoff.update(zip(js, xo))
        yoff.update(zip(js, yo))
    xh_pack = {t: torch.zeros(xtot[t], dtype=t).pin_memory() for t in tdts}
    for j, p in enumerate(prods):
        xh_pack[p["x"].dtype][xoff[j]:xoff[j] + p["A"].n] = p["x"].cpu()
    yh_pack = [{t: torch.zeros(ytot[t], dtype=t).pin_memory() for t in tdts} for _ in range(2)]
    Xd = [{t: torch.zeros(xtot[t], dtype=t, device=dev) for t in tdts} for _ in range(2)]
    Yd = [{t: torch.zeros(ytot[t], dtype=t, device=dev) for t in tdts} for _ in range(2)]
    xv = [[Xd[q][p["x"].dtype][xoff[j]:xoff[j] + p["A"].n] for j, p in enumerate(prods)] for q in range(2)]
    yv = [[Yd[q][p["x"].dtype][yoff[j]:yoff[j] + p["A"].m] for j, p in enumerate(prods)] for q in range(2)]
    mats = [p["M"] for p in prods]
    s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    run_done = [torch.cuda.Event(), torch.cuda.Event()]
    out_done = [torch.cuda.Event(), torch.cuda.Event()]
    x_ready = [torch.cuda.Event(), torch.cuda.Event()]
    for q in range(2):
        run_done[q].record(s_run)
        out_done[q].record(s_out)
    n_e2e = [0]

    def e2e_pipelined():
        q = n_e2e[0] % 2
        n_e2e[0] += 1
        s_in.wait_event(run_done[q])
        with torch.cuda.stream(s_in):
            for t in tdts:
                Xd[q][t].copy_(xh_pack[t], non_blocking=True)
        x_ready[q].record(s_in)
        s_run.wait_event(x_ready[q])
        s_run.wait_event(out_done[q])
        if args.concurrent:
            smat.spmv_many(mats, xv[q], yv[q], stream=s_run)
        else:
            for M, x, y in zip(mats, xv[q], yv[q]):
                M.spmv(x, y, stream=s_run)
        run_done[q].record(s_run)
        s_out.wait_event(run_done[q])
        with torch.cuda.stream(s_out):
            for t in tdts:
                yh_pack[q][t].copy_(Yd[q][t], non_blocking=True)
        out_done[q].record(s_out)

    e2e_pipelined()
    e2e_pipelined()
    torch.cuda.synchronize()
    # the products that came back equal the ones timed above (same x)
    for q in range(2):
        for j, p in enumerate(prods):
            ref = p["y"].cpu()
            got = yh_pack[q][p["x"].dtype][yoff[j]:yoff[j] + p["A"].m]
            err = (got - ref).abs().max().item() if p["A"].m else 0.0
            if not err <= 1e-12 * max(ref.abs().max().item() if p["A"].m else 0.0, 1e-300):
                raise RuntimeError(f"end-to-end product of {p['A'].name} {p['dt']} differs from the timed one ({err:g})")

    # Through the C ABI with host buffers (the figure reported as e2e):
    # smat_spmv_host_pipelined per product from its own pinned x and y: each
    # handle copies in, computes and copies out on streams of its own with two
    # staging sets used in turn, so one step's transfers overlap the previous
    # step's products and the products of different handles overlap each
    # other; the current stream waits for every copy out, and the timed region
    # ends when it is done (all y on the host).  Issued in e2e_issue_order's
    # order; two pinned y buffers per product alternate between steps, so two
    # steps in flight never write the same host buffer.  Reported beside it:
    # smat_spmv_host_async per product on a stream of its own (the handle's
    # single staging set), every step synchronised.
    pinned = []
    for p in prods:
        pinned.append((p["x"].cpu().pin_memory(),
                       [torch.zeros(p["A"].m, dtype=p["x"].dtype).pin_memory() for _ in range(2)]))
    h2d = sum(xh.numel() * xh.element_size() for xh, _ in pinned)
    d2h = sum(yh[0].numel() * yh[0].element_size() for _, yh in pinned)
    order = e2e_issue_order([p["pick_ms"] for p in prods])
    streams = [torch.cuda.Stream() for _ in range(len(prods))]
    n_host = [0]

    def e2e_host_pipelined():
        q = n_host[0] % 2
        n_host[0] += 1
        for j in order:
            xh, yh = pinned[j]
            prods[j]["M"].spmv_host_pipelined(xh, yh[q])

    def e2e_host_synced():
        for j in order:
            xh, yh = pinned[j]
            prods[j]["M"].spmv_host_async(xh, yh[0], stream=streams[j])
        for st in streams:
            st.synchronize()

    e2e_host_pipelined()
    e2e_host_pipelined()
    e2e_host_synced()
    torch.cuda.synchronize()
    E = max(2, args.e2e_steps)
    e2e_rates = {}
    for mode, fn in (("pipelined", e2e_host_pipelined), ("synced", e2e_host_synced), ("packed", e2e_pipelined)):
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(E):
            fn()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
        e2e_rates[mode] = weak_scaling_throughput(flops_step * E, e2e_s, world) / 1e9
    e2e_value = e2e_rates["pipelined"]

    extra = selector_regret(prods, time_variant) if args.workload == "selector" else None
    line = None
    if rank == 0:
        cpu = cpu_baseline([(p["A"], p["v64"], p["x"].double().cpu().numpy()) for p in prods], args.cpu_seconds) \
            if world == 1 else None
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(ms / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "+".join(dtypes), "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "scale": args.scale, "selector": select,
                       "streams": ("smat_spmv_many (the products side by side on library streams) on the "
                                   f"steps without per-product events; every {stride}th step carries them and "
                                   "runs its products one after another on one stream")
                       if args.concurrent else "one stream",
                       "l2": "inputs larger than L2: the step streams "
                             f"{sum(algorithmic_bytes(p['f'], p['plan']['variant'], p['dt']) for p in prods) / 1e6:.0f}"
                             " MB and each matrix is evicted by the other products between its launches",
                       "parallelism": f"replicas x{world}"},
            "parity": {"bound": {dt: TOL[dt] for dt in dtypes}, "checked_by": PARITY_TESTS[args.workload]},
            "roofline": {"bound": rb["bound"], "kernel": dom_key, "achieved": round(rb["achieved"], 3),
                         "peak": round(rb["peak"], 4),
                         "peak_kind": (peak_kind if rb["bound"] == "hbm" else
                                       "measured: smat_measure_fp64_rate (FP64 fused multiply-adds x 2)"),
                         "unit": rb["unit"], "frac": round(rb["frac"], 4), "traffic": traffic,
                         "alg_bytes_per_launch": rb["alg_bytes"], "hbm_frac": round(rb["hbm_frac"], 4),
                         "fp64_frac": round(rb["fp64_frac"], 4) if "fp64_frac" in rb else None,
                         "gather_peak_gps": round(gather_peak / 1e9, 1), "gather_frac": round(gather_frac, 4),
                         "l2_sectors_per_launch": sectors, "l2_sector_peak_gps": round(sector_peak / 1e9, 1),
                         "l2_sector_frac": round(sector_frac, 4)},
            "step_hbm_frac": round(sum(algorithmic_bytes(p["f"], p["plan"]["variant"], p["dt"]) for p in prods)
                                   / (ms / K / 1e3) / 1e9 / peak, 4),
            "gpu_launches": launches_per_step * K,
            "clocks": ck,
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": E,
                    "how": "smat_spmv_host_pipelined (the C ABI's host-buffer call on the handle's own streams "
                           "and two staging sets) per product from pinned host x/y, issued shortest first with the "
                           "two longest at the second and middle places; steps pipelined, the current stream "
                           "waiting for every copy out, synced at the end of the timed region",
                    "synced_per_step": round(e2e_rates["synced"], 3),
                    "synced_how": "smat_spmv_host_async per product on a stream of its own, every step synchronised",
                    "packed_device_api": {
                        "value": round(e2e_rates["packed"], 3),
                        "how": "the device-pointer calls with the transfers arranged by the caller: each storage "
                               "type's x of all products copied from one pinned host buffer as one transfer, the "
                               "products side by side (smat_spmv_many), the y copied back as one transfer per "
                               "storage type; two sets of device buffers alternate between steps; copies in, "
                               "products and copies out on three streams; same bytes per step"}},
            "cpu_baseline": cpu,
            "per_matrix": per,
        }
        if extra is not None:
            line["selector"] = extra
    for p in prods:
        p["M"].close()
    return line


def batch_kind(variant):
    """Format kind of the batched kernel a member's plan runs through."""
    return {5: "ell", 6: "dia", 10: "sell"}.get(variant, "csr")


def run_batched(args, ctx):
    """One batched launch (the autotuned plan: persistent kernels per format
    kind in a CUDA graph, or the members' own launches when faster) over the
    multigrid-like hierarchy and 64 mixed matrices, FP64."""
    import torch
    import torch.distributed as dist
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    from paper_1210_2536_gb300.roofline import algorithmic_bytes
    from paper_1210_2536_gb300.dist import max_over_ranks, weak_scaling_throughput
    dev, world, rank, select = ctx["dev"], ctx["world"], ctx["rank"], ctx["select"]
    mats = batched_mats(args.scale)
    hs, xs, ys, x64 = [], [], [], []
    for A in mats:
        M = smat.SpMatrix(A.m, A.n, torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                          torch.from_numpy(A.val).to(dev), "f64")
        M.tune(select, keep_formats=0)
        hs.append(M)
        x = synth.uniform(0, 1, A.n)
        x64.append(x)
        xs.append(torch.from_numpy(x).to(dev))
        ys.append(torch.zeros(A.m, dtype=torch.float64, device=dev))
    nnz = sum(A.nnz for A in mats)
    plans = [M.plan()["variant"] for M in hs]
    byts = sum(algorithmic_bytes(M.features(), v, "f64") for M, v in zip(hs, plans))
    t0 = time.perf_counter()
    B = smat.Batch(hs).tune()
    tune_s = time.perf_counter() - t0
    info = B.info()

    def time_it(fn, reps=20):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    def per_matrix():
        for M, x, y in zip(hs, xs, ys):
            M.spmv(x, y)

    t_loop = time_it(per_matrix)
    K, W = args.steps, args.warmup
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]

    def step(k):
        if k >= 0:
            evs[k][0].record()
        B.spmv(xs, ys)
        if k >= 0:
            evs[k][1].record()

    ms, ck = timed_region(K, W, step, world, dev)
    d = statistics.mean(a.elapsed_time(b) for a, b in evs)
    value = weak_scaling_throughput(2.0 * nnz * K, ms / 1e3, world) / 1e9
    peak, peak_kind = measured_peak()
    if info["per_matrix"]:
        launches = sum(M.launches() for M in hs)
    else:
        launches = len({batch_kind(v) for v in plans})

    # end to end: all members' x in one pinned host buffer and all y back
    # into one, copied as one transfer each way (one copy per member made
    # the 138 small copies the bound).  Two sets of device buffers, each with
    # its own batch over the same handles (a batch's graph keeps its members'
    # pointers), so that a step's copies overlap the other set's product:
    # the copies in of a step wait until the product two steps back has read
    # that set's x, its product until that set's previous copies out have
    # read y, and its copies out until its product is done.
    def packed(sizes):
        offs, o = [], 0
        for k in sizes:
            offs.append(o)
            o += (k + 31) // 32 * 32            # every member 256-byte aligned
        return offs, o
    xoff, xtot = packed([A.n for A in mats])
    yoff, ytot = packed([A.m for A in mats])
    xh_all = torch.zeros(xtot, dtype=torch.float64).pin_memory()
    for o, x in zip(xoff, x64):
        xh_all[o:o + len(x)] = torch.from_numpy(x)
    yh_all = [torch.zeros(ytot, dtype=torch.float64).pin_memory() for _ in range(2)]
    X = [torch.zeros(xtot, dtype=torch.float64, device=dev) for _ in range(2)]
    Y = [torch.zeros(ytot, dtype=torch.float64, device=dev) for _ in range(2)]
    xs_set = [[X[q][o:o + A.n] for o, A in zip(xoff, mats)] for q in range(2)]
    ys_set = [[Y[q][o:o + A.m] for o, A in zip(yoff, mats)] for q in range(2)]
    B2 = smat.Batch(hs).tune(tile_scale=info["tile_scale"], ctas_per_sm=info["ctas_per_sm"],
                             own_launches=info["own_launches"],
                             mode=2 if info["per_matrix"] else 1)   # the plan B chose
    Bs = [B, B2]
    s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    run_done = [torch.cuda.Event(), torch.cuda.Event()]
    out_done = [torch.cuda.Event(), torch.cuda.Event()]
    x_ready = [torch.cuda.Event(), torch.cuda.Event()]
    for q in range(2):
        run_done[q].record(s_run)
        out_done[q].record(s_out)
    n_e2e = [0]

    def e2e_step():
        q = n_e2e[0] % 2
        n_e2e[0] += 1
        s_in.wait_event(run_done[q])
        with torch.cuda.stream(s_in):
            X[q].copy_(xh_all, non_blocking=True)
        x_ready[q].record(s_in)
        s_run.wait_event(x_ready[q])
        s_run.wait_event(out_done[q])
        Bs[q].spmv(xs_set[q], ys_set[q], stream=s_run)
        run_done[q].record(s_run)
        s_out.wait_event(run_done[q])
        with torch.cuda.stream(s_out):
            yh_all[q].copy_(Y[q], non_blocking=True)
        out_done[q].record(s_out)

    e2e_step()
    e2e_step()
    torch.cuda.synchronize()
    # the packed copies hold the same products as the per-member buffers
    for q in range(2):
        for o, y, A in zip(yoff, ys, mats):
            ref = y.cpu()
            err = (yh_all[q][o:o + A.m] - ref).abs().max().item() if A.m else 0.0
            if not err <= 1e-12 * max(ref.abs().max().item() if A.m else 0.0, 1e-300):
                raise RuntimeError(f"end-to-end product of {A.name} differs from the timed product ({err:g})")
    E = max(2, min(args.e2e_steps, 50))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(E):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    line = None
    if rank == 0:
        cpu = cpu_baseline([(A, A.val, x) for A, x in zip(mats, x64)], args.cpu_seconds) if world == 1 else None
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(ms / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["batched"], "scale": args.scale, "selector": select,
                       "matrices": len(mats), "nnz": nnz,
                       "l2": f"inputs larger than L2: a step streams {byts / 1e6:.0f} MB",
                       "parallelism": f"replicas x{world}"},
            "parity": {"bound": {"f64": TOL["f64"]}, "checked_by": PARITY_TESTS["batched"]},
            "roofline": {"bound": "hbm", "kernel": "batched launch (one persistent kernel per format kind, "
                                                   "graph-replayed; or the members' own launches)",
                         "achieved": round(byts / (d / 1e3) / 1e9, 3), "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": round(byts / (d / 1e3) / 1e9 / peak, 4), "traffic": None,
                         "alg_bytes_per_launch": byts},
            "gpu_launches": launches * K,
            "clocks": ck,
            "e2e": {"value": round(weak_scaling_throughput(2.0 * nnz * E, e2e_s, world) / 1e9, 3), "unit": UNIT,
                    "h2d_bytes_per_step": xh_all.numel() * 8,
                    "d2h_bytes_per_step": yh_all[0].numel() * 8, "steps": E,
                    "how": "all members' x copied from one pinned host buffer as one transfer, one batched "
                           "product, all y copied back as one transfer; two sets of device buffers, each "
                           "with its own batch over the same handles, alternate between steps; copies in, "
                           "product and copies out on three streams ordered by events, steps pipelined and "
                           "synced at the end"},
            "cpu_baseline": cpu,
            "batched": {"batched_ms": round(d, 5), "per_matrix_launches_ms": round(t_loop, 5),
                        "speedup_vs_per_matrix": round(t_loop / d, 3), "batch_info": info,
                        "batch_tune_s": round(tune_s, 2),
                        "picks": {smat.VARIANT_NAMES[v]: plans.count(v) for v in sorted(set(plans))}},
        }
    B.close()
    B2.close()
    for M in hs:
        M.close()
    return line


def run_cg(args, ctx):
    """Mixed-precision CG on the 3-D 7-point Laplacian: each step is a solve
    from x = 0 capped at 500 inner FP32 iterations; the metric counts the
    SpMV flops it ran (inner FP32 products plus the FP64 residual products)."""
    import torch
    import torch.distributed as dist
    import paper_1210_2536_gb300 as smat
    from paper_1210_2536_gb300 import synth
    from paper_1210_2536_gb300.roofline import algorithmic_bytes
    from paper_1210_2536_gb300.dist import max_over_ranks, weak_scaling_throughput
    dev, world, rank, select = ctx["dev"], ctx["world"], ctx["rank"], ctx["select"]
    L = cg_matrix(args.scale)
    rp, ci = torch.from_numpy(L.rowptr).to(dev), torch.from_numpy(L.colidx).to(dev)
    H64 = smat.SpMatrix(L.m, L.n, rp, ci, torch.from_numpy(L.val).to(dev), "f64").tune(select)
    H32 = smat.SpMatrix(L.m, L.n, rp, ci, torch.from_numpy(L.val.astype(np.float32)).to(dev), "f32").tune(select)
    xt = synth.uniform(0, 5, L.n)
    bd = H64.spmv(torch.from_numpy(xt).to(dev))        # b = A x_true on the device
    xd = torch.zeros(L.n, dtype=torch.float64, device=dev)
    inner = 500
    last = {}

    def step(k):
        xd.zero_()
        last.update(smat.cg_mixed(H64, H32, bd, xd, max_total_inner=inner, rtol=1e-10, max_inner=inner))

    K, W = args.steps, max(1, args.warmup)
    ms, ck = timed_region(K, W, step, world, dev)
    products32 = last["inner_total"]
    products64 = last["outer"] + 1
    flops_step = 2.0 * L.nnz * (products32 + products64)
    value = weak_scaling_throughput(flops_step * K, ms / 1e3, world) / 1e9
    # the inner FP32 product, timed alone, against its roof
    x32 = torch.from_numpy(synth.uniform(1, 1, L.n).astype(np.float32)).to(dev)
    y32 = torch.zeros(L.n, dtype=torch.float32, device=dev)
    for _ in range(3):
        H32.spmv(x32, y32)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in ev:
        a.record()
        H32.spmv(x32, y32)
        b.record()
    torch.cuda.synchronize()
    t32 = statistics.median(a.elapsed_time(b) for a, b in ev)
    peak, peak_kind = measured_peak()
    f32 = H32.features()
    b32 = algorithmic_bytes(f32, H32.plan()["variant"], "f32")
    # the solve to 1e-10 (5000 inner iterations at most), once, outside the timed region
    xd.zero_()
    full = smat.cg_mixed(H64, H32, bd, xd, max_total_inner=5000, rtol=1e-10, max_inner=2000)
    # end to end: b from pinned host memory, the capped solve, x back to the host
    bh = bd.cpu().pin_memory()
    xh = torch.zeros(L.n, dtype=torch.float64).pin_memory()

    def e2e_step():
        bd.copy_(bh, non_blocking=True)
        xd.zero_()
        smat.cg_mixed(H64, H32, bd, xd, max_total_inner=inner, rtol=1e-10, max_inner=inner)
        xh.copy_(xd, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    E = max(1, min(args.e2e_steps, 10))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(E):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    line = None
    if rank == 0:
        cpu = cpu_baseline([(L, L.val, xt), (L, L.val.astype(np.float32).astype(np.float64),
                                             xt.astype(np.float32).astype(np.float64))], args.cpu_seconds) \
            if world == 1 else None
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": round(ms / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["cg"], "scale": args.scale, "selector": select, "n": L.n,
                       "nnz": L.nnz, "l2": "inputs larger than L2: each FP32 product streams "
                                            f"{b32 / 1e6:.0f} MB",
                       "parallelism": f"replicas x{world}"},
            "parity": {"bound": {"f64": TOL["f64"], "f32": TOL["f32"], "relres": 1e-10},
                       "checked_by": PARITY_TESTS["cg"]},
            "roofline": {"bound": "hbm", "kernel": f"inner FP32 product ({H32.plan()['name']}), timed alone",
                         "achieved": round(b32 / (t32 / 1e3) / 1e9, 3), "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": round(b32 / (t32 / 1e3) / 1e9 / peak, 4), "traffic": None,
                         "alg_bytes_per_launch": b32},
            "gpu_launches": None,
            "clocks": ck,
            "e2e": {"value": round(weak_scaling_throughput(flops_step * E, e2e_s, world) / 1e9, 3), "unit": UNIT,
                    "h2d_bytes_per_step": L.n * 8, "d2h_bytes_per_step": L.n * 8, "steps": E,
                    "how": "b from pinned host memory, the capped solve through smat_cg_mixed, x back to the host"},
            "cpu_baseline": cpu,
            "cg": {"inner_per_step": products32, "outer_per_step": last["outer"],
                   "relres_after_step": last["relres"], "fp32_product_ms": round(t32, 5),
                   "plans": {"f64": H64.plan()["name"], "f32": H32.plan()["name"]},
                   "to_1e-10": {"inner_total": full["inner_total"], "outer": full["outer"],
                                "relres": full["relres"], "seconds": round(full["seconds"], 4),
                                "converged": full["converged"]}},
        }
    H64.close()
    H32.close()
    return line


def kernel_label(M, variant):
    """The kernel behind a DIA / ELL plan (measured per handle), else None."""
    import paper_1210_2536_gb300 as smat
    names = {smat.SMAT_V_DIA: ("direct", "staged1", "staged2"),
             smat.SMAT_V_ELL: ("rows", "lanes")}
    if variant not in names:
        return None
    try:
        return names[variant][M.kernel(variant)]
    except Exception:
        return None


def selector_regret(prods, time_variant):
    """Regret of each tuned pick (learned selector plus its execute-and-
    measure fallback over the further formats) against the fastest variant
    the library can run on that matrix: the eight classes of Sec. 5 and the
    further formats, every one that builds timed alone here (the mean of the
    middle half of 20 repetitions), the pick among them in the same loop.  Measured twice: with the
    repetitions back to back as the tuner's trials run them (`warm`, the
    conditions the selector's labels were taken under), and with L2 flushed
    before each (`cold_l2`, the conditions of the step, whose other products
    evict each matrix).  The paper's accuracy and slowdown of the prediction
    (Sec. 7.3), live on this GPU."""
    import paper_1210_2536_gb300 as smat
    import torch
    further = (smat.SMAT_V_HYB, smat.SMAT_V_SELL, smat.SMAT_V_BCSR, smat.SMAT_V_SPLIT)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    dev_idx = torch.cuda.current_device() if torch.cuda.is_available() else 0
    out = {}
    for mode, cold in (("warm", False), ("cold_l2", True)):
        clocks = Clocks(vis.split(",")[dev_idx] if vis else str(dev_idx))
        clocks.start()
        rows = []
        for p in prods:
            adm = p["f"]["admissible"]
            pick = p["plan"]["variant"]
            t = {}
            for v in sorted({v for v in range(smat.SMAT_NUM_VARIANTS) if (adm >> v) & 1} | set(further) | {pick}):
                try:
                    t[v] = time_variant(p, v, cold=cold)
                except smat.SmatError:        # a further format this matrix does not admit
                    if v == pick:
                        raise
            best_v = min(t, key=t.get)
            rows.append({"matrix": p["A"].name, "pick": p["plan"]["name"], "best": smat.VARIANT_NAMES[best_v],
                         "regret": round(t[pick] / t[best_v] - 1.0, 4), "hit": t[pick] <= 1.02 * t[best_v],
                         "trialled": p["plan"]["trialled"], "confidence": round(p["plan"]["confidence"], 3),
                         "us": {smat.VARIANT_NAMES[v]: round(ms * 1e3, 2) for v, ms in t.items()},
                         "tuner_us": {smat.VARIANT_NAMES[v]: round(float(ms) * 1e3, 2)
                                      for v, ms in enumerate(p["M"].timings()) if ms > 0}})
        reg = sorted(r["regret"] for r in rows)
        out[mode] = {"matrices": len(rows), "mean_regret": round(sum(reg) / len(reg), 4),
                     "p90_regret": reg[min(len(reg) - 1, int(0.9 * len(reg)))], "max_regret": reg[-1],
                     "accuracy_within_2pct": round(sum(r["hit"] for r in rows) / len(rows), 4),
                     "clocks": clocks.stop(), "rows": rows}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
