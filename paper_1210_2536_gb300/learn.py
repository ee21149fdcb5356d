"""Offline stage of the learned selector (the counterpart of the paper's data
mining stage, Sec. 5): label seeded synthetic matrices with measured
timings, train the MLP on the GPU with libsmat's own kernels, and evaluate it
on held-out matrices against the exhaustive search (regret) and against the
paper's rules.

  python -m paper_1210_2536_gb300.learn label --out ds.jsonl [--count 2400]
  python -m paper_1210_2536_gb300.learn train --data ds.jsonl --model m.bin --report r.json
  python -m paper_1210_2536_gb300.learn influence --data ds.jsonl --out influence.json

Dataset line (JSON): id, kind, params, m, n, nnz, features (12 selector
inputs), admissible mask, timings_ms[8] (-1 = not admissible), rules pick.
Labelling appends one line per matrix and resumes after the last id present.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import time

import numpy as np

from . import synth

NV = 8
TIE = 1.02  # variants within 2 % of the fastest are all correct labels (Sec. 7.3 counts near-ties as hits)


# ---------------------------------------------------------------------------
# Labelling
# ---------------------------------------------------------------------------

def _generate_pinned(kind, params, seed, torch):
    """A CSR matrix generated straight into pinned host buffers."""
    L = synth.lib()
    p = (ctypes.c_double * 4)(*(list(map(float, params)) + [0.0] * (4 - len(params))))
    nr, nc = ctypes.c_int64(), ctypes.c_int64()
    L.synth_dims(kind, p, ctypes.byref(nr), ctypes.byref(nc))
    m, n = nr.value, nc.value
    rowlen = np.empty(m, dtype=np.int32)
    L.synth_rowlen(kind, p, seed, rowlen.ctypes.data, 0)
    rp64 = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(rowlen, out=rp64[1:])
    nnz = int(rp64[-1])
    col = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
    val = torch.empty(nnz, dtype=torch.float64, pin_memory=True)
    L.synth_fill(kind, p, seed, rp64.ctypes.data, col.data_ptr(), val.data_ptr(), 0)
    rp = torch.from_numpy(rp64.astype(np.int32)).pin_memory()
    return m, n, nnz, rp, col, val


def label(out_path, count=synth.DATASET_SIZE, start=0, reps=7, budget_ms=20000.0, log_every=50):
    import torch

    import paper_1210_2536_gb300 as smat
    done = set()
    if os.path.exists(out_path):
        for line in open(out_path):
            try:
                done.add(json.loads(line)["id"])
            except Exception:
                pass
    dev = torch.device("cuda:0")
    t0 = time.time()
    with open(out_path, "a") as fout:
        for mid in range(start, count):
            if mid in done:
                continue
            kind, params, seed = synth.dataset_spec(mid)
            m, n, nnz, rp, col, val = _generate_pinned(kind, params, seed, torch)
            d_rp, d_col, d_val = rp.to(dev, non_blocking=True), col.to(dev, non_blocking=True), val.to(dev,
                                                                                                        non_blocking=True)
            torch.cuda.synchronize()
            M = smat.SpMatrix(m, n, d_rp, d_col, d_val, "f64")
            del d_rp, d_col, d_val
            feats = M.features()
            fv = M.feature_vector()
            M.tune("rules")
            rules_pick = M.plan()["variant"]
            # the selector's 8 classes only (the further formats are not classes)
            # every class timed fully (no racing): the labels are all 8 medians
            M.tune("exhaustive", trial_reps=reps, trial_warmup=2, trial_budget_ms=budget_ms, allowed=0xFF,
                   trial_race=0.0)
            tm = M.timings()[:8]
            tune_ms = M.plan()["tune_ms"]
            M.close()
            rec = {"id": mid, "kind": synth.KIND_NAMES[kind], "params": [float(v) for v in params], "m": m, "n": n,
                   "nnz": nnz, "features": [float(v) for v in fv], "admissible": int(feats["admissible"]),
                   "timings_ms": [float(v) for v in tm], "rules": int(rules_pick), "exhaustive_tune_ms": tune_ms,
                   "raw": {k: feats[k] for k in ("max_rd", "min_rd", "ndiags", "ntdiags", "var_rd", "er_dia",
                                                  "er_ell", "r", "r_valid")}}
            fout.write(json.dumps(rec) + "\n")
            fout.flush()
            if log_every and (mid + 1) % log_every == 0:
                print(f"labelled {mid + 1}/{count}  {time.time() - t0:.0f}s", flush=True)
            del rp, col, val


# ---------------------------------------------------------------------------
# Dataset helpers
# ---------------------------------------------------------------------------

def load(path):
    recs = [json.loads(l) for l in open(path) if l.strip()]
    recs.sort(key=lambda r: r["id"])
    return recs


def split(recs, every=5):
    """Held-out split stratified by generator kind: within each kind, every
    `every`-th matrix (by id) is held out (1922 / 478 for the 2400 matrices)."""
    by = {}
    for r in recs:
        by.setdefault(r["kind"], []).append(r)
    train, held = [], []
    for kind in sorted(by):
        for j, r in enumerate(sorted(by[kind], key=lambda r: r["id"])):
            (held if j % every == every - 1 else train).append(r)
    return train, held


def arrays(recs):
    X = np.array([r["features"] for r in recs], dtype=np.float64)
    T = np.array([r["timings_ms"] for r in recs], dtype=np.float64)
    adm = np.array([[(r["admissible"] >> v) & 1 for v in range(NV)] for r in recs], dtype=bool)
    T = np.where(adm & (T > 0), T, np.inf)
    return X, T, adm


def soft_targets(T):
    best = T.min(axis=1, keepdims=True)
    hit = (T <= TIE * best) & np.isfinite(T)
    return hit / hit.sum(axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# Training on the GPU with libsmat's MLP kernels
# ---------------------------------------------------------------------------

def init_params(seed=0):
    rng = np.random.default_rng(seed)
    p = []
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 8)):
        bound = math.sqrt(6.0 / fan_in)
        p.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)).ravel())
        p.append(np.zeros(fan_out))
    return np.concatenate(p).astype(np.float32)


def train(recs, epochs=400, batch=128, lr=3e-3, seed=0, log=None):
    import torch

    import paper_1210_2536_gb300 as smat
    dev = torch.device("cuda:0")
    X, T, adm = arrays(recs)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std < 1e-6] = 1.0
    Xs = torch.tensor((X - mean) / std, dtype=torch.float32, device=dev)
    Y = torch.tensor(soft_targets(T), dtype=torch.float32, device=dev)
    B = len(recs)
    p = torch.tensor(init_params(seed), device=dev)
    m1, v1 = torch.zeros_like(p), torch.zeros_like(p)
    g = torch.zeros_like(p)
    loss = torch.zeros(1, device=dev)
    work = torch.empty(smat.smat_mlp_work_floats(batch), device=dev)
    rng = np.random.default_rng(seed + 1)
    step = 0
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(B)).to(dev)
        tot = 0.0
        for s0 in range(0, B, batch):
            idx = perm[s0:s0 + batch]
            xb, yb = Xs[idx].contiguous(), Y[idx].contiguous()
            nb = len(idx)
            st = smat.smat_mlp_loss_grad(p.data_ptr(), xb.data_ptr(), yb.data_ptr(), nb, g.data_ptr(),
                                         loss.data_ptr(), work.data_ptr(), torch.cuda.current_stream().cuda_stream)
            assert st == 0
            step += 1
            st = smat.smat_mlp_adam(p.data_ptr(), g.data_ptr(), m1.data_ptr(), v1.data_ptr(), p.numel(), step, lr,
                                    0.9, 0.999, 1e-8, torch.cuda.current_stream().cuda_stream)
            assert st == 0
            tot += float(loss.item()) * nb
        hist.append(tot / B)
        if log and (ep % 50 == 0 or ep == epochs - 1):
            log(f"epoch {ep} loss {hist[-1]:.4f}")
    return p.cpu().numpy(), mean.astype(np.float32), std.astype(np.float32), hist


def predict(params, mean, std, recs, forward=None):
    """Softmax probabilities over the admissible variants (GPU kernel by default)."""
    X, T, adm = arrays(recs)
    Xs = ((X - mean) / std).astype(np.float32)
    if forward is None:
        import torch

        import paper_1210_2536_gb300 as smat
        dev = torch.device("cuda:0")
        xp = torch.tensor(Xs, device=dev)
        pp = torch.tensor(params, device=dev)
        z = torch.empty((len(recs), NV), dtype=torch.float32, device=dev)
        assert smat.smat_mlp_forward(pp.data_ptr(), xp.data_ptr(), len(recs), z.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream) == 0
        Z = z.cpu().numpy().astype(np.float64)
    else:
        Z = forward(params, Xs)
    Z = np.where(adm, Z, -np.inf)
    Z = Z - Z.max(axis=1, keepdims=True)
    P = np.exp(Z)
    return P / P.sum(axis=1, keepdims=True)


def evaluate(P, recs, conf=0.6, topk=3):
    """Accuracy (pick within 2 % of the best), regret t_pick / t_best - 1, and
    the same for the paper's rules and fixed choices (the ablation)."""
    X, T, adm = arrays(recs)
    best = T.min(axis=1)
    csr = T[:, 0]

    def score(pick, trials=None):
        tp = T[np.arange(len(recs)), pick]
        reg = tp / best - 1.0
        d = {"accuracy": float(np.mean(tp <= TIE * best)), "regret_mean": float(np.mean(reg)),
             "regret_p90": float(np.percentile(reg, 90)), "regret_max": float(np.max(reg)),
             "speedup_vs_csr_scalar_geomean": float(np.exp(np.mean(np.log(csr / tp))))}
        if trials is not None:
            d["trials_mean"] = float(np.mean(trials))
        return d

    mlp = P.argmax(axis=1)
    fb = mlp.copy()
    trials = np.zeros(len(recs))
    for i in range(len(recs)):
        if P[i, mlp[i]] < conf:
            cand = [v for v in np.argsort(-P[i])[:topk] if np.isfinite(T[i, v])]
            fb[i] = cand[int(np.argmin(T[i, cand]))]
            trials[i] = len(cand)
    rules = np.array([r["rules"] for r in recs])
    out = {"n": len(recs), "mlp": score(mlp), "mlp_with_fallback": score(fb, trials),
           "fallback_rate": float(np.mean(trials > 0)), "rules": score(rules),
           "always_csr_scalar": score(np.zeros(len(recs), dtype=int))}
    for name, v in (("always_csr_merge", 4), ("always_coo", 7)):
        out[name] = score(np.full(len(recs), v))
    out["exhaustive"] = score(T.argmin(axis=1))
    out["best_variant_counts"] = {str(v): int(np.sum(T.argmin(axis=1) == v)) for v in range(NV)}
    return out


# ---------------------------------------------------------------------------
# Parameter influence (Sec. 4 and its figures on Ndiags and max_RD, ER_DIA
# and ER_ELL, NTdiags_ratio and var_RD): the matrices of the labelled set
# binned by one parameter at a time, and in each bin how many of those that
# admit the format the parameter steers are GOOD for it, i.e. that format's
# time lies within 2 % of the fastest of the eight classes (the rest are
# BAD).  The paper reads its thresholds off such counts; the same counts on
# this GPU show where those thresholds still hold.  Each bin also counts the
# matrices of at least LARGE_NNZ stored entries apart: below that a product
# takes a few microseconds and most classes tie within the 2 %.
# ---------------------------------------------------------------------------

LARGE_NNZ = 1_000_000

INF = float("inf")
# (parameter, variant it steers, bin edges, the paper's reading)
INFLUENCE = [
    ("ndiags", 6, [1, 25, 100, 500, INF], "nearly every matrix with Ndiags < 25 is good for DIA, few above 500"),
    ("er_dia", 6, [0.0, 0.2, 0.4, 0.6, 0.8, INF], "DIA wins when ER_DIA > 60 %"),
    ("ntdiags_ratio", 6, [0.0, 0.2, 0.4, 0.6, 0.8, INF], "DIA benefits when NTdiags_ratio > 40 %"),
    ("max_rd", 5, [0, 5, 10, 50, INF], "ELL is most often best when max_RD < 5"),
    ("er_ell", 5, [0.0, 0.5, 0.7, 0.9, INF], "ELL may benefit only when ER_ELL > 90 %"),
    ("var_rd", 5, [0.0, 0.5, 2.0, 10.0, INF], "ELL benefits only when var_RD < 0.5"),
    ("r", 7, [-INF, 1.0, 4.0, INF], "COO for small-world matrices, R in [1, 4)"),
]
VARIANT_SHORT = ["csr_scalar", "csr_vec4", "csr_vec8", "csr_vec32", "csr_merge", "ell", "dia", "coo"]


def parameter_value(rec, name):
    """The raw feature `name` of a dataset record (NTdiags_ratio = true
    diagonals / Ndiags, 0 without diagonals; R is None where undefined)."""
    raw = rec["raw"]
    if name == "ntdiags_ratio":
        return raw["ntdiags"] / raw["ndiags"] if raw["ndiags"] > 0 else 0.0
    if name == "r":
        return raw["r"] if raw["r_valid"] else None
    return raw[name]


def is_good(rec, v, tie=TIE):
    """Variant v admissible and within `tie` of the fastest admissible class."""
    t = rec["timings_ms"]
    if not (rec["admissible"] >> v) & 1 or not t[v] > 0:
        return None
    best = min(x for j, x in enumerate(t) if (rec["admissible"] >> j) & 1 and x > 0)
    return t[v] <= tie * best


def influence(recs):
    out = {"matrices": len(recs), "tie": round(TIE - 1.0, 4), "large_nnz": LARGE_NNZ, "parameters": []}
    for name, v, edges, reading in INFLUENCE:
        bins = [{"lo": None if edges[k] == -INF else edges[k], "hi": None if edges[k + 1] == INF else edges[k + 1],
                 "n": 0, "good": 0, "n_large": 0, "good_large": 0} for k in range(len(edges) - 1)]
        undefined = {"n": 0, "good": 0, "n_large": 0, "good_large": 0}
        for r in recs:
            g = is_good(r, v)
            if g is None:
                continue
            x = parameter_value(r, name)
            if x is None:
                slot = undefined
            else:
                slot = next(b for k, b in enumerate(bins) if edges[k] <= x < edges[k + 1])
            slot["n"] += 1
            slot["good"] += int(g)
            if r["nnz"] >= LARGE_NNZ:
                slot["n_large"] += 1
                slot["good_large"] += int(g)
        for b in bins + [undefined]:
            b["good_share"] = round(b["good"] / b["n"], 4) if b["n"] else None
            b["good_share_large"] = round(b["good_large"] / b["n_large"], 4) if b["n_large"] else None
        entry = {"parameter": name, "format": VARIANT_SHORT[v], "paper": reading, "bins": bins}
        if name == "r":
            entry["undefined"] = undefined
        out["parameters"].append(entry)
    return out


def influence_table(rep):
    """The report as markdown: one row per parameter bin."""
    lines = ["| parameter | format | bin | admissible | good | good share | admissible, nnz ≥ 10⁶ | good | good share |",
             "|---|---|---|---|---|---|---|---|---|"]
    for p in rep["parameters"]:
        rows = [(f"[{b['lo'] if b['lo'] is not None else '-inf'}, {b['hi'] if b['hi'] is not None else 'inf'})", b)
                for b in p["bins"]]
        if "undefined" in p:
            rows.append(("undefined", p["undefined"]))
        for label, b in rows:
            share = f"{100 * b['good_share']:.0f} %" if b["good_share"] is not None else "—"
            large = f"{100 * b['good_share_large']:.0f} %" if b["good_share_large"] is not None else "—"
            lines.append(f"| {p['parameter']} | {p['format']} | {label} | {b['n']} | {b['good']} | {share} | "
                         f"{b['n_large']} | {b['good_large']} | {large} |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("label")
    a.add_argument("--out", required=True)
    a.add_argument("--count", type=int, default=synth.DATASET_SIZE)
    a.add_argument("--start", type=int, default=0)
    a.add_argument("--reps", type=int, default=7)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--model", required=True)
    t.add_argument("--report", required=True)
    t.add_argument("--epochs", type=int, default=400)
    t.add_argument("--lr", type=float, default=3e-3)
    t.add_argument("--seed", type=int, default=0)
    f = sub.add_parser("influence")
    f.add_argument("--data", required=True)
    f.add_argument("--out", required=True)
    args = ap.parse_args()
    if args.cmd == "influence":     # bookkeeping over the labelled set only: no GPU, no build
        rep = influence(load(args.data))
        json.dump(rep, open(args.out, "w"), indent=1)
        print(influence_table(rep))
        return
    import __graft_entry__
    __graft_entry__.build()
    import paper_1210_2536_gb300 as smat
    if args.cmd == "label":
        label(args.out, args.count, args.start, args.reps)
        return
    recs = load(args.data)
    tr, he = split(recs)
    t0 = time.time()
    params, mean, std, hist = train(tr, epochs=args.epochs, lr=args.lr, seed=args.seed, log=print)
    train_s = time.time() - t0
    smat.write_model(args.model, params, mean, std)
    rep = {"train_size": len(tr), "heldout_size": len(he), "epochs": args.epochs, "lr": args.lr,
           "train_seconds": train_s, "loss_first": hist[0], "loss_last": hist[-1],
           "train": evaluate(predict(params, mean, std, tr), tr),
           "heldout": evaluate(predict(params, mean, std, he), he)}
    # the six primary structure classes alone, and each class on its own
    prim = [r for r in he if r["id"] < synth.DATASET_PRIMARY]
    rep["heldout_primary"] = evaluate(predict(params, mean, std, prim), prim)
    rep["heldout_by_kind"] = {}
    for kind in sorted({r["kind"] for r in he}):
        sub = [r for r in he if r["kind"] == kind]
        ev = evaluate(predict(params, mean, std, sub), sub)
        rep["heldout_by_kind"][kind] = {"n": ev["n"], "mlp": ev["mlp"], "mlp_with_fallback": ev["mlp_with_fallback"],
                                        "rules": ev["rules"]}
    json.dump(rep, open(args.report, "w"), indent=1)
    h = rep["heldout"]
    print(json.dumps({k: h[k] for k in ("mlp", "mlp_with_fallback", "rules", "always_csr_scalar", "fallback_rate")},
                     indent=1))


if __name__ == "__main__":
    main()
