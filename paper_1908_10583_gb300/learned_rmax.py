"""Training and evaluation of the learned r_max (all GPU work through the C ABI).

1. measure: every training source runs the batched query at 8 log-spaced r_max
   values around the rule of Section 3.2 (multipliers 2^-1.5 ... 2^2, the rule itself
   included); each run
   yields per-source counters (edge pushes, node pushes, walks, walk moves) and the
   batch's measured phase times;
2. calibrate: per-unit costs from the measured times by non-negative least squares,
   push_ms ~ a_e edge_pushes + a_p pushes and walk_ms ~ b_w walks + b_m moves;
3. label: each source's cost at the 8 multipliers, and the log2 multiplier that
   minimises it (parabolic refinement around the best grid point);
4. train: the 16-64-64-1 BF16 network on (features, label) with the device Adam;
5. evaluate: held-out sources, batched, with the rule and with the learned r_max:
   measured step time and modelled cost.

    python -m paper_1908_10583_gb300.learned_rmax --scale 20 --deg 16 --train 10000 \\
        --eval 2000 --model-out paper_1908_10583_gb300/models/rmax_rmat20_deg16.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

MULTS = 2.0 ** ((np.arange(8) - 3) / 2.0)  # index 3 is the rule's r_max


def _torch():
    import torch
    return torch


def measure(g, sources, params, mults=MULTS, batch=256):
    """Counters [S, len(mults), 4] (edge pushes, pushes, walks, moves) and per-run timings."""
    torch = _torch()
    import paper_1908_10583_gb300 as fora
    r_rule = g.resolve(params)[0]
    S = len(sources)
    cnt = np.zeros((S, len(mults), 4))
    runs = []
    ids = torch.empty((batch, params.k), dtype=torch.int32, device="cuda")
    vals = torch.empty((batch, params.k), dtype=torch.float64, device="cuda")
    for lo in range(0, S, batch):
        chunk = sources[lo:lo + batch]
        for j, mlt in enumerate(mults):
            _, _, st = g.ssppr_batch_rmax(chunk, np.full(len(chunk), r_rule * mlt), params,
                                         out_ids=ids[:len(chunk)], out_vals=vals[:len(chunk)])
            for i, s in enumerate(st):
                cnt[lo + i, j] = (s.edge_pushes, s.pushes, s.walks, s.walk_steps)
            c = cnt[lo:lo + len(chunk), j].sum(0)
            runs.append({"mult": float(mlt), "n": len(chunk), "edge_pushes": c[0], "pushes": c[1],
                         "walks": c[2], "moves": c[3], "ms_push": st[0].ms_push,
                         "ms_walk": st[0].ms_residual + st[0].ms_walk})
    return cnt, runs, fora


def calibrate(runs):
    """Per-unit costs (ms) from the measured phase times: non-negative least squares."""
    from scipy.optimize import nnls
    A = np.array([[r["edge_pushes"], r["pushes"]] for r in runs])
    a, _ = nnls(A / A.max(0), np.array([r["ms_push"] for r in runs]))
    a = a / A.max(0)
    B = np.array([[r["walks"], r["moves"]] for r in runs])
    b, _ = nnls(B / B.max(0), np.array([r["ms_walk"] for r in runs]))
    b = b / B.max(0)
    return {"edge_push": a[0], "push": a[1], "walk": b[0], "move": b[1]}


def cost(cnt, coef):
    return (coef["edge_push"] * cnt[..., 0] + coef["push"] * cnt[..., 1]
            + coef["walk"] * cnt[..., 2] + coef["move"] * cnt[..., 3])


def labels(costs, mults=MULTS):
    """log2 of the cost-minimising multiplier per source (parabola through the best point
    and its neighbours on the log2 grid)."""
    lg = np.log2(mults)
    best = costs.argmin(1)
    out = lg[best].astype(np.float64)
    for i, j in enumerate(best):
        if 0 < j < len(mults) - 1:
            y0, y1, y2 = costs[i, j - 1], costs[i, j], costs[i, j + 1]
            den = y0 - 2 * y1 + y2
            if den > 0:
                out[i] += 0.5 * (lg[1] - lg[0]) * (y0 - y2) / den
    return np.clip(out, lg[0], lg[-1])


def train(features, target, epochs=80, batch=256, lr=2e-3, seed=0):
    import paper_1908_10583_gb300 as fora
    m = fora.Model(seed)
    hist = m.train(features, target.astype(np.float32), epochs=epochs, batch=batch, lr=lr,
                   seed=seed + 1)
    return m, hist


def evaluate(g, model, sources, params, coef, batch=256):
    """Rule vs learned on held-out sources: measured ms per batch and modelled cost."""
    torch = _torch()
    ids = torch.empty((batch, params.k), dtype=torch.int32, device="cuda")
    vals = torch.empty((batch, params.k), dtype=torch.float64, device="cuda")
    res = {"rule": {"ms": 0.0, "cost": 0.0}, "learned": {"ms": 0.0, "cost": 0.0}}
    stream = torch.cuda.current_stream()
    for lo in range(0, len(sources), batch):
        chunk = sources[lo:lo + batch]
        for name in ("rule", "learned"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if name == "rule":
                _, _, st = g.ssppr_batch(chunk, params, out_ids=ids[:len(chunk)],
                                         out_vals=vals[:len(chunk)], stream=stream)
            else:
                _, _, st = g.ssppr_batch_learned(chunk, params, model, out_ids=ids[:len(chunk)],
                                                 out_vals=vals[:len(chunk)], stream=stream)
            e1.record(stream)
            e1.synchronize()
            res[name]["ms"] += e0.elapsed_time(e1)
            c = np.array([[s.edge_pushes, s.pushes, s.walks, s.walk_steps] for s in st])
            res[name]["cost"] += float(cost(c, coef).sum())
    for name in res:
        res[name]["queries_per_s"] = len(sources) / (res[name]["ms"] / 1e3)
    res["time_gain"] = 1.0 - res["learned"]["ms"] / res["rule"]["ms"]
    res["cost_gain"] = 1.0 - res["learned"]["cost"] / res["rule"]["cost"]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--deg", type=float, default=16)
    ap.add_argument("--graph-seed", type=int, default=2)
    ap.add_argument("--train", type=int, default=10000)
    ap.add_argument("--eval", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--k", type=int, default=500)
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--epochs", type=int, default=80)
    ap.add_argument("--model-out", default=None)
    ap.add_argument("--out", default=None, help="results JSON")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import inputs
    import paper_1908_10583_gb300 as fora
    from paper_1908_10583_gb300 import build as fbuild
    fbuild.build()
    rp, col = inputs.rmat_csr(args.scale, args.deg, args.graph_seed)
    n = len(rp) - 1
    g = fora.Graph(rp, col)
    params = fora.Params.make(eps=args.eps, k=args.k, seed=inputs.WALK_SEED)
    pool = inputs.uniform_sources(n, args.train + args.eval, 777)
    tr, ev = pool[:args.train], pool[args.train:]
    t0 = time.time()
    cnt, runs, _ = measure(g, tr, params, batch=args.batch)
    coef = calibrate(runs)
    y = labels(cost(cnt, coef))
    x = np.concatenate([g.features(tr[i:i + 4096], params) for i in range(0, len(tr), 4096)])
    t1 = time.time()
    model, hist = train(x, y, epochs=args.epochs, batch=256)
    t2 = time.time()
    res = evaluate(g, model, ev, params, coef, batch=args.batch)
    ycost = cost(cnt, coef)
    out = {"graph": {"scale": args.scale, "avg_deg": args.deg, "n": n, "m": int(rp[-1])},
           "train_sources": len(tr), "eval_sources": len(ev), "multipliers": MULTS.tolist(),
           "coef_ms": coef, "label_mean": float(y.mean()), "label_std": float(y.std()),
           "best_multiplier_cost_gain_train": float(1 - ycost.min(1).sum() / ycost[:, 3].sum()),
           "loss_first_last": [float(hist[0]), float(hist[-1])], "eval": res,
           "seconds": {"measure": t1 - t0, "train": t2 - t1, "eval": time.time() - t2}}
    print(json.dumps(out, indent=1))
    if args.model_out:
        os.makedirs(os.path.dirname(os.path.abspath(args.model_out)), exist_ok=True)
        model.save(args.model_out)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    return out


if __name__ == "__main__":
    main()
