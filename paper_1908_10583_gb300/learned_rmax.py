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
5. comparators: the best constant multiple of the rule (measured on training sources over
   the grid and the paper's r*, 2r*, ..., 7r*, Section 8 "Tuning r_max") and the balanced
   push of Section 4.2 (Alg. 3) with the calibrated costs;
   anchor: the network's output is moved so that its mean over the training sources is
   the chosen constant, and its per-source deviations are kept at the share (0, 1/4, 1/2
   or 1) with the least measured time on the training sources (0: the constant itself);
6. evaluate: held-out sources, batched, with the rule, the constant, the balanced push and
   the learned r_max: measured time per batch and modelled cost; optionally also on a
   second (larger) graph, whose per-unit costs the balanced push gets from a short
   calibration of its own.

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


FEATURES = ("edge_pushes", "pushes", "push_rounds", "walks", "walk_steps", "residual_nodes")


def measure(g, sources, params, mults=MULTS, batch=256):
    """Counters [S, len(mults), 6] (FEATURES: edge pushes, node pushes, push rounds, walks,
    moves, residual nodes) and per-run timings."""
    torch = _torch()
    import paper_1908_10583_gb300 as fora
    r_rule = g.resolve(params)[0]
    S = len(sources)
    cnt = np.zeros((S, len(mults), len(FEATURES)))
    runs = []
    ids = torch.empty((batch, params.k), dtype=torch.int32, device="cuda")
    vals = torch.empty((batch, params.k), dtype=torch.float64, device="cuda")
    for lo in range(0, S, batch):
        chunk = sources[lo:lo + batch]
        for j, mlt in enumerate(mults):
            _, _, st = g.ssppr_batch_rmax(chunk, np.full(len(chunk), r_rule * mlt), params,
                                         out_ids=ids[:len(chunk)], out_vals=vals[:len(chunk)])
            for i, s in enumerate(st):
                cnt[lo + i, j] = [getattr(s, f) for f in FEATURES]
            c = cnt[lo:lo + len(chunk), j].sum(0)
            runs.append({"mult": float(mlt), "n": len(chunk),
                         **{f: float(c[k]) for k, f in enumerate(FEATURES)},
                         "ms_push": st[0].ms_push,
                         "ms_walk": st[0].ms_residual + st[0].ms_walk})
    return cnt, runs, fora


PUSH_TERMS = ("edge_pushes", "pushes", "push_rounds")
WALK_TERMS = ("walks", "walk_steps", "residual_nodes")


def _nnls_fit(runs, terms, target):
    """Non-negative per-unit costs of `terms` plus a free-standing per-run constant (fixed
    work that no source's r_max changes), fitted to the measured ms; R^2 of the fit."""
    from scipy.optimize import nnls
    A = np.array([[r[t] for t in terms] + [1.0] for r in runs])
    y = np.array([r[target] for r in runs])
    scale = np.maximum(A.max(0), 1e-30)
    x, _ = nnls(A / scale, y)
    x = x / scale
    pred = A @ x
    r2 = 1.0 - float(((y - pred) ** 2).sum() / max(((y - y.mean()) ** 2).sum(), 1e-30))
    return dict(zip(terms, x[:-1])), float(x[-1]), r2


def calibrate(runs):
    """Per-unit costs (ms) from the measured phase times by non-negative least squares:
    push_ms ~ edge pushes, node pushes, push rounds (each round scans the source's
    residues) + constant; walk_ms ~ walks, moves, residual entries + constant."""
    push, push0, r2p = _nnls_fit(runs, PUSH_TERMS, "ms_push")
    walk, walk0, r2w = _nnls_fit(runs, WALK_TERMS, "ms_walk")
    return {"edge_push": push["edge_pushes"], "push": push["pushes"],
            "push_round": push["push_rounds"], "walk": walk["walks"], "move": walk["walk_steps"],
            "residual": walk["residual_nodes"], "push_fixed": push0, "walk_fixed": walk0,
            "r2_push": r2p, "r2_walk": r2w}


def cost(cnt, coef):
    """Modelled cost (ms) of counters [..., FEATURES] (the per-run constants left out)."""
    keys = ("edge_push", "push", "push_round", "walk", "move", "residual")
    return sum(coef.get(k, 0.0) * cnt[..., i] for i, k in enumerate(keys))


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


# Offsets of the output layer in the model's parameter vector
# (W1[64][16] | b1[64] | W2[64][64] | b2[64] | W3[64] | b3).
OFF_W3 = 64 * 16 + 64 + 64 * 64 + 64
OFF_B3 = OFF_W3 + 64


def anchored(params, pred, const_mult, lam):
    """Output-layer change that anchors the network at a measured constant: the new output
    is log2(const_mult) + lam * (y - mean y), y the current output and the mean over the
    training sources (clamped to +-3 as the query clamps it); W3 is scaled by lam (a power
    of two or 0: exact in BF16) and b3 moved accordingly.  lam = 0 is the constant itself."""
    p = np.array(params, dtype=np.float32, copy=True)
    mu = float(np.clip(pred, -3.0, 3.0).mean())
    p[OFF_W3:OFF_B3] *= np.float32(lam)
    p[OFF_B3] = np.float32(lam * float(params[OFF_B3]) + (np.log2(const_mult) - lam * mu))
    return p


def select_lambda(g, model, sources, features, params, const_mult, lams=(0.0, 0.25, 0.5, 1.0),
                  batch=256):
    """The lam of `anchored` with the least measured time on `sources` (training sources);
    the model is left at that choice.  -> (lam, {lam: ms})."""
    torch = _torch()
    base, norm = model.get()
    pred = model.predict(features)
    ids = torch.empty((batch, params.k), dtype=torch.int32, device="cuda")
    vals = torch.empty((batch, params.k), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    times = {}
    for lam in lams:
        model.set(anchored(base, pred, const_mult, lam), norm)
        ms = 0.0
        for lo in range(0, len(sources), batch):
            chunk = sources[lo:lo + batch]
            ms += _timed(lambda: g.ssppr_batch_learned(chunk, params, model, out_ids=ids[:len(chunk)],
                                                      out_vals=vals[:len(chunk)], stream=stream),
                         stream)[0]
        times[float(lam)] = ms
    best = min(times, key=times.get)
    model.set(anchored(base, pred, const_mult, best), norm)
    return best, times


def train(features, target, epochs=80, batch=256, lr=2e-3, seed=0):
    import paper_1908_10583_gb300 as fora
    m = fora.Model(seed)
    hist = m.train(features, target.astype(np.float32), epochs=epochs, batch=batch, lr=lr,
                   seed=seed + 1)
    return m, hist


PAPER_MULTS = np.arange(1.0, 8.0)  # r*, 2r*, ..., 7r* (Section 8, "Tuning r_max")


def balance_costs(coef, alpha=0.2, zero_hop=False):
    """Costs of the balanced push (Alg. 3) from calibrated per-unit costs: one edge push,
    one node push, and one walk with its expected (1 - alpha) / alpha moves (one more for
    a zero-hop walk's forced first move).  Alg. 3's rule has no per-round or per-entry
    term, so those calibrated costs are not part of it."""
    moves = (1.0 - alpha) / alpha + (1.0 if zero_hop else 0.0)
    return (coef["edge_push"], coef["push"], coef["walk"] + moves * coef["move"])


def _timed(fn, stream):
    torch = _torch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def best_constant(g, sources, params, mults, batch=256):
    """The constant multiple of the rule's r_max with the least measured time on `sources`
    (each candidate run once on every batch after one warm-up batch) -> (mult, {mult: ms})."""
    torch = _torch()
    r_rule = g.resolve(params)[0]
    ids = torch.empty((batch, params.k), dtype=torch.int32, device="cuda")
    vals = torch.empty((batch, params.k), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    times = {}
    for mlt in mults:
        ms = 0.0
        for lo in range(0, len(sources), batch):
            chunk = sources[lo:lo + batch]
            ms += _timed(lambda: g.ssppr_batch_rmax(chunk, np.full(len(chunk), r_rule * mlt), params,
                                                   out_ids=ids[:len(chunk)],
                                                   out_vals=vals[:len(chunk)], stream=stream),
                         stream)[0]
        times[float(mlt)] = ms
    best = min(times, key=times.get)
    return best, times


def evaluate(g, model, sources, params, coef, batch=256, const_mult=None, balance=None):
    """Rule, constant multiple, balanced push (Alg. 3) and learned r_max on held-out sources:
    measured ms per batch (CUDA events on the launching stream) and modelled cost.  Each
    batch runs every arm once after one warm-up of the first arm."""
    torch = _torch()
    ids = torch.empty((batch, params.k), dtype=torch.int32, device="cuda")
    vals = torch.empty((batch, params.k), dtype=torch.float64, device="cuda")
    r_rule = g.resolve(params)[0]
    arms = {"rule": lambda c, o: g.ssppr_batch(c, params, **o)}
    if const_mult is not None:
        arms["constant"] = lambda c, o: g.ssppr_batch_rmax(c, np.full(len(c), r_rule * const_mult),
                                                           params, **o)
    if balance is not None:
        arms["balanced"] = lambda c, o: g.ssppr_batch_balanced(c, params, balance, **o)
    if model is not None:
        arms["learned"] = lambda c, o: g.ssppr_batch_learned(c, params, model, **o)
    res = {name: {"ms": 0.0, "cost": 0.0, "rmax_over_rule_mean": 0.0} for name in arms}
    stream = torch.cuda.current_stream()
    for lo in range(0, len(sources), batch):
        chunk = sources[lo:lo + batch]
        o = {"out_ids": ids[:len(chunk)], "out_vals": vals[:len(chunk)], "stream": stream}
        if lo == 0:
            arms["rule"](chunk, o)
        for name, fn in arms.items():
            ms, (_, _, st) = _timed(lambda: fn(chunk, o), stream)
            res[name]["ms"] += ms
            c = np.array([[getattr(s, f) for f in FEATURES] for s in st])
            res[name]["cost"] += float(cost(c, coef).sum())
            res[name]["rmax_over_rule_mean"] += sum(s.rmax / r_rule for s in st)
    for name in arms:
        res[name]["queries_per_s"] = len(sources) / (res[name]["ms"] / 1e3)
        res[name]["rmax_over_rule_mean"] /= len(sources)
    for name in arms:
        if name != "rule":
            res[f"time_gain_{name}"] = 1.0 - res[name]["ms"] / res["rule"]["ms"]
    if "learned" in res:
        res["time_gain"] = res["time_gain_learned"]
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
    ap.add_argument("--const-sources", type=int, default=1024,
                    help="training sources on which the constant multipliers are timed")
    ap.add_argument("--large-scale", type=int, default=0,
                    help="also evaluate on R-MAT 2^scale (0: no second graph)")
    ap.add_argument("--large-deg", type=float, default=32)
    ap.add_argument("--large-seed", type=int, default=3)
    ap.add_argument("--large-eval", type=int, default=256)
    ap.add_argument("--large-batch", type=int, default=64)
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
    del col
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
    if args.model_out:
        os.makedirs(os.path.dirname(os.path.abspath(args.model_out)), exist_ok=True)
        model.save(args.model_out)
    # comparators: the best constant multiple (grid and the paper's r* .. 7r*), Alg. 3
    cands = sorted(set(MULTS.tolist()) | set(PAPER_MULTS.tolist()))
    const_mult, const_times = best_constant(g, tr[:args.const_sources], params, cands,
                                            batch=args.batch)
    # anchor the network at the measured constant; keep the measured share of its deviations
    lam, lam_times = select_lambda(g, model, tr[:args.const_sources], x, params, const_mult,
                                   batch=args.batch)
    if args.model_out:
        model.save(args.model_out)
    bal = balance_costs(coef)
    res = evaluate(g, model, ev, params, coef, batch=args.batch, const_mult=const_mult,
                   balance=bal)
    ycost = cost(cnt, coef)
    out = {"graph": {"scale": args.scale, "avg_deg": args.deg, "n": n, "m": int(rp[-1])},
           "train_sources": len(tr), "eval_sources": len(ev), "multipliers": MULTS.tolist(),
           "coef_ms": coef, "label_mean": float(y.mean()), "label_std": float(y.std()),
           "best_multiplier_cost_gain_train": float(1 - ycost.min(1).sum() / ycost[:, 3].sum()),
           "constant": {"chosen": const_mult, "ms_on_training_sources": const_times,
                        "sources": min(args.const_sources, len(tr))},
           "anchor": {"lambda": lam, "ms_on_training_sources": lam_times},
           "balance_costs_ms": {"edge_push": bal[0], "push": bal[1], "walk": bal[2]},
           "loss_first_last": [float(hist[0]), float(hist[-1])], "eval": res,
           "seconds": {"measure": t1 - t0, "train": t2 - t1, "eval": time.time() - t2}}
    print(json.dumps(out, indent=1), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    if args.large_scale:
        # the second graph: the same model and constant; Alg. 3 gets costs calibrated there
        g.close()
        rp2, col2 = inputs.rmat_csr(args.large_scale, args.large_deg, args.large_seed)
        n2 = len(rp2) - 1
        g2 = fora.Graph(rp2, col2)
        del col2
        ev2 = inputs.uniform_sources(n2, args.large_eval + args.large_batch, 778)
        cal, ev2 = ev2[:args.large_batch], ev2[args.large_batch:]
        _, runs2, _ = measure(g2, cal, params, mults=MULTS[[1, 3, 5]], batch=args.large_batch)
        coef2 = calibrate(runs2)
        bal2 = balance_costs(coef2)
        res2 = evaluate(g2, model, ev2, params, coef2, batch=args.large_batch,
                        const_mult=const_mult, balance=bal2)
        out["large"] = {"graph": {"scale": args.large_scale, "avg_deg": args.large_deg, "n": n2,
                                  "m": int(rp2[-1])},
                        "eval_sources": len(ev2), "calibration_sources": len(cal),
                        "coef_ms": coef2,
                        "balance_costs_ms": {"edge_push": bal2[0], "push": bal2[1],
                                             "walk": bal2[2]},
                        "eval": res2}
        print(json.dumps(out["large"], indent=1), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    return out


if __name__ == "__main__":
    main()
