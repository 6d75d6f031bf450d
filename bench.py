#!/usr/bin/env python3
"""Throughput benchmark of the batched FORA SSPPR query on one GB300 (or N replicas).

Workload (default ``rmat20_deg16``): directed R-MAT graph, n = 2^20, average
out-degree 16 (0.57, 0.19, 0.19, 0.05), dangling nodes fixed with one uniform
edge; alpha = 0.2, eps = 0.5, delta = p_f = 1/n, r_max by the rule of Section
3.2, 256 uniform sources per launch, top-500 per source.  A step is one batched
query of 256 sources: push rounds, walk phase, estimate and top-k, all on the
device; the graph stays resident and each step draws new sources.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SSPPR queries/s and p99 latency at ε=0.5, batched+learned r_max vs plain FORA"
UNIT = "queries/s"
WALK_BYTES_PER_MOVE = 12      # row_ptr pair (8 B) + col entry (4 B)
WALK_BYTES_PER_WALK = 24      # count RMW (4+4 B) + acc RMW (8+8 B)
WALK_BYTES_PER_ENTRY = 24     # residual entry, offset, weight (8 B each)
PUSH_BYTES_PER_EDGE = 20      # col entry (4 B) + FP64 read-modify-write of r(u) (16 B)
PUSH_BYTES_PER_VERTEX = 44    # row pair, r(v) read and zero, reserve RMW, queue append


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fora", "reference"], default="fora")
    ap.add_argument("--workload", default="rmat20_deg16")
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--cpu-sources", type=int, default=None,
                    help="sources in each bounded CPU-oracle sample (default: one per oracle "
                         "thread)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stats", action="store_true", help="per-step counters to stderr")
    ap.add_argument("--tune", action="append", default=[],
                    help="launch-shape parameter key=value (fora_graph_tune)")
    ap.add_argument("--rmax", choices=["auto", "rule", "learned"], default="auto",
                    help="learned: per-source r_max from paper_1908_10583_gb300/models/"
                         "rmax_<workload>.npz (auto: when that file exists)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip fora_graph_autotune (launch shapes at their defaults / --tune)")
    ap.add_argument("--plain-sources", type=int, default=16,
                    help="single-source queries timed for the plain-FORA comparison")
    ap.add_argument("--no-index", action="store_true",
                    help="skip the FORA+ (walk index, Section 3.3) comparison")
    return ap.parse_args(argv)


def workload(args):
    import inputs
    w = dict(inputs.WORKLOADS[args.workload])
    if args.batch:
        w["n_sources"] = args.batch
    if args.k:
        w["k"] = args.k
    return w


class ClockSampler:
    """nvidia-smi clock and throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for name, val in zip(names, f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        finally:
            os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_values(kernel, wl):
    """'key: value' lines of a committed ncu summary (profiles/<kernel>_<wl>.txt), {} if
    there is none."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{wl}.txt")
    out = {}
    try:
        for line in open(path):
            if ":" in line and not line.startswith(" ") and not line.startswith("#"):
                key, val = line.split(":", 1)
                try:
                    out[key.strip()] = float(val.split()[0])
                except (ValueError, IndexError):
                    pass
    except OSError:
        return {}
    return out


def profiled_traffic(kernel, wl, launches_per_step=1, key="dram_bytes_per_launch"):
    """DRAM bytes per launch (or per step, with key) from a committed ncu summary, or None
    when there is none or it was taken with another split of the step into launches."""
    v = profile_values(kernel, wl)
    if key not in v or int(v.get("launches_per_step", 1)) != launches_per_step:
        return None
    return int(v[key])


def oracle_threads():
    """Host threads of both CPU-oracle legs (the reference arm and cpu_baseline): one
    oracle query per thread, at most 8 threads."""
    return max(1, min(os.cpu_count() or 1, 8))


def cpu_oracle_sample(rp, col, sources, w, eps, threads):
    """The oracle as it stands on the host cores: wall time of `sources` queries."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda s: oracle.ssppr(rp, col, int(s), eps=eps, k=w["k"]), sources))
    return time.perf_counter() - t0


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_sources(n, count, rank, step):
    """Sources of one step on one replica: a seeded uniform draw per (rank, step), so the
    replicas of an N-GPU run work on disjoint streams of new queries."""
    import inputs
    return inputs.uniform_sources(n, count, inputs.SOURCE_SEED + 1_000_003 * rank + 7919 * step)


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over the ranks of the process group (x itself at N = 1)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second, with `seconds` the slowest rank's time."""
    return units_per_rank * world / seconds


def run_reference(args):
    """CPU oracle arm: each step is a bounded sample of the workload on the host cores."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import inputs
    import oracle
    oracle.build()
    w = workload(args)
    rp, col = inputs.rmat_csr(w["scale"], w["avg_deg"], w["graph_seed"])
    n = len(rp) - 1
    threads = oracle_threads()
    per_step = args.cpu_sources or threads
    for i in range(args.warmup):
        src = inputs.uniform_sources(n, per_step, inputs.SOURCE_SEED + 7919 * (i + 1))
        cpu_oracle_sample(rp, col, src, w, args.eps, threads)
    times = []
    for i in range(args.steps):
        src = inputs.uniform_sources(n, per_step, inputs.SOURCE_SEED + 104729 * (i + 1))
        times.append(cpu_oracle_sample(rp, col, src, w, args.eps, threads))
    total = sum(times)
    value = per_step * args.steps / total
    sample = (f"{per_step} sources per step of the {args.workload} workload (top-{w['k']}, "
              f"eps={args.eps}, rule r_max), one oracle query per thread on {threads} host "
              f"threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "m": int(rp[-1]),
                       "sources_per_step": per_step, "k": w["k"], "eps": args.eps,
                       "alpha": 0.2, "delta": "1/n", "pf": "1/n", "rmax": "rule"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_fora(args):
    import numpy as np
    import torch

    import inputs
    world, rank, local = dist_setup()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1908_10583_gb300 import build as fbuild
    fbuild.build()
    import paper_1908_10583_gb300 as fora

    w = workload(args)
    B, k = w["n_sources"], w["k"]
    rp, col = inputs.rmat_csr(w["scale"], w["avg_deg"], w["graph_seed"])
    n = len(rp) - 1
    g = fora.Graph(rp, col)
    tuning = {}
    for kv in args.tune:
        key, val = kv.split("=")
        g.tune(key, int(val))
        tuning[key] = int(val)
    params = fora.Params.make(eps=args.eps, k=k, seed=inputs.WALK_SEED)
    stream = torch.cuda.current_stream()
    ids = torch.empty((B, k), dtype=torch.int32, device="cuda")
    vals = torch.empty((B, k), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    model_path = os.path.join(ROOT, "paper_1908_10583_gb300", "models",
                              f"rmax_{args.workload}.npz")
    mode = args.rmax
    if mode == "auto":
        mode = "learned" if os.path.exists(model_path) else "rule"
    model = fora.Model.load_file(model_path) if mode == "learned" else None

    def sources(step):
        return replica_sources(n, B, rank, step)

    def one_step(src, use_model):
        if use_model is not None:
            return g.ssppr_batch_learned(src, params, use_model, out_ids=ids, out_vals=vals,
                                         stream=stream)[2]
        return g.ssppr_batch(src, params, out_ids=ids, out_vals=vals, stream=stream)[2]

    def timed(use_model, nsteps, collect=None):
        out = []
        for step in range(nsteps):
            src = sources(step)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = one_step(src, use_model)
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
            if collect is not None:
                collect(step, st, out[-1])
        return out

    if not args.no_autotune and not args.tune:
        # autotuned frontier segments and walk-block shapes on a batch of the workload
        tuning.update(g.autotune(sources(-100), params, stream=stream))
    tuning["spread_hot"] = g.tuning("spread_hot")
    tuning["hot_nodes"] = g.tuning("hot_nodes")
    for i in range(args.warmup):
        one_step(sources(-1 - i), model)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    walk_ms, walk_bytes = [], []
    push_ms, push_bytes = [], []
    phase = {"ms_push": 0.0, "ms_residual": 0.0, "ms_walk": 0.0, "ms_topk": 0.0}
    counters = {"launches": 0, "walks": 0, "moves": 0}

    def part_bounds(nsrc):
        """The library's split of a batch into pipeline parts (at least 32 sources each):
        each part has its own launches and its own phase times in its stats."""
        parts = max(1, min(g.tuning("pipeline"), nsrc // 32))
        return [(nsrc * k // parts, nsrc * (k + 1) // parts) for k in range(parts)]

    def collect(step, st, ms):
        bounds = part_bounds(len(st))
        rounds = max(s.push_rounds for s in st)
        for lo, hi in bounds:
            r_k = max(s.push_rounds for s in st[lo:hi])
            # push: the seed, then (rounds + 1) passes of the loop body (spread, take,
            # advance); residuals 4, walks 1, estimate 1, top-k select 19
            counters["launches"] += 1 + 3 * (r_k + 1) + 4 + 1 + 1 + 19
        if model is not None:
            counters["launches"] += 3  # features, forward, r_max (whole batch)
        # kernel time of each phase, summed over the parts (parts overlap in time)
        for key in phase:
            phase[key] += sum(getattr(st[lo], key) for lo, _ in bounds)
        walk_ms.append(sum(st[lo].ms_walk for lo, _ in bounds))
        push_ms.append(sum(st[lo].ms_push for lo, _ in bounds))
        push_bytes.append(PUSH_BYTES_PER_EDGE * sum(s.edge_pushes for s in st) +
                          PUSH_BYTES_PER_VERTEX * sum(s.pushes for s in st))
        nw = sum(s.walks for s in st)
        ns = sum(s.walk_steps for s in st)
        nr = sum(s.residual_nodes for s in st)
        counters["walks"] += nw
        counters["moves"] += ns
        walk_bytes.append(WALK_BYTES_PER_MOVE * ns + WALK_BYTES_PER_WALK * nw +
                          WALK_BYTES_PER_ENTRY * nr)
        if args.stats:
            print(json.dumps({"step": step, "ms": ms, "rounds": rounds, "parts": len(bounds),
                              "pushes": sum(s.pushes for s in st),
                              "edge_pushes": sum(s.edge_pushes for s in st),
                              "residual_nodes": nr, "walks": nw, "moves": ns,
                              "rmax_mean": sum(s.rmax for s in st) / len(st),
                              **{k_: sum(getattr(st[lo], k_) for lo, _ in bounds)
                                 for k_ in phase}}), file=sys.stderr)

    step_ms = timed(model, args.steps, collect)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = whole_job_rate(B * args.steps, world, total_ms / 1e3)
    launches = counters["launches"]
    walks_total, steps_total = counters["walks"], counters["moves"]

    # the comparison of the metric: batched rule r_max, and plain FORA one query at a time
    comparison = {"rmax_mode": mode, f"batched_{mode}_qps": value}
    if mode == "learned":
        rule_ms = timed(None, args.steps)
        comparison["batched_rule_qps"] = B * args.steps / (sum(rule_ms) / 1e3)
        # the learned model's comparators, with the constant multiple and the per-unit costs
        # its training run chose on this workload (models/rmax_<workload>.json): a constant
        # multiple of the rule's r_max, and the balanced push of Section 4.2 (Alg. 3)
        report_path = os.path.splitext(model_path)[0] + ".json"
        if os.path.exists(report_path):
            rep = json.load(open(report_path))
            r_rule = g.resolve(params)[0]
            cmult = float(rep["constant"]["chosen"])
            bc = rep["balance_costs_ms"]
            costs = (bc["edge_push"], bc["push"], bc["walk"])
            arms = {
                "constant": lambda src: g.ssppr_batch_rmax(src, [r_rule * cmult] * len(src), params,
                                                           out_ids=ids, out_vals=vals,
                                                           stream=stream),
                "balanced": lambda src: g.ssppr_batch_balanced(src, params, costs, out_ids=ids,
                                                               out_vals=vals, stream=stream)}
            for name, fn in arms.items():
                fn(sources(-77))
                tot = 0.0
                for step in range(args.steps):
                    src = sources(step)
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn(src)
                    e1.record(stream)
                    e1.synchronize()
                    tot += e0.elapsed_time(e1)
                comparison[f"batched_{name}_qps"] = B * args.steps / (tot / 1e3)
            comparison["constant_multiple"] = cmult
            comparison["balance_costs_ms"] = bc
    # the same batches with zero-hop pruning (Section 4.1: alpha of every residue goes to the
    # estimate directly and each walk starts with a forced move), rule r_max
    zparams = fora.Params.from_buffer_copy(params)
    zparams.flags |= fora.FORA_ZERO_HOP
    g.ssppr_batch(sources(-78), zparams, out_ids=ids, out_vals=vals, stream=stream)
    ztot = 0.0
    for step in range(args.steps):
        src = sources(step)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.ssppr_batch(src, zparams, out_ids=ids, out_vals=vals, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ztot += e0.elapsed_time(e1)
    comparison["batched_zero_hop_rule_qps"] = B * args.steps / (ztot / 1e3)
    if args.plain_sources > 0:
        # plain FORA: one query at a time through fora_ssppr (rule r_max, host results),
        # each query's latency on the host clock around the synchronous call
        plain_src = inputs.uniform_sources(n, args.plain_sources, inputs.SOURCE_SEED + 31337)
        g.ssppr(int(plain_src[0]), params)  # warm the single-source workspace
        torch.cuda.synchronize()
        plain_ms = []
        t0 = time.perf_counter()
        for s_ in plain_src:
            t1 = time.perf_counter()
            g.ssppr(int(s_), params)
            plain_ms.append(1e3 * (time.perf_counter() - t1))
        comparison["plain_fora_qps"] = len(plain_src) / (time.perf_counter() - t0)
        lp = sorted(plain_ms)
        comparison["plain_fora_latency_ms"] = {
            "p50": lp[len(lp) // 2], "p99": lp[min(len(lp) - 1, int(0.99 * len(lp)))],
            "queries": len(lp)}
    if not args.no_index:
        # FORA+: the walk phase served from a walk index built for the rule's r_max
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.build_index(params, stream=stream)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        iparams = fora.Params.from_buffer_copy(params)
        iparams.flags |= fora.FORA_USE_INDEX
        g.ssppr_batch(sources(-50), iparams, out_ids=ids, out_vals=vals, stream=stream)
        idx_ms = []
        for step in range(args.steps):
            src = sources(step)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.ssppr_batch(src, iparams, out_ids=ids, out_vals=vals, stream=stream)
            e1.record(stream)
            e1.synchronize()
            idx_ms.append(e0.elapsed_time(e1))
        comparison["fora_plus_qps"] = B * args.steps / (sum(idx_ms) / 1e3)
        comparison["fora_plus_index"] = {"walks_stored": g.index_info()[2],
                                         "bytes": g.index_info()[2] * 4 + (n + 1) * 8,
                                         "build_s": build_s, "rmax": "rule"}
        g.drop_index()

    # end to end through the public API: host sources in, host results out
    h_ids = torch.empty((B, k), dtype=torch.int32, pin_memory=True).numpy()
    h_vals = torch.empty((B, k), dtype=torch.float64, pin_memory=True).numpy()
    e2e_s = 0.0
    for step in range(args.steps):  # the timed steps' sources, L2 flushed before each
        src = sources(step)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if model is not None:
            g.ssppr_batch_learned(src, params, model, stream=stream)
        else:
            g.ssppr_batch_host(src, params, h_ids, h_vals, stream=stream)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e = {"value": whole_job_rate(B * args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": B * (4 + 8),
           "d2h_bytes_per_step": B * k * (4 + 8)}

    peak, peak_kind = measured_peak_hbm()
    # per launch of the walk kernel (one per pipeline part of a step): the launches'
    # algorithmic bytes over their summed CUDA-event durations
    launches_per_step = len(part_bounds(B))
    bytes_per_launch = sum(walk_bytes) / (len(walk_bytes) * launches_per_step)
    ms_per_launch = sum(walk_ms) / (len(walk_ms) * launches_per_step)
    achieved = bytes_per_launch / (ms_per_launch / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_walks", "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic("k_walks", args.workload, launches_per_step),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "launches_per_step": launches_per_step}
    # the walk kernel is bound by issue and latency rather than by DRAM: its issue-slot and
    # L2 fractions from the committed ncu section capture of the same kernel (64 sources)
    wp = profile_values("k_walks", args.workload)
    if "issue_active_frac" in wp:
        roofline["issue_frac"] = wp["issue_active_frac"]
        roofline["l2_frac"] = wp.get("lts_throughput_frac")
        roofline["issue_l2_source"] = "ncu section capture, profiles/k_walks_" + args.workload + ".txt"
    # the push phase (all its rounds: spread, take, advance) against the same peak
    achieved_push = (sum(push_bytes) / len(push_bytes)) / (statistics.mean(push_ms) / 1e3) / 1e9
    spread_kernel = ("k_push_spread_hot" if tuning.get("spread_hot") and tuning.get("hot_nodes")
                     else "k_push_spread")
    roofline_push = {"bound": "hbm", "kernels": spread_kernel + "+k_push_take+k_push_advance",
                     "achieved": achieved_push, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": achieved_push / peak,
                     "traffic": profiled_traffic("push", args.workload, 1, "dram_bytes_per_step"),
                     "traffic_unit": "bytes per step (all push launches)",
                     "algorithmic_bytes_per_step": sum(push_bytes) / len(push_bytes)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = oracle_threads()
        nsamp = args.cpu_sources or threads
        src = inputs.uniform_sources(n, nsamp, inputs.SOURCE_SEED + 424242)
        secs = cpu_oracle_sample(rp, col, src, w, args.eps, threads)
        cpu = {"value": nsamp / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{nsamp} sources of the {args.workload} workload "
                         f"(top-{k}, eps={args.eps}, rule r_max), one oracle query per "
                         f"thread on {threads} host threads"}

    lat = sorted(step_ms)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "m": int(rp[-1]),
                       "avg_out_degree": w["avg_deg"], "sources_per_launch": B, "k": k,
                       "eps": args.eps, "alpha": 0.2, "delta": "1/n", "pf": "1/n",
                       "rmax": mode, "parallelism": f"replicas{world}",
                       "l2": "512 MiB buffer written between timed steps",
                       "tuning": tuning},
            "latency_ms": {"p50": lat[len(lat) // 2],
                           "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "note": "per query of the batched path: every query of a batch "
                                   "completes with its batch; plain FORA's per-query "
                                   "latency is comparison.plain_fora_latency_ms"},
            "phase_ms_per_step": {k_: v / args.steps for k_, v in phase.items()},
            "walks_per_step": walks_total / args.steps,
            "walk_moves_per_step": steps_total / args.steps,
            "gpu_launches": launches,
            "comparison": comparison,
            "roofline": roofline,
            "roofline_push": roofline_push,
            "e2e": e2e,
            "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fora(args)


if __name__ == "__main__":
    main()
