"""Poisson load against the continuous-batching server (fora_server_*).

Queries arrive as a Poisson process of the given rate over resident R-MAT graphs;
each picks a graph, a uniform source, k in {50, 500} and eps in {0.5, 0.3}.  Reports
p50/p99 latency (submit to result) and queries/s.

    python -m paper_1908_10583_gb300.serve --graphs 18:16:4,22:16:5 --rate 300 --duration 20
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np


def run(graph_specs, rate, duration, lanes, max_batch, window_ms, budget, seed=1, warm=True):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import inputs
    import paper_1908_10583_gb300 as fora
    from paper_1908_10583_gb300 import build as fbuild
    fbuild.build()
    graphs = []
    for scale, deg, gseed in graph_specs:
        graphs.append(fora.Graph(*inputs.rmat_csr(scale, deg, gseed)))
    server = fora.Server(graphs, lanes_per_graph=lanes, max_batch=max_batch,
                         memory_budget_bytes=budget, batch_window_ms=window_ms)
    caps = [server.lane_capacity(i) for i in range(len(graphs) * lanes)]
    rng = np.random.default_rng(seed)
    n_req = int(rate * duration)
    gaps = rng.exponential(1.0 / rate, n_req)
    arrivals = np.cumsum(gaps)
    gsel = rng.integers(0, len(graphs), n_req)
    ks = rng.choice([50, 500], n_req)
    epss = rng.choice([0.5, 0.3], n_req)
    srcs = [int(rng.integers(0, graphs[g].n)) for g in gsel]
    tickets = [None] * n_req
    if warm:  # one query per (graph, eps) so the lanes' first-use costs are out of the way
        for gi in range(len(graphs)):
            for e in (0.5, 0.3):
                p = fora.Params.make(eps=e, k=500, seed=3)
                server.wait(server.submit(gi, 0, p), 500)
    done = threading.Event()
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        for i in range(n_req):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            p = fora.Params.make(eps=float(epss[i]), k=int(ks[i]), seed=3)
            tickets[i] = (server.submit(int(gsel[i]), srcs[i], p), int(ks[i]))
            ready.release()
        done.set()

    th = threading.Thread(target=submitter)
    th.start()
    lat, batch_sizes, ends, subs = [], [], [], []
    for i in range(n_req):
        ready.acquire()
        t, k = tickets[i]
        _, _, info = server.wait(t, k)
        lat.append(info.end_ms - info.submit_ms)
        batch_sizes.append(info.batch_size)
        ends.append(info.end_ms)
        subs.append(info.submit_ms)
    th.join()
    st = server.stats()
    server.close()
    lat = np.array(lat)
    span_s = (max(ends) - min(subs)) / 1e3
    return {"graphs": [{"scale": s, "avg_deg": d, "seed": g} for s, d, g in graph_specs],
            "offered_rate": rate, "requests": n_req, "duration_s": duration,
            "lanes_per_graph": lanes, "lane_slots": [c[1] for c in caps],
            "batch_window_ms": window_ms, "queries_per_s": n_req / span_s,
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "mean_batch": float(np.mean(batch_sizes)), "server": st}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--graphs", default="18:16:4,22:16:5",
                    help="comma-separated scale:avg_deg:seed")
    ap.add_argument("--rate", type=float, default=300.0)
    ap.add_argument("--duration", type=float, default=20.0)
    ap.add_argument("--lanes", type=int, default=2)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--window-ms", type=float, default=1.0)
    ap.add_argument("--budget-gb", type=float, default=0.0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    specs = [tuple(int(float(x)) if i != 1 else float(x) for i, x in enumerate(g.split(":")))
             for g in args.graphs.split(",")]
    res = run(specs, args.rate, args.duration, args.lanes, args.max_batch, args.window_ms,
              int(args.budget_gb * (1 << 30)))
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
