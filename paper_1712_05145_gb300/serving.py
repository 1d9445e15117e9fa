"""Serving stream of RVE solves: Poisson arrivals, mixed grids and orders, p50/p99 latency.

Requests draw a grid from {32, 48, 64, 96, 128}^3 plus 32 x 64 x 128, order 0 or 1 with
probability 1/2, and a random-sphere microstructure (volume fraction 0.3, radii 4-10 voxels of a
128 grid) whose inclusion/matrix stiffness contrast is log-uniform in [2, 1000] (nu = 0.3).
Geometries come from a seeded pool of a few per grid (the contrast is drawn per request).
Arrivals are Poisson at a rate of 0.8 x the capacity measured on a back-to-back batch of the
first --capacity-requests requests (or --rate).  The server (FP32 fields, FP64 reductions and
refinement) admits requests by free device memory, batches order-0 requests of one grid into one
handle (--max-batch) and keeps handles resident; the comparison is the plain FP64 form, one
request after the other, each in its own handle.

    python -m paper_1712_05145_gb300.serving --requests 2000
"""
import argparse
import json
import math
import random
import time


def build_pool(per_grid, seed):
    from paper_1712_05145_gb300 import synthetic
    grids = [(32, 32, 32), (48, 48, 48), (64, 64, 64), (96, 96, 96), (128, 128, 128), (32, 64, 128)]
    pool = {}
    for gi, g in enumerate(grids):
        pool[g] = [synthetic.random_spheres(g, seed=seed + 97 * gi + k) for k in range(per_grid)]
    return grids, pool


def make_requests(n, grids, pool, seed):
    from paper_1712_05145_gb300 import synthetic
    rng = random.Random(seed)
    reqs = []
    for _ in range(n):
        g = grids[rng.randrange(len(grids))]
        geo = pool[g][rng.randrange(len(pool[g]))]
        contrast = math.exp(rng.uniform(math.log(2.0), math.log(1000.0)))
        lame = [synthetic.lame_from_young(1.0, 0.3), synthetic.lame_from_young(contrast, 0.3)]
        lam0, mu0 = synthetic.midpoint_reference(lame)
        ms = synthetic.Microstructure(geo.phase, __import__("numpy").array(lame), lam0, mu0, "serving",
                                      {"contrast": contrast})
        reqs.append((ms, rng.randrange(2)))
    return reqs


def run_stream(reqs, rate, max_active, max_batch, tol, seed, with_counters=False):
    from paper_1712_05145_gb300 import hom
    rng = random.Random(seed + 1)
    s = hom.hom_server_create(0, max_active, max_batch)
    t0 = time.perf_counter()
    t_next = 0.0
    ids = []
    for ms, order in reqs:
        t_next += rng.expovariate(rate) if rate > 0 else 0.0
        delay = t0 + t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        ids.append(hom.hom_server_submit(s, ms, order, tol))
    res = [hom.hom_server_wait(s, i) for i in ids]
    wall = time.perf_counter() - t0
    counters = hom.hom_server_counters(s)
    hom.hom_server_destroy(s)
    return (res, wall, counters) if with_counters else (res, wall)


def serve_benchmark(n_requests, max_active=6, max_batch=8, capacity_requests=200, baseline_requests=60, tol=1e-6,
                    seed=1715, pool_per_grid=3, rate=0.0):
    """Capacity on a back-to-back batch of the first capacity_requests requests, then the Poisson
    stream of n_requests at 0.8 x that capacity (or `rate`), then the plain FP64 form, one solve
    per handle after the other, on the first baseline_requests requests.  Returns one dict."""
    import numpy as np
    from paper_1712_05145_gb300 import hom
    grids, pool = build_pool(pool_per_grid, seed)
    reqs = make_requests(n_requests, grids, pool, seed)
    cap_n = min(capacity_requests, len(reqs))
    res, wall = run_stream(reqs[:cap_n], 0.0, max_active, max_batch, tol, seed)
    capacity = cap_n / wall
    rate = rate if rate > 0 else 0.8 * capacity
    res, wall, counters = run_stream(reqs, rate, max_active, max_batch, tol, seed, with_counters=True)
    lat = np.array([r["latency_ms"] for r in res])
    ok = sum(1 for r in res if r["status"] == 0)
    failed = [{"grid": list(reqs[i][0].grid), "order": reqs[i][1], "contrast": reqs[i][0].meta["contrast"],
               "status": res[i]["status"], "iterations": res[i]["iterations"],
               "message": res[i]["message"]}
              for i in range(len(res)) if res[i]["status"] != 0]
    # plain FP64, one solve after the other, on the first baseline requests
    nb = min(baseline_requests, len(reqs))
    t0 = time.perf_counter()
    for ms, order in reqs[:nb]:
        H = hom.Homogenization(ms, precision=hom.HOM_FP64, scheme=hom.HOM_CG)
        H.solve(0, tol)
        H.effective(0)
        if order:
            H.solve(1, tol)
            H.effective(1)
        H.close()
    fp64_s = time.perf_counter() - t0
    return {"metric": "solves/s + p50/p99 at 1e-6 resid (serving stream)", "requests": len(reqs), "ok": ok,
            "rate_per_s": rate, "capacity_per_s": capacity, "max_active": max_active, "max_batch": max_batch,
            "solves_per_s": len(reqs) / wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_run_ms": float(np.mean([r["run_ms"] for r in res])),
            "server_counters": counters,
            "fp64_sequential": {"requests": nb, "seconds": fp64_s, "solves_per_s": nb / fp64_s},
            "served_over_fp64_sequential": (len(reqs) / wall) / (nb / fp64_s), "failed": failed[:20]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals per second (0: 0.8 x measured capacity)")
    ap.add_argument("--max-active", type=int, default=6)
    ap.add_argument("--max-batch", type=int, default=8, help="order-0 requests of one grid per batched handle")
    ap.add_argument("--capacity-requests", type=int, default=200)
    ap.add_argument("--pool", type=int, default=3)
    ap.add_argument("--baseline-requests", type=int, default=60)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--seed", type=int, default=1715)
    args = ap.parse_args()
    from paper_1712_05145_gb300 import build

    build.build()
    out = serve_benchmark(args.requests, args.max_active, args.max_batch, args.capacity_requests,
                          args.baseline_requests, args.tol, args.seed, args.pool, args.rate)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
