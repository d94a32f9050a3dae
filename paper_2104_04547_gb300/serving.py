"""Serving benchmark: Poisson arrivals of synthetic poses into the continuous-batching server.

    python -m paper_2104_04547_gb300.serving [--mix bf16,fp8] [--loads 0.25 0.5 0.9] [--requests 20000]
    python -m paper_2104_04547_gb300.serving --pool-groups 10000 --jobs 16 --requests 1000000 --loads 0.9

Poses are drawn at random from a pool of docked-pose stand-ins with uneven
sizes (ligands log-normal around 32 heavy atoms, pockets 150-1000 atoms,
--pool-rot rigid rotations per ligand; 10000 ligands x 10 rotations is the
100k-pose uneven-batching pool).  Each request is scored in one of the --mix
dtypes (requests cycle through them; the server runs slots of each).  First
the peak rate is measured with requests queued all at once; then, for each
offered load (a fraction of that peak), requests arrive as a Poisson process
and the per-pose latency (submission to completion, measured by the server)
is reported as p50 / p99 / p99.9 with the achieved poses/s, together with how
late the load generator itself submitted (a stall there arrives as a burst).
One JSON line per measurement.
"""

from __future__ import annotations

import argparse
import gc
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _collect(server, tickets):
    lat = np.empty(len(tickets))
    aff = np.empty(len(tickets), dtype=np.float32)
    for i, t in enumerate(tickets):
        r = server.poll(t)
        while r is None:
            time.sleep(0.0002)
            r = server.poll(t)
        aff[i], lat[i] = r
    return aff, lat


def _pct(lat):
    return {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
            "p99.9": 1e3 * float(np.percentile(lat, 99.9)), "max": 1e3 * float(lat.max())}


def run(args):
    import torch

    from paper_2104_04547_gb300 import build
    build.build()
    from paper_2104_04547_gb300 import fusion as F
    from synth import configs, poses, weights

    mix = args.mix.split(",")
    pool = poses.make_uneven_pool(args.pool_groups, args.pool_rot, jobs=args.jobs)
    torch.cuda.set_device(0)
    desc = configs.model("fusion-48grid-c64", dtype=mix[0])
    W = weights.init_weights(desc, 0)
    blob = weights.to_blob(desc, W)
    srv = F.Server(desc, blob, max_batch=args.max_batch, slots=args.slots, batch_window_us=args.window_us,
                   hbm_budget_bytes=int(args.budget_gb * (1 << 30)), queue_capacity=1 << 22, max_atoms=1200,
                   dtypes=tuple(mix[1:]))
    st = srv.stats()
    base = {"mix": mix, "model": "fusion-48grid-c64", "pool": f"{len(pool)} uneven poses "
            f"({args.pool_groups} ligands x {args.pool_rot} rigid poses), drawn at random",
            "slots": st["slots_by_dtype"], "slot_gb": round(st["slot_bytes"] / 2 ** 30, 2),
            "max_batch": args.max_batch, "batch_window_us": args.window_us, "hbm_budget_gb": args.budget_gb}
    rng = np.random.default_rng(7)

    def submit(i, pick):
        x, f, nl = pool[pick]
        return srv.submit(x, f, nl, dtype=mix[i % len(mix)])

    # warm-up
    _collect(srv, [submit(i, i % len(pool)) for i in range(2 * args.max_batch)])
    gc.collect()
    gc.disable()                       # no collector pauses in the load generator
    try:
        # peak: requests queued all at once
        n = min(args.requests, args.peak_requests)
        picks = rng.integers(0, len(pool), size=n)
        t0 = time.perf_counter()
        tickets = [submit(i, int(picks[i])) for i in range(n)]
        srv.drain()
        peak_s = time.perf_counter() - t0
        _aff, lat = _collect(srv, tickets)
        peak = n / peak_s
        print(json.dumps({**base, "offered": "saturating", "poses_per_s": peak, "requests": n,
                          "latency_ms": _pct(lat)}), flush=True)
        for load in args.loads:
            rate = load * peak
            n = args.requests
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
            picks = rng.integers(0, len(pool), size=n)
            tickets, lag = [], np.empty(n)
            t0 = time.perf_counter()
            for i in range(n):
                target = t0 + arrivals[i]
                while True:
                    now = time.perf_counter()
                    if now >= target:
                        break
                    if target - now > 0.002:
                        time.sleep(target - now - 0.001)
                lag[i] = time.perf_counter() - target
                tickets.append(submit(i, int(picks[i])))
            srv.drain()
            elapsed = time.perf_counter() - t0
            lat = _collect(srv, tickets)[1]
            slow = np.nonzero(lat > 0.010)[0]
            print(json.dumps({**base, "offered": load, "offered_poses_per_s": rate, "poses_per_s": n / elapsed,
                              "requests": n, "seconds": elapsed, "latency_ms": _pct(lat),
                              "generator_lag_ms": {"p99.9": 1e3 * float(np.percentile(lag, 99.9)),
                                                   "max": 1e3 * float(lag.max())},
                              "over_10ms": int(len(slow))}), flush=True)
    finally:
        gc.enable()
    print(json.dumps({**base, "stats": srv.stats()}), flush=True)
    srv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mix", default="bf16,fp8", help="comma-separated dtypes the requests cycle through")
    ap.add_argument("--loads", type=float, nargs="*", default=[0.25, 0.5, 0.9])
    ap.add_argument("--requests", type=int, default=20000, help="requests per offered load")
    ap.add_argument("--peak-requests", type=int, default=20000, help="requests of the saturating measurement")
    ap.add_argument("--pool-groups", type=int, default=32)
    ap.add_argument("--pool-rot", type=int, default=10)
    ap.add_argument("--jobs", type=int, default=1, help="processes generating the pool")
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--window-us", type=float, default=2000.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    run(ap.parse_args())


if __name__ == "__main__":
    main()
