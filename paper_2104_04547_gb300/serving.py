"""Serving benchmark: Poisson arrivals of synthetic poses into the continuous-batching server.

    python -m paper_2104_04547_gb300.serving [--dtype fp8] [--loads 0.25 0.5 0.9] [--requests 20000]

Poses are drawn (cycling) from a pool of docked-pose stand-ins with uneven sizes
(ligands log-normal around 32 heavy atoms, pockets 150-1000 atoms, 8 rigid
rotations per ligand).  First the peak rate is measured with every request
queued at once; then, for each offered load (a fraction of that peak), requests
arrive as a Poisson process and the per-pose latency (submission to completion,
measured by the server) is reported as p50 / p99 / p99.9 with the achieved
poses/s.  One JSON line per measurement.
"""

from __future__ import annotations

import argparse
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


def run(args):
    import torch

    from paper_2104_04547_gb300 import build
    build.build()
    from paper_2104_04547_gb300 import fusion as F
    from synth import configs, poses, weights

    torch.cuda.set_device(0)
    desc = configs.model("fusion-48grid-c64", dtype=args.dtype)
    W = weights.init_weights(desc, 0)
    blob = weights.to_blob(desc, W)
    pool = poses.make_uneven_pool(args.pool_groups, 8)
    srv = F.Server(desc, blob, max_batch=args.max_batch, slots=args.slots, batch_window_us=args.window_us,
                   hbm_budget_bytes=int(args.budget_gb * (1 << 30)), queue_capacity=1 << 22, max_atoms=1200)
    st = srv.stats()
    base = {"dtype": args.dtype, "model": "fusion-48grid-c64", "pool": f"{len(pool)} uneven poses",
            "slots": st["slots"], "slot_gb": round(st["slot_bytes"] / 2 ** 30, 2), "max_batch": args.max_batch,
            "batch_window_us": args.window_us, "hbm_budget_gb": args.budget_gb}

    def submit(i):
        x, f, nl = pool[i % len(pool)]
        return srv.submit(x, f, nl)

    # warm-up
    _collect(srv, [submit(i) for i in range(2 * args.max_batch)])
    # peak: all requests queued at once
    n = args.requests
    t0 = time.perf_counter()
    tickets = [submit(i) for i in range(n)]
    srv.drain()
    peak_s = time.perf_counter() - t0
    _aff, lat = _collect(srv, tickets)
    peak = n / peak_s
    print(json.dumps({**base, "offered": "saturating", "poses_per_s": peak, "requests": n,
                      "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                     "p99": 1e3 * float(np.percentile(lat, 99)),
                                     "p99.9": 1e3 * float(np.percentile(lat, 99.9))}}), flush=True)
    rng = np.random.default_rng(7)
    for load in args.loads:
        rate = load * peak
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        tickets = []
        t0 = time.perf_counter()
        for i in range(n):
            target = t0 + arrivals[i]
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 0.002:
                    time.sleep(target - now - 0.001)
            tickets.append(submit(i))
        srv.drain()
        elapsed = time.perf_counter() - t0
        _aff, lat = _collect(srv, tickets)
        lat = np.asarray(lat)
        slow = np.nonzero(lat > 0.010)[0]
        print(json.dumps({**base, "offered": load, "offered_poses_per_s": rate, "poses_per_s": n / elapsed,
                          "requests": n,
                          "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                         "p99": 1e3 * float(np.percentile(lat, 99)),
                                         "p99.9": 1e3 * float(np.percentile(lat, 99.9)),
                                         "max": 1e3 * float(lat.max())},
                          # requests slower than 10 ms: how many, and when they arrived (s after the start)
                          "over_10ms": {"count": int(len(slow)),
                                        "arrivals_s": [round(float(arrivals[i]), 3) for i in slow[:20]]}}),
              flush=True)
    print(json.dumps({**base, "stats": srv.stats()}), flush=True)
    srv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", choices=["f32", "bf16", "fp8"], default="fp8")
    ap.add_argument("--loads", type=float, nargs="*", default=[0.25, 0.5, 0.9])
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--pool-groups", type=int, default=32)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--window-us", type=float, default=2000.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    run(ap.parse_args())


if __name__ == "__main__":
    main()
