"""Uneven batching: pack poses of different sizes into batches by atom count.

Docked poses vary widely in size (ligands of 8-90 heavy atoms, pockets of
150-1000 atoms).  The grid half of the model costs the same per pose, but the
graph half scales with atoms, so poses are sorted by atom count and cut into
batches of similar total size; each batch is one scoring call (optionally a
CUDA-graph replay).

    python -m paper_2104_04547_gb300.batching [--groups 100] [--dtype bf16] [--passes 5] [--jobs 16]
    python -m paper_2104_04547_gb300.batching --groups 10000 --passes 1 --graphs-only --jobs 16   # 100k poses

measures poses/s over the packed batches with plain launches, with CUDA graphs,
and with graphs after the conv tile autotuner, and prints one JSON line each.

    python -m paper_2104_04547_gb300.batching --batch-sweep 1,12,23,56,64,128,256

is the batch-size study (the paper compares 12, 23 and 56 poses per rank and
transfer, Section 4.3): for each size, the same pool is cut into batches of at
most that many poses and scored end to end through the host-pointer call
(host-to-device copy of each batch and device-to-host copy of its affinities
included), one JSON line per size with poses/s and the per-call latency.
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


def pack_by_atoms(sizes, max_poses: int, atom_budget: int):
    """Batches (lists of indices) of poses sorted by atom count, each with at most
    max_poses poses and at most atom_budget atoms (a pose larger than the budget
    gets a batch of its own)."""
    order = np.argsort(np.asarray(sizes), kind="stable")
    batches, cur, cur_atoms = [], [], 0
    for i in order.tolist():
        n = int(sizes[i])
        if cur and (len(cur) == max_poses or cur_atoms + n > atom_budget):
            batches.append(cur)
            cur, cur_atoms = [], 0
        cur.append(i)
        cur_atoms += n
    if cur:
        batches.append(cur)
    return batches


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
    pool = poses.make_uneven_pool(args.groups, 10, jobs=args.jobs)
    sizes = [len(p[0]) for p in pool]
    batches = pack_by_atoms(sizes, args.max_batch, args.max_batch * 700)
    packed = [poses.pack([pool[i] for i in b]) for b in batches]
    dev = [{k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in pb.items()} for pb in packed]
    stream = torch.cuda.Stream()          # non-NULL, so the model launches on it and the events order with it
    torch.cuda.set_stream(stream)
    m = F.Model(desc, blob, max_poses=args.max_batch, max_atoms=1200, stream=stream.cuda_stream)
    out = torch.empty(args.max_batch, device="cuda")
    base = {"workload": f"{len(pool)} poses = {args.groups} ligands x 10 rigid poses, ligands log-normal "
                        f"(median 32, 8-90 atoms), pockets 150-1000 atoms", "dtype": args.dtype,
            "batches": len(batches), "max_batch": args.max_batch,
            "atoms_per_pose_mean": float(np.mean(sizes))}

    def timed(label, passes=args.passes):
        # one untimed pass over every batch: each batch size's graph is captured here, not in the timed loop;
        # then `passes` timed passes over the pool, reported as the median (and the range)
        for pb, db in zip(packed, dev):
            m.score(db, n_poses=len(pb["n_lig"]), out=out, on_device=True)
        torch.cuda.synchronize()
        rates = []
        for _ in range(passes):
            t0 = time.perf_counter()
            for pb, db in zip(packed, dev):
                m.score(db, n_poses=len(pb["n_lig"]), out=out, on_device=True)
            torch.cuda.synchronize()
            rates.append(len(pool) / (time.perf_counter() - t0))
        print(json.dumps({**base, "mode": label, "poses_per_s": float(np.median(rates)),
                          "poses_per_s_range": [float(min(rates)), float(max(rates))], "passes": passes}), flush=True)

    if not args.graphs_only:
        timed("plain launches")
    m.use_cuda_graphs(True)
    timed("cuda graphs")
    if args.graphs_only:
        m.close()
        return
    m.autotune(packed[len(packed) // 2])
    print(json.dumps({**base, "autotuned_tiles": m.conv_tiles(), "graph_nodes_per_warp": m.graph_nodes_per_warp()}),
          flush=True)
    timed("cuda graphs + autotuned tiles")
    # per-compound ranking as the paper does it: each ligand's strongest affinity over its 10 poses
    aff = np.empty(len(pool), dtype=np.float32)
    for b, pb, db in zip(batches, packed, dev):
        m.score(db, n_poses=len(pb["n_lig"]), out=out, on_device=True)
        aff[b] = out[:len(b)].cpu().numpy()
    best, idx = F.fusion_best_per_compound(aff, np.arange(len(pool)) // 10, args.groups)
    top = np.argsort(-best, kind="stable")[:5]
    print(json.dumps({**base, "per_compound_best": {"compounds": int(args.groups),
                      "top5": [{"compound": int(c), "affinity": float(best[c]), "pose": int(idx[c])} for c in top]}}),
          flush=True)
    m.close()


def batch_sweep(args):
    import torch

    from paper_2104_04547_gb300 import build
    build.build()
    from paper_2104_04547_gb300 import fusion as F
    from synth import configs, poses, weights

    torch.cuda.set_device(0)
    desc = configs.model("fusion-48grid-c64", dtype=args.dtype)
    blob = weights.to_blob(desc, weights.init_weights(desc, 0))
    pool = poses.make_uneven_pool(args.groups, 10, jobs=args.jobs)
    sizes = [len(p[0]) for p in pool]
    for mb in [int(v) for v in args.batch_sweep.split(",")]:
        batches = pack_by_atoms(sizes, mb, mb * 700)
        packed = [poses.pack([pool[i] for i in b]) for b in batches]
        m = F.Model(desc, blob, max_poses=mb, max_atoms=1200)
        for pb in packed[:2]:
            m.score(pb)
        lat = []
        t0 = time.perf_counter()
        for pb in packed:
            t = time.perf_counter()
            m.score(pb)                      # host inputs in, affinities back on the host
            lat.append(time.perf_counter() - t)
        dt = time.perf_counter() - t0
        m.close()
        print(json.dumps({"study": "poses per call", "dtype": args.dtype, "max_batch": mb, "calls": len(packed),
                          "poses": len(pool), "poses_per_s": len(pool) / dt,
                          "call_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                      "p99": 1e3 * float(np.percentile(lat, 99))}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--groups", type=int, default=100)
    ap.add_argument("--dtype", choices=["f32", "bf16", "fp8"], default="bf16")
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--batch-sweep", default="", help="comma-separated batch sizes: run the batch-size study")
    ap.add_argument("--passes", type=int, default=5, help="timed passes over the pool per mode (median reported)")
    ap.add_argument("--graphs-only", action="store_true", help="time only the CUDA-graph mode (large pools)")
    ap.add_argument("--jobs", type=int, default=1, help="processes generating the pool")
    args = ap.parse_args()
    if args.batch_sweep:
        batch_sweep(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
