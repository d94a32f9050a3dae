#!/usr/bin/env python
"""Throughput of Coherent Fusion pose scoring on GB300.

One step = one scoring call over a batch of 64 synthetic poses (ligands 20-50
heavy atoms, pockets 300-600 atoms, seeds 1..64) with the full-size model
(48^3 x 19 grid, conv 19->64 7^3, two residual 64-channel 7^3 blocks, conv
64->128 5^3 stride 2, pool, dense 256; 3+3 gated graph steps at hidden 64,
gated ligand pooling to 128; head 384->256->64->1): voxelize, 3D-CNN, radius
graph, graph convolution, gather and head, all in the CUDA library.

    python bench.py [--steps K] [--warmup W] [--dtype f32|bf16|fp8] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank scores its own copy of the
batch with no data-path collective (replicas; weak scaling).  Rank 0 prints
one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "poses/sec + p50/p99 latency on 1 GB300, BF16/FP8 vs FP32 at |Δaffinity|≤0.05"
MODEL = "fusion-48grid-c64"
WORKLOAD = "batch64-lig20to50-pocket300to600"
WEIGHTS_SEED = 0
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz maximum SM clock.
F32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the four conv launches of one step, taken
# with ncu on a 16-pose batch of this workload (activations 226 MB > L2) and scaled x4 to 64 poses (every
# tensor but the weights scales with the pose count).  Valid only for the kernel source they were taken
# on: the sha256 prefix of the conv kernel's source code (comments removed); other code reports null.
CONV_TRAFFIC = {
    "src": "bee8dc0556ebdbad",
    "poses": 64,
    "bf16": [1135.8e6, 1680.9e6, 1647.2e6, 1080.4e6],
    "fp8": [1148.8e6, 2113.4e6, 2113.5e6, 554.4e6],
}


def conv_source_hash():
    """sha256 prefix of the conv kernel's source files with comments and blank lines removed (a code
    change invalidates the measured traffic; an edit of a comment does not)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("k_conv_tc.cu", "tc_ptx.cuh"):
        with open(os.path.join(ROOT, "paper_2104_04547_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(l.rstrip() for l in src.splitlines() if l.strip()).encode())
    return h.hexdigest()[:16]


def conv_traffic(dtype, n_poses, model=MODEL):
    """Measured DRAM bytes per conv launch (mean of the step's launches), or None."""
    if (model != MODEL or dtype not in CONV_TRAFFIC or n_poses != CONV_TRAFFIC["poses"] or
            conv_source_hash() != CONV_TRAFFIC["src"]):
        return None
    v = CONV_TRAFFIC[dtype]
    return sum(v) / len(v)


def conv_algorithmic_bytes(desc, dtype, n_poses):
    """Input + output (+ the bf16 residual source for FP8) + arranged weights, per conv launch (mean).

    The first layer reads the stored grid: 32 bf16 channels per voxel, or for FP8 the folded grid of
    n x n x (n + 1) voxels x 64 codes; its weights are arranged for the folded input (BF16: 7 + 2
    x-offsets per kernel row for k = 7; FP8: 4 + 1).  Other layers: k^3 x 32 bytes x C_out of weights
    per 32-byte channel chunk."""
    n, tot, cin = desc["grid_n"], [], 32
    elem = 1 if dtype == "fp8" else 2
    for i, cv in enumerate(desc["conv"]):
        p = cv["k"] // 2
        m = (n + 2 * p - cv["k"]) // cv["stride"] + 1
        k, co = cv["k"], cv["c_out"]
        folded = i == 0 and grid_folded(desc)
        if folded and elem == 2:
            b_in = n ** 3 * 32 * 2
            wbytes = k ** 3 * co * 32 + k * (1 if k <= 5 else 2) * k * co * 32
        elif folded:
            b_in = n * n * (n + 1) * 64
            wbytes = k * ((k + 1) // 2 + 1) * k * co * 32
        else:
            b_in = n ** 3 * cin * elem
            wbytes = (cin * elem // 32) * k ** 3 * co * 32
        b = b_in + m ** 3 * co * 2
        if elem == 1 and cv["residual"]:
            b += n ** 3 * cin * 2
        tot.append(b * n_poses + wbytes)
        n, cin = m, co
    return sum(tot) / len(tot)


def conv_flops_per_pose(desc):
    n, tot = desc["grid_n"], 0
    for cv in desc["conv"]:
        p = cv["k"] // 2
        n = (n + 2 * p - cv["k"]) // cv["stride"] + 1
        tot += 2 * n ** 3 * cv["c_out"] * cv["c_in"] * cv["k"] ** 3
    return tot


def launches_per_step(desc):
    # prep + voxelize, the convs, the pool, dense + its reduction, the radius graph (count, scan, fill),
    # a transform per stage, the steps, the gather, the head
    return (2 + len(desc["conv"]) + (1 if desc["pool"] > 1 else 0) + 2 + 3 +
            len(desc["sg_stages"]) + sum(s["steps"] for s in desc["sg_stages"]) + 1 + 1)


def grid_folded(desc):
    """The bf16 path stores the grid's channels 16..18 folded along x (one extra pass after voxelize)."""
    c0 = desc["conv"][0]
    return c0["stride"] == 1 and c0["k"] in (3, 5, 7) and not c0["residual"] and c0["c_in"] == 19


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def cpu_baseline(desc, W, batch, n_poses=1):
    """The FP64 oracle as it stands on this host's cores, over the first n_poses poses."""
    from oracle import fusion_oracle as O
    from synth import poses
    t = time.perf_counter()
    for p in range(n_poses):
        O.score_pose(desc, W, *poses.pose_slice(batch, p))
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": n_poses / dt, "unit": "poses/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_poses} of 64 poses of the workload (full FP64 forward per pose), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import configs, poses, weights
    desc = configs.model(args.model)
    W = weights.init_weights(desc, WEIGHTS_SEED)
    batch = poses.make_batch(configs.WORKLOADS[WORKLOAD])
    from oracle import fusion_oracle as O
    # one step = the oracle's full forward of one pose of the batch (a bounded sample)
    for w in range(args.warmup):
        O.score_pose(desc, W, *poses.pose_slice(batch, w % 64))
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        O.score_pose(desc, W, *poses.pose_slice(batch, (args.warmup + k) % 64))
        times.append(time.perf_counter() - t)
    tot = sum(times)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    v = args.steps / tot
    line = {"metric": METRIC, "value": v, "unit": "poses/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.model} scoring, {WORKLOAD}", "sample_per_step": "1 pose"},
            "cpu_baseline": {"value": v, "unit": "poses/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} poses of the workload, one per step"},
            "e2e": {"value": v, "unit": "poses/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_2104_04547_gb300 import build
    build.build()
    from paper_2104_04547_gb300 import fusion as F
    from synth import configs, poses, weights

    desc = configs.model(args.model, dtype=args.dtype)
    W = weights.init_weights(desc, WEIGHTS_SEED)
    blob = weights.to_blob(desc, W)
    batch = poses.make_batch(configs.WORKLOADS[WORKLOAD])
    if args.poses < len(batch["n_lig"]):
        batch = poses.subset(batch, range(args.poses))     # profiling captures only
    B = len(batch["n_lig"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(desc, W, batch, 1)

    stream = torch.cuda.current_stream()
    model = F.Model(desc, blob, max_poses=B, max_atoms=1200, max_degree=64, stream=stream.cuda_stream)
    devb = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in batch.items()}
    out = torch.empty(B, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        model.score(devb, n_poses=B, out=out, on_device=True)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(dev)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_ms = []
    for k in range(args.steps):
        flush.zero_()                     # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        model.score(devb, n_poses=B, out=out, on_device=True)
        ev[k][1].record(stream)
        stage_ms.append(model.timings())
    barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    tot_ms = sum(step_ms)
    t = torch.tensor([tot_ms], device="cuda", dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot_ms = float(t.item())
    value = world * B * args.steps / (tot_ms / 1000.0)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in batch.items()}
        host = {k: v.numpy() for k, v in pinned.items()}
        hout = torch.empty(B, dtype=torch.float32).pin_memory().numpy()
        model.score(host, n_poses=B, out=hout)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            model.score(host, n_poses=B, out=hout)
        barrier()
        wall = time.perf_counter() - t0
        tw = torch.tensor([wall], device="cuda", dtype=torch.float64)
        if dist is not None:
            dist.all_reduce(tw, op=dist.ReduceOp.MAX)
        wall = float(tw.item())
        h2d = sum(int(v.nbytes) for v in host.values())
        e2e = {"value": world * B * args.steps / wall, "unit": "poses/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 4 * B}

    # |affinity difference| against the FP32 path on the same batch (outside the timed region)
    delta = None
    fp32_path = None
    if args.dtype != "f32" and not args.no_f32_compare:
        got = out.float().cpu().numpy().copy()
        d32 = configs.model(args.model, dtype="f32")
        m32 = F.Model(d32, weights.to_blob(d32, W), max_poses=B, max_atoms=1200, max_degree=64,
                      stream=stream.cuda_stream)
        ref = m32.score(batch).copy()
        # the plain FP32 path (CUDA cores) on the same GPU in the same run: one more step, timed
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out32 = torch.empty(B, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        e0.record(stream)
        m32.score(devb, n_poses=B, out=out32, on_device=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t32 = e0.elapsed_time(e1)
        fp32_path = {"value": B / (t32 / 1000.0), "unit": "poses/s", "ms_per_step": t32,
                     "note": "FP32 CUDA-core path, same batch and GPU, one step after one untimed step"}
        m32.close()
        dd = np.abs(got - ref)
        delta = {"vs": "f32 path, same poses and weights", "mean": float(dd.mean()), "max": float(dd.max()),
                 "tolerance": 0.05}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    conv_names = [f"conv{i}" for i in range(len(desc["conv"]))]
    conv_ms = statistics.mean(sum(s[n] for n in conv_names) for s in stage_ms)
    conv_flops = conv_flops_per_pose(desc) * B
    achieved = conv_flops / (conv_ms / 1000.0) / 1e12
    pk, pk_src = peaks()
    traffic = conv_traffic(args.dtype, B, args.model)
    if args.dtype == "f32":
        roof = {"bound": "alu", "achieved": achieved, "peak": F32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / F32_ALU_PEAK_TFLOPS, "traffic": None,
                "kernel": f"conv3d_f32_kernel ({len(conv_names)} launches per step)",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    else:
        # The burst peak: the step keeps the SM clock at its maximum (see `clocks`), while the sustained
        # figure was taken with the clock held down by the power cap, so it would flatter the kernel.
        # No FP8 peak is measured: FP8 uses the BF16 figure x the nominal FP8/BF16 ratio (4.5 / 2.25).
        ratio = 2.0 if args.dtype == "fp8" else 1.0
        p = pk["bf16_tflops"] * ratio
        ps = pk["bf16_tflops_sustained"] * ratio
        roof = {"bound": "tensor", "achieved": achieved, "peak": p, "unit": "TFLOP/s", "frac": achieved / p,
                "traffic": traffic, "kernel": f"conv3d_tc_kernel {args.dtype} ({len(conv_names)} launches per step)",
                "peak_source": f"bf16_tflops burst ({pk_src})" + (" x 2 (nominal fp8/bf16 ratio)" if ratio != 1 else ""),
                "frac_of_sustained": achieved / ps}
    if args.dtype != "f32":
        roof["traffic_unit"] = f"DRAM bytes per conv launch (mean of the step's {len(conv_names)}), ncu"
        roof["algorithmic_bytes"] = conv_algorithmic_bytes(desc, args.dtype, B)
    stage_mean = {n: statistics.mean(s[n] for s in stage_ms) for n in stage_ms[0]}
    line = {
        "metric": METRIC, "value": value, "unit": "poses/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": f"{args.model} scoring, {WORKLOAD}", "batch": B,
                   "grid": f"{desc['grid_n']}^3x19 at {desc['grid_h']:g} A",
                   "l2": "256 MiB written between timed steps; step working set (activations) > L2",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "note": "per-pose latency = its batch's latency (all 64 poses finish together)"},
        "stage_ms": {k: round(v, 4) for k, v in stage_mean.items() if v > 0},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": (launches_per_step(desc) + (len(desc["conv"]) if args.dtype == "fp8" else 0) +
                         (1 if args.dtype == "bf16" and grid_folded(desc) else 0)) * args.steps,
        "clocks": clk,
        "affinity_std": float(out.float().std().item()),
    }
    if delta is not None:
        line["delta_affinity"] = delta
    if fp32_path is not None:
        line["fp32_path"] = fp32_path
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["f32", "bf16", "fp8"], default="bf16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f32-compare", action="store_true")
    ap.add_argument("--poses", type=int, default=64, help="first N poses of the batch (small profiling captures)")
    ap.add_argument("--model", default=MODEL,
                    help="model preset (synth.configs); the benchmark model by default, others for comparison")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
