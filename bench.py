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
    "src": "08911989fe3505da",
    "poses": 64,
    "bf16": [1134.8e6, 1660.2e6, 1671.1e6, 1055.5e6],
    "fp8": [1149.1e6, 2102.8e6, 2101.0e6, 552.1e6],
}


# DRAM bytes of one voxelize launch at 64 poses (ncu dram__bytes_read.sum + dram__bytes_write.sum), valid for the
# voxelize source they were taken on (sha256 prefix as for the conv); otherwise null.
# Taken on 32 poses (171.96 MB = 3.46 MB read + 168.50 MB written) and scaled x2: the grid and the records scale
# with the pose count.  Part of a launch's writes can still sit in L2 when it ends, so this undercounts slightly.
VOX_TRAFFIC = {
    "src": "d333f95110c47935",
    "poses": 64,
    "bf16": 2 * 171.96e6,
}


def conv_source_hash(files=("k_conv_tc.cu", "tc_ptx.cuh")):
    """sha256 prefix of the kernel's source files with comments and blank lines removed (a code
    change invalidates the measured traffic; an edit of a comment does not)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
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


def vox_traffic(dtype, n_poses, model=MODEL):
    """Measured DRAM bytes of one voxelize launch, or None."""
    if (model != MODEL or n_poses != VOX_TRAFFIC["poses"] or dtype not in VOX_TRAFFIC or
            conv_source_hash(("k_voxelize.cu",)) != VOX_TRAFFIC["src"]):
        return None
    return VOX_TRAFFIC[dtype]


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
    # prep + voxelize, the convs, the pool, dense + its reduction (and a second dense layer's two), the radius
    # graph (count, scan, fill),
    # a transform per stage, the steps (tensor-core models: message sums, then the tensor-core GRU), the gather,
    # the head
    per_step = 2 if desc.get("dtype", "f32") != "f32" else 1
    return (2 + len(desc["conv"]) + (1 if desc["pool"] > 1 else 0) + 2 + (2 if desc.get("cnn_dense2") else 0) + 3 +
            len(desc["sg_stages"]) + per_step * sum(s["steps"] for s in desc["sg_stages"]) + 1 + 1)


def golden_affinities():
    """Stored FP64 oracle affinities of this workload's poses ({pose: affinity}; written by the committed golden
    script, which calls only the oracle), or {} when the file is missing."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "full64_w0.json")) as f:
            g = json.load(f)
    except OSError:
        return {}
    if g.get("model") != MODEL or g.get("workload") != WORKLOAD or g.get("weights_seed") != WEIGHTS_SEED:
        return {}
    return {int(k): float(v["affinity"]) for k, v in g["poses"].items()}


def delta_vs_oracle(got, model_name, batch_digest, gold_digest, gold):
    """|affinity - stored FP64 oracle| over the stored poses (None if they do not apply to this run)."""
    import numpy as np
    if model_name != MODEL or not gold or batch_digest != gold_digest:
        return None
    idx = sorted(p for p in gold if p < len(got))
    d = np.abs(np.asarray([got[p] for p in idx], dtype=np.float64) - np.asarray([gold[p] for p in idx]))
    return {"vs": f"FP64 oracle, stored values of {len(idx)} poses", "mean": float(d.mean()), "max": float(d.max()),
            "tolerance": 0.05}


def voxelize_algorithmic_bytes(desc, dtype, n_atoms):
    """Grid write n^3 x 19 channels x element size per pose + atom reads (12 B coordinates + 76 B features)."""
    esz = 4 if dtype == "f32" else 2
    return desc["grid_n"] ** 3 * 19 * esz, 88 * n_atoms


def graph_branch_flops(desc, n_atoms, n_lig, e_cov, e_nc):
    """Algorithmic flops of the gated graph convolution and gather of one pose: 2 per multiply-add of the edge
    transforms, stage gate, GRU (input and hidden matrices) and gather matrices, plus H additions per directed
    edge in the message sums.  The radius graph is integer and compare work, not counted."""
    H, G = desc["sg_hidden"], desc["sg_gather_width"]
    N = n_atoms
    f = 0
    for s, st in enumerate(desc["sg_stages"]):
        types = [e for e, bit in ((e_cov, 1), (e_nc, 2)) if st["edges"] & bit]
        nt = len(types)
        if s > 0 and desc["sg_gate"]:
            f += N * (2 * 2 * H * H + 2 * H * H)             # sigmoid(W_i [h, h0] + b) * (W_j h + b)
        if st["steps"] > 0:
            f += N * nt * 2 * H * H                          # first transforms W_e h + b_e
        for k in range(st["steps"]):
            f += N * 2 * 2 * 3 * H * H                       # GRU: W_ih m and W_hh h, three gates each
            f += sum(types) * H                              # message sums over the directed edges
            if k + 1 < st["steps"]:
                f += N * nt * 2 * H * H                      # transforms of the new states
    f += n_lig * (2 * 2 * H * G + 2 * H * G if desc["sg_gather"] == "gated" else 2 * H * G)
    return f


def measure_fp8_peak(torch):
    """Dense FP8 E4M3 GEMM throughput on this GPU (torch._scaled_mm, 8192^3, best of 10 with and without fast
    accumulation), TFLOP/s; None when the call is unavailable."""
    n = 8192
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda", dtype=torch.float32)
        best = None
        for fast in (False, True):
            for _ in range(3):
                torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16, use_fast_accum=fast)
            for _ in range(10):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16, use_fast_accum=fast)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3
                v = 2 * n ** 3 / t / 1e12
                best = v if best is None else max(best, v)
        del a, b
        torch.cuda.empty_cache()
        return best
    except Exception:
        return None


def grid_folded(desc):
    """The bf16 path stores the grid's channels 16..18 folded along x (written so by voxelize)."""
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


def time_steps(model, devb, B, out, stream, flush, steps, warmup, barrier):
    """W untimed calls, then K calls each bracketed by CUDA events on the model's stream, with the L2 flushed
    between them outside the events.  Returns (per-step ms, per-step stage timings)."""
    import torch
    for _ in range(warmup):
        model.score(devb, n_poses=B, out=out, on_device=True)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stage_ms = []
    for k in range(steps):
        flush.zero_()                     # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        model.score(devb, n_poses=B, out=out, on_device=True)
        ev[k][1].record(stream)
        stage_ms.append(model.timings())
    barrier()
    return [s.elapsed_time(e) for s, e in ev], stage_ms


def paper_final_run(F, torch, batch, devb, B, stream, flush, steps, warmup, barrier):
    """The `fusion-paper-final` model on this batch: BF16 and FP8 poses/s (K timed calls each, as for the main
    line), and each dtype's |affinity difference| against the model's FP32 path (one call)."""
    import numpy as np
    from synth import configs, weights
    name = "fusion-paper-final"
    W = weights.init_weights(configs.model(name), WEIGHTS_SEED)
    d32 = configs.model(name, dtype="f32")
    m32 = F.Model(d32, weights.to_blob(d32, W), max_poses=B, max_atoms=1200, max_degree=64, stream=stream.cuda_stream)
    ref = m32.score(batch).copy()
    m32.close()
    res = {"model": f"{name} (3D-CNN 32/64 filters, SG-CNN widths 19 and 24, 6 + 3 graph steps)"}
    for dt in ("bf16", "fp8"):
        d = configs.model(name, dtype=dt)
        m = F.Model(d, weights.to_blob(d, W), max_poses=B, max_atoms=1200, max_degree=64, stream=stream.cuda_stream)
        o = torch.empty(B, dtype=torch.float32, device="cuda")
        sm, _st = time_steps(m, devb, B, o, stream, flush, steps, warmup, barrier)
        got = o.float().cpu().numpy().copy()
        m.close()
        dd = np.abs(got.astype(np.float64) - ref)
        res[dt] = {"value": B * steps / (sum(sm) / 1000.0), "unit": "poses/s", "ms_per_step": sum(sm) / steps,
                   "delta_vs_fp32_path": {"mean": float(dd.mean()), "max": float(dd.max()), "tolerance": 0.05}}
    return res


def conv_roofline(desc, dtype, B, stage_ms, pk, pk_src, model_name, fp8_peak=None):
    import statistics as st
    conv_names = [f"conv{i}" for i in range(len(desc["conv"]))]
    conv_ms = st.mean(sum(s[n] for n in conv_names) for s in stage_ms)
    achieved = conv_flops_per_pose(desc) * B / (conv_ms / 1000.0) / 1e12
    if dtype == "f32":
        return {"bound": "alu", "achieved": achieved, "peak": F32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / F32_ALU_PEAK_TFLOPS, "traffic": None,
                "kernel": f"conv3d_f32_kernel ({len(conv_names)} launches per step)",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    # The burst peak: the step keeps the SM clock at its maximum (see `clocks`), while the sustained figure was
    # taken with the clock held down by the power cap, so it would flatter the kernel.
    if dtype == "fp8" and fp8_peak:
        p, src = fp8_peak, "FP8 E4M3 GEMM measured in this run (torch._scaled_mm 8192^3, best of 10)"
        ps = None
    else:
        ratio = 2.0 if dtype == "fp8" else 1.0
        p = pk["bf16_tflops"] * ratio
        ps = pk["bf16_tflops_sustained"] * ratio
        src = f"bf16_tflops burst ({pk_src})" + (" x 2 (nominal fp8/bf16 ratio)" if ratio != 1 else "")
    roof = {"bound": "tensor", "achieved": achieved, "peak": p, "unit": "TFLOP/s", "frac": achieved / p,
            "traffic": conv_traffic(dtype, B, model_name),
            "kernel": f"conv3d_tc_kernel {dtype} ({len(conv_names)} launches per step)", "peak_source": src}
    if ps:
        roof["frac_of_sustained"] = achieved / ps
    roof["traffic_unit"] = f"DRAM bytes per conv launch (mean of the step's {len(conv_names)}), ncu"
    roof["algorithmic_bytes"] = conv_algorithmic_bytes(desc, dtype, B)
    return roof


def edge_counts(F, model, batch, B):
    """Directed covalent and non-covalent edges of each pose of the last call (from the CSR sizes)."""
    off = batch["atom_off"]
    ec, en = [], []
    for p in range(B):
        N = int(off[p + 1] - off[p])
        ec.append(F.fusion_stage_bytes(model.handle, F.STAGE_EDGES_COV, p) // 4 - N - 1)
        en.append(F.fusion_stage_bytes(model.handle, F.STAGE_EDGES_NC, p) // 4 - N - 1)
    return ec, en


def side_rooflines(F, model, desc, dtype, batch, B, devb, out, stage_ms, pk, pk_src):
    """Voxelize (HBM), the graph branch (FP32 ALU) and the CNN dense (HBM, its weight stream): each kernel
    group's algorithmic work over its own CUDA-event time.  Voxelize is timed in the timed steps (it runs on
    the grid branch's stream); the graph branch overlaps the convolutions there, so it is timed in three more
    calls with both branches on one stream (FUSION_OPT_SERIAL_BRANCHES), median per stage."""
    import statistics as st
    import torch
    off = batch["atom_off"]
    n_atoms = [int(off[p + 1] - off[p]) for p in range(B)]
    grid_b, atom_b = voxelize_algorithmic_bytes(desc, dtype, 1)
    vox_bytes = B * grid_b + atom_b * sum(n_atoms)
    vox_ms = st.mean(s["voxelize"] for s in stage_ms)
    hbm = pk["hbm_gbs"]
    vox_gbs = vox_bytes / (vox_ms / 1e3) / 1e9
    model.serial_branches(True)
    ser = []
    for _ in range(3):
        model.score(devb, n_poses=B, out=out, on_device=True)
        ser.append(model.timings())
    model.serial_branches(False)
    torch.cuda.synchronize()
    vox_alone = st.median(s["voxelize"] for s in ser)
    out_ = {"voxelize": {"bound": "hbm", "achieved": vox_gbs, "peak": hbm, "unit": "GB/s", "frac": vox_gbs / hbm,
                         "traffic": vox_traffic(dtype, B, desc["name"]), "algorithmic_bytes": vox_bytes,
                         "kernel_ms": vox_ms, "kernel": f"voxelize_kernel ({dtype} grid, one launch per step)",
                         "peak_source": f"hbm_gbs ({pk_src})",
                         "alone": {"kernel_ms": vox_alone, "frac": vox_bytes / (vox_alone / 1e3) / 1e9 / hbm,
                                   "note": "the same launch with the graph branch serialised after the grid branch "
                                           "(in the timed steps the graph branch's first kernels share the GPU)"}}}
    ec, en = edge_counts(F, model, batch, B)
    fl = sum(graph_branch_flops(desc, n_atoms[p], int(batch["n_lig"][p]), ec[p], en[p]) for p in range(B))
    g_ms = st.median(s["sg_steps"] + s["sg_gather"] for s in ser)
    r_ms = st.median(s["radius_graph"] for s in ser)
    g_tf = fl / (g_ms / 1e3) / 1e12
    out_["graph_branch"] = {
        "bound": "alu", "achieved": g_tf, "peak": F32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": g_tf / F32_ALU_PEAK_TFLOPS, "traffic": None, "algorithmic_flops": fl, "kernel_ms": g_ms,
        "radius_graph_ms": r_ms, "edges_per_pose": (sum(ec) + sum(en)) / B,
        "kernel": ("sg_transform_kernel + sg_step_kernel + sg_gather_kernel (FP32 CUDA cores)" if dtype == "f32" else
                   "sg_stage_tc_kernel (stage gate and first transforms) + per step sg_message_kernel and "
                   "sg_gru_tc_kernel (GRU and next transforms), the contractions on the tcgen05 tensor cores with "
                   "three BF16 terms per product, + sg_gather_kernel") +
                  ", timed with the branches serialised",
        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz" +
                       ("" if dtype == "f32" else "; achieved counts the FP32 algorithmic flops once (the "
                                                  "tensor cores execute the products three times)")}
    if dtype != "f32":
        K = model_flat(desc)
        wbytes = desc["cnn_dense"] * K * 2
        d_ms = st.median(s["cnn_dense"] for s in ser)
        d_gbs = (wbytes + B * K * 2) / (d_ms / 1e3) / 1e9
        out_["cnn_dense"] = {"bound": "hbm", "achieved": d_gbs, "peak": hbm, "unit": "GB/s", "frac": d_gbs / hbm,
                             "traffic": None, "algorithmic_bytes": wbytes + B * K * 2, "kernel_ms": d_ms,
                             "kernel": "dense_tc_kernel + dense_reduce_kernel (bf16 weight stream)",
                             "peak_source": f"hbm_gbs ({pk_src})"}
    return out_


def model_flat(desc):
    n, c = desc["grid_n"], 19
    for cv in desc["conv"]:
        n = (n + 2 * (cv["k"] // 2) - cv["k"]) // cv["stride"] + 1
        c = cv["c_out"]
    if desc["pool"] and desc["pool"] > 1:
        n //= desc["pool"]
    return c * n ** 3


def serving_run(F, desc_name, W, blob_of, requests, seconds_cap=60.0):
    """A bounded serving measurement: one server with BF16 and FP8 slots (requests alternate between the two,
    as in the serving workload's mix), uneven poses (ligands log-normal around 32 atoms, pockets 150-1000),
    first saturating (all queued at once) for the peak, then (after 500 unmeasured requests) Poisson arrivals
    at 25% (three runs), 50% and 90% of it.  Per-pose latency is the server's submission-to-completion time;
    `generator_lag_ms` is how late the load generator submitted (a stall there shows up as a burst)."""
    import gc

    import numpy as np

    from synth import configs, poses
    desc = configs.model(desc_name, dtype="bf16")
    pool = poses.make_uneven_pool(16, 8)
    srv = F.Server(desc, blob_of("bf16"), max_batch=64, slots=4, batch_window_us=2000.0,
                   hbm_budget_bytes=120 << 30, queue_capacity=1 << 22, max_atoms=1200, dtypes=("fp8",))
    dts = ["bf16", "fp8"]

    def submit(i):
        x, f, nl = pool[i % len(pool)]
        return srv.submit(x, f, nl, dtype=dts[i % 2])

    def collect(tickets):
        lat = np.empty(len(tickets))
        for i, t in enumerate(tickets):
            r = srv.poll(t)
            while r is None:
                time.sleep(0.0002)
                r = srv.poll(t)
            lat[i] = r[1]
        return lat

    def pct(lat):
        return {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
                "p99.9": 1e3 * float(np.percentile(lat, 99.9)), "max": 1e3 * float(lat.max())}

    def poisson(rate, n, rng):
        """n requests at Poisson arrivals of `rate`; returns (latencies, achieved poses/s, generator lag)."""
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
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
            tickets.append(submit(i))
        srv.drain()
        elapsed = time.perf_counter() - t0
        return collect(tickets), n / elapsed, lag

    collect([submit(i) for i in range(256)])            # warm-up
    gc.collect()
    gc.disable()                                       # no collector pauses in the load generator
    try:
        t0 = time.perf_counter()
        tickets = [submit(i) for i in range(requests)]
        srv.drain()
        peak = requests / (time.perf_counter() - t0)
        res = {"saturating": {"poses_per_s": peak, "requests": requests, "latency_ms": pct(collect(tickets))}}
        rng = np.random.default_rng(7)
        poisson(0.25 * peak, 500, rng)                 # unmeasured: the generator and the slots settle first
        for load, reps in ((0.25, 3), (0.5, 1), (0.9, 1)):
            n = int(min(requests, load * peak * seconds_cap / 10))
            for r in range(reps):
                lat, achieved, lag = poisson(load * peak, n, rng)
                res[f"load_{int(load * 100)}" + (f"_run{r + 1}" if reps > 1 else "")] = {
                    "offered_poses_per_s": load * peak, "poses_per_s": achieved, "requests": n,
                    "latency_ms": pct(lat),
                    "generator_lag_ms": {"p99.9": 1e3 * float(np.percentile(lag, 99.9)),
                                         "max": 1e3 * float(lag.max())}}
    finally:
        gc.enable()
    st = srv.stats()
    srv.close()
    res.update({"slots": st["slots_by_dtype"], "slot_gb": round(st["slot_bytes"] / 2 ** 30, 2), "max_batch": 64,
                "batch_window_us": 2000.0, "hbm_budget_gb": 120, "dtype_mix": "requests alternate bf16 / fp8",
                "pool": f"{len(pool)} uneven poses (16 ligands x 8 rigid poses)",
                "latency": "per pose, submission to completion (server clock)"})
    return res


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
    full_digest = poses.digest(batch)
    if args.poses < len(batch["n_lig"]):
        batch = poses.subset(batch, range(args.poses))     # profiling captures only
    B = len(batch["n_lig"])
    gold = golden_affinities() if B == 64 else {}
    gold_digest = full_digest if B == 64 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(desc, W, batch, 1)

    # a stream of our own, made current: the model launches on it (a NULL handle, torch's legacy default stream,
    # would make the model create a stream of its own), so the L2 flush, the timing events and the model's work
    # are ordered on one stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    model = F.Model(desc, blob, max_poses=B, max_atoms=1200, max_degree=64, stream=stream.cuda_stream)
    devb = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in batch.items()}
    out = torch.empty(B, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(dev)
    step_ms, stage_ms = time_steps(model, devb, B, out, stream, flush, args.steps, args.warmup, barrier)
    clk = clocks.stop()
    tot_ms = sum(step_ms)
    t = torch.tensor([tot_ms], device="cuda", dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot_ms = float(t.item())
    value = world * B * args.steps / (tot_ms / 1000.0)
    got = out.float().cpu().numpy().copy()

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

    pk, pk_src = peaks()
    extra = {}
    # dense FP8 GEMM throughput measured on this GPU in this run (the FP8 conv's roofline denominator)
    fp8_peak = measure_fp8_peak(torch) if rank == 0 and args.dtype in ("bf16", "fp8") and not args.no_extras else None
    if rank == 0 and not args.no_extras:
        extra["rooflines"] = side_rooflines(F, model, desc, args.dtype, batch, B, devb, out, stage_ms, pk, pk_src)

    # |affinity difference| against the stored FP64 oracle values, and against the FP32 path on the same batch
    delta = delta_vs_oracle(got, args.model, full_digest if B == 64 else None, gold_digest, gold)
    fp32_path = None
    if args.dtype != "f32" and not args.no_f32_compare:
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
        dd = np.abs(got - ref)
        fp32_path = {"value": B / (t32 / 1000.0), "unit": "poses/s", "ms_per_step": t32,
                     "note": "FP32 CUDA-core path, same batch and GPU, one step after one untimed step",
                     "delta_vs_this_dtype": {"mean": float(dd.mean()), "max": float(dd.max())},
                     "delta_vs_oracle": delta_vs_oracle(ref, args.model, full_digest if B == 64 else None,
                                                        gold_digest, gold)}
        m32.close()

    # the other tensor-core dtype (FP8 beside a BF16 run, BF16 beside FP8): same batch, same timing rules
    if rank == 0 and args.dtype in ("bf16", "fp8") and not args.no_extras:
        other = "fp8" if args.dtype == "bf16" else "bf16"
        d2 = configs.model(args.model, dtype=other)
        m2 = F.Model(d2, weights.to_blob(d2, W), max_poses=B, max_atoms=1200, max_degree=64, stream=stream.cuda_stream)
        out2 = torch.empty(B, dtype=torch.float32, device="cuda")
        sm2, st2 = time_steps(m2, devb, B, out2, stream, flush, args.steps, args.warmup, barrier)
        got2 = out2.float().cpu().numpy().copy()
        m2.close()
        extra[other] = {"value": B * args.steps / (sum(sm2) / 1000.0), "unit": "poses/s",
                        "ms_per_step": sum(sm2) / args.steps,
                        "latency_ms": {"p50": float(np.percentile(sm2, 50)), "p99": float(np.percentile(sm2, 99))},
                        "stage_ms": {k: round(statistics.mean(s[k] for s in st2), 4) for k in st2[0]
                                     if statistics.mean(s[k] for s in st2) > 0},
                        "roofline": conv_roofline(d2, other, B, st2, pk, pk_src, args.model, fp8_peak),
                        "delta_affinity": delta_vs_oracle(got2, args.model, full_digest if B == 64 else None,
                                                          gold_digest, gold)}
        extra["fp8_peak_tflops"] = {"value": fp8_peak, "how": "torch._scaled_mm E4M3 8192^3, best of 10 "
                                                              "(with and without fast accumulation), this run"}

    # the paper's final architecture (Tables II, III, V) on the same batch: BF16 and FP8 throughput under the same
    # timing rules, |affinity difference| against its FP32 path
    if rank == 0 and args.model == MODEL and not args.no_extras and B == 64:
        extra["paper_final"] = paper_final_run(F, torch, batch, devb, B, stream, flush, args.steps, args.warmup,
                                               barrier)

    if rank == 0 and world == 1 and not args.no_serving and args.model == MODEL:
        extra["serving"] = serving_run(F, args.model, W, lambda dt: weights.to_blob(configs.model(args.model, dt), W),
                                       args.serving_requests)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    roof = conv_roofline(desc, args.dtype, B, stage_ms, pk, pk_src, args.model, fp8_peak)
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
                       "note": "per-pose latency = its batch's latency (all 64 poses finish together); "
                               "per-pose serving latency under load is in `serving`"},
        "stage_ms": {k: round(v, 4) for k, v in stage_mean.items() if v > 0},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": (launches_per_step(desc) + (len(desc["conv"]) if args.dtype == "fp8" else 0)) * args.steps,
        "clocks": clk,
        "affinity_std": float(np.std(got)),
    }
    if delta is not None:
        line["delta_affinity"] = delta
    if fp32_path is not None:
        line["fp32_path"] = fp32_path
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update(extra)
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
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-kernel-group rooflines, the other tensor-core dtype's run and the "
                         "paper-final model's run")
    ap.add_argument("--no-serving", action="store_true", help="skip the bounded serving measurement")
    ap.add_argument("--serving-requests", type=int, default=4000)
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
