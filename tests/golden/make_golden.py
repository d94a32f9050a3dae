"""Write stored oracle outputs for the parity tests.

Calls only ``oracle/`` (and the seeded input generators); nothing here comes
from the CUDA path.  The full-size model takes one to two minutes per pose in
the oracle on one core, so the GPU tests compare against these stored values
instead of re-running the oracle on the GPU host.  Poses are scored in a pool
of worker processes (one numpy thread each); the values do not depend on the
pool, since each pose is scored alone.

    python tests/golden/make_golden.py [file ...] [--workers N]   # writes tests/golden/*.json
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

CASES = [
    # (file, model, weights seed, workload, sampled pose indices)
    ("full64_w0.json", "fusion-48grid-c64", 0, "batch64-lig20to50-pocket300to600", list(range(64))),
    ("tiny1_w0.json", "fusion-24grid-c32", 0, "pose1-lig24-pocket200", [0]),
    ("batch256_w0.json", "fusion-48grid-c64", 0, "batch256-lig15to60-pocket250to800",
     sorted(set(range(0, 256, 4)) | {85, 170, 255})),
]


def _score(args):
    model, wseed, workload, p = args
    sys.path.insert(0, ROOT)
    from oracle import fusion_oracle as O
    from synth import configs, poses, weights
    desc = configs.model(model)
    W = weights.init_weights(desc, wseed)
    batch = poses.make_batch(configs.WORKLOADS[workload])
    t = time.time()
    st = {}
    xyz, feat, n_lig = poses.pose_slice(batch, p)
    a = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
    return p, dict(affinity=a, cnn_latent=st["cnn_latent"].tolist(), sg_latent=st["sg_latent"].tolist(),
                   origin=[float(v) for v in st["origin"]]), time.time() - t


def _write(path, head, per_pose):
    """One pose per line, so the files diff pose by pose."""
    lines = ["{"]
    for k, v in head.items():
        lines.append(f" {json.dumps(k)}: {json.dumps(v)},")
    lines.append(' "poses": {')
    keys = sorted(per_pose, key=int)
    for i, k in enumerate(keys):
        sep = "," if i + 1 < len(keys) else ""
        lines.append(f"  {json.dumps(str(k))}: {json.dumps(per_pose[k], separators=(',', ':'))}{sep}")
    lines.append(" }")
    lines.append("}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def make(pool, fname, model, wseed, workload, idx):
    sys.path.insert(0, ROOT)
    from synth import configs, poses
    batch = poses.make_batch(configs.WORKLOADS[workload])
    head = dict(model=model, weights_seed=wseed, workload=workload, input_digest=poses.digest(batch))
    out = {}
    for p, rec, dt in pool.imap_unordered(_score, [(model, wseed, workload, p) for p in idx]):
        out[p] = rec
        print(f"{fname} pose {p}: {rec['affinity']:.8f} ({dt:.1f} s, {len(out)}/{len(idx)})", flush=True)
    _write(os.path.join(HERE, fname), head, out)


if __name__ == "__main__":
    args = sys.argv[1:]
    workers = max(1, (os.cpu_count() or 2) - 2)
    if "--workers" in args:
        i = args.index("--workers")
        workers = int(args[i + 1])
        del args[i:i + 2]
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(workers) as pool:
        for case in CASES:
            if args and case[0] not in args:
                continue
            make(pool, *case)
