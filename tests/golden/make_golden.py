"""Write stored oracle outputs for the parity tests.

Calls only ``oracle/`` (and the seeded input generators); nothing here comes
from the CUDA path.  The full-size model takes about a minute per pose in the
oracle, so the GPU tests compare sampled poses against these stored values
instead of re-running the oracle on the GPU host.

    python tests/golden/make_golden.py            # writes tests/golden/*.json
"""

from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fusion_oracle as O  # noqa: E402
from synth import configs, poses, weights  # noqa: E402

CASES = [
    # (file, model, weights seed, workload, sampled pose indices)
    ("full64_w0.json", "fusion-48grid-c64", 0, "batch64-lig20to50-pocket300to600", [0, 21, 42, 63]),
    ("tiny1_w0.json", "fusion-24grid-c32", 0, "pose1-lig24-pocket200", [0]),
    ("batch256_w0.json", "fusion-48grid-c64", 0, "batch256-lig15to60-pocket250to800", [0, 85, 170, 255]),
]


def make(fname, model, wseed, workload, idx):
    desc = configs.model(model)
    W = weights.init_weights(desc, wseed)
    batch = poses.make_batch(configs.WORKLOADS[workload])
    out = dict(model=model, weights_seed=wseed, workload=workload, input_digest=poses.digest(batch),
               poses={})
    for p in idx:
        t = time.time()
        st = {}
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        a = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
        out["poses"][str(p)] = dict(affinity=a, cnn_latent=st["cnn_latent"].tolist(),
                                    sg_latent=st["sg_latent"].tolist(),
                                    origin=[float(v) for v in st["origin"]])
        print(f"{fname} pose {p}: {a:.8f} ({time.time() - t:.1f} s)", flush=True)
    with open(os.path.join(HERE, fname), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    only = sys.argv[1:]
    for case in CASES:
        if only and case[0] not in only:
            continue
        make(*case)
