"""Precision on the 256-pose batch (ligands 15-60, pockets 250-800 atoms):
FP32, BF16 and FP8 affinities against the stored FP64 oracle values of 67
poses (every fourth pose and three more) within 1e-4 / 0.05 / 0.05, and
against the FP32 path on all 256 poses; the mean and max |d affinity| per
dtype are printed."""

import numpy as np
import pytest

from gpu_common import golden, require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


def test_bf16_fp8_against_fp64_oracle_and_fp32_path():
    F = require_gpu()
    batch = poses.make_batch(configs.WORKLOADS["batch256-lig15to60-pocket250to800"])
    g = golden("batch256_w0.json")
    assert g["input_digest"] == poses.digest(batch)
    W = weights.init_weights(configs.model("fusion-48grid-c64"), 0)
    res = {}
    for dt in ("f32", "bf16", "fp8"):
        desc = configs.model("fusion-48grid-c64", dtype=dt)
        m = F.Model(desc, weights.to_blob(desc, W), max_poses=256, max_atoms=1200)
        res[dt] = m.score(batch).copy()
        m.close()
    idx = [int(k) for k in g["poses"]]
    ref = np.array([g["poses"][str(i)]["affinity"] for i in idx])
    for dt, tol in (("f32", 1e-4), ("bf16", 0.05), ("fp8", 0.05)):
        d_or = np.abs(res[dt][idx] - ref)
        d_32 = np.abs(res[dt] - res["f32"])
        print(f"{dt}: vs FP64 oracle ({len(idx)} poses) mean {d_or.mean():.2e} max {d_or.max():.2e}; "
              f"vs FP32 path (256 poses) mean {d_32.mean():.2e} max {d_32.max():.2e}")
        assert d_or.max() <= tol
        assert d_32.max() <= max(tol, 1e-6)
