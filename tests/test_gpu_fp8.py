"""FP8 (E4M3) path: tcgen05 kind::f8f6f4 convolutions with per-output-channel
weight scales and per-pose activation scales, through the C ABI.

* affinity within 0.05 of the FP64 oracle on the small model, the 20^3
  stride-2 model over a mixed batch, and sampled poses of the full-size batch;
* against the FP32 path on all 64 poses of the full-size batch (<= 0.05);
* one conv layer in isolation: the GPU's bf16 input quantized on the host with
  the same per-pose rule (scale = max|x| / 448, E4M3 round to nearest even)
  and E4M3 weights with per-channel scales, convolved in float64;
* a pose scores the same alone and inside a batch (scales are per pose).
"""

import numpy as np
import pytest

from gpu_common import check_layer_fp8, golden, require_gpu
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu

FP8_AFFINITY_TOL = 0.05


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def test_tiny_fp8(F):
    desc = configs.model("fusion-24grid-c32", dtype="fp8")
    W = weights.init_weights(desc, 0)
    batch = poses.make_batch(configs.WORKLOADS["pose1-lig24-pocket200"])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=2, max_atoms=512, keep_stages=True)
    got = m.score(batch)
    xyz, feat, n_lig = poses.pose_slice(batch, 0)
    exp = O.score_pose(desc, W, xyz, feat, n_lig)
    n = desc["grid_n"]
    x = m.fetch(F.STAGE_GRID, 0).reshape(n, n, n, 19)
    y = m.fetch(F.STAGE_CONV, 0).reshape(n, n, n, 32)
    check_layer_fp8(x, W["conv0.w"], W["conv0.b"], desc["conv"][0], y)
    assert abs(float(got[0]) - exp) <= FP8_AFFINITY_TOL, (got[0], exp)


def test_ragged_fp8_and_batch_independence(F):
    desc = configs.model("fusion-20grid-ragged", dtype="fp8")
    W = weights.init_weights(desc, 7)
    specs = [(101, (20, 30), (60, 120)), (102, (8, 12), (20, 40)), (103, (30, 40), (150, 200)),
             (104, (5, 5), (0, 0)), (105, (15, 25), (80, 100))]
    batch = poses.pack([poses.make_pose(s, a, b) for s, a, b in specs])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512)
    got = m.score(batch).copy()
    for p in range(len(batch["n_lig"])):
        exp = O.score_pose(desc, W, *poses.pose_slice(batch, p))
        assert abs(float(got[p]) - exp) <= FP8_AFFINITY_TOL, (p, got[p], exp)
    alone = m.score(poses.subset(batch, [3]))
    assert alone[0] == got[3]


def test_full_size_fp8(F):
    desc = configs.model("fusion-48grid-c64", dtype="fp8")
    W = weights.init_weights(desc, 0)
    batch = poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"])
    g = golden("full64_w0.json")
    assert g["input_digest"] == poses.digest(batch)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=64, max_atoms=1200, keep_stages=True)
    got = m.score(batch).copy()
    idx = [int(k) for k in g["poses"]]
    d_or = np.abs(got[idx] - np.array([g["poses"][str(i)]["affinity"] for i in idx]))
    print(f"vs the FP64 oracle over {len(idx)} stored poses: mean |d| {d_or.mean():.2e}, max |d| {d_or.max():.2e}")
    for k, v in g["poses"].items():
        assert abs(float(got[int(k)]) - v["affinity"]) <= FP8_AFFINITY_TOL, (k, got[int(k)], v["affinity"])
    # the first residual layer of pose 7 in isolation
    x = m.fetch(F.STAGE_CONV, (0 << 16) | 7).reshape(48, 48, 48, 64)
    y = m.fetch(F.STAGE_CONV, (1 << 16) | 7).reshape(48, 48, 48, 64)
    check_layer_fp8(x, W["conv1.w"], W["conv1.b"], desc["conv"][1], y)
    d32 = configs.model("fusion-48grid-c64", dtype="f32")
    m32 = F.Model(d32, weights.to_blob(d32, W), max_poses=64, max_atoms=1200)
    ref32 = m32.score(batch)
    delta = np.abs(got - ref32)
    print(f"fp8 vs f32 over 64 poses: mean |d| {delta.mean():.4f}, max |d| {delta.max():.4f}")
    assert delta.max() <= FP8_AFFINITY_TOL
