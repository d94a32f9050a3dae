"""BF16 path (tcgen05 tensor-core convolutions) through the C ABI.

* each conv layer in isolation: the GPU's own bf16 input map and bf16-rounded
  weights, convolved in float64 on the CPU, must match the GPU layer output up
  to the output's bf16 rounding (plus FP32 accumulation);
* edges stay bit-exact and the grid matches the oracle to bf16 rounding;
* affinity within 0.05 of the FP64 oracle (the BF16 target), on the small
  model, a 20^3 model with a stride-2 layer over a mixed batch, and sampled
  poses of the full-size 64-pose batch;
* a pose scores the same alone and inside a batch.
"""

import numpy as np
import pytest

from gpu_common import check_layer_bf16, golden, layers_in_isolation, require_gpu, split_csr
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu

BF16_AFFINITY_TOL = 0.05


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _layers_in_isolation(F, m, desc, W, p, layers=None):
    layers_in_isolation(F, m, desc, W, p, check_layer_bf16, layers)


def test_tiny_bf16(F):
    desc = configs.model("fusion-24grid-c32", dtype="bf16")
    W = weights.init_weights(desc, 0)
    batch = poses.make_batch(configs.WORKLOADS["pose1-lig24-pocket200"])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=2, max_atoms=512, keep_stages=True)
    got = m.score(batch)
    xyz, feat, n_lig = poses.pose_slice(batch, 0)
    st = {}
    exp = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
    G = m.fetch(F.STAGE_GRID, 0).reshape(st["grid"].shape)
    np.testing.assert_allclose(G, st["grid"], rtol=8e-3, atol=1e-6)
    _layers_in_isolation(F, m, desc, W, 0)
    assert abs(float(got[0]) - exp) <= BF16_AFFINITY_TOL, (got[0], exp)


def _ragged_batch():
    specs = [(101, (20, 30), (60, 120)), (102, (8, 12), (20, 40)), (103, (30, 40), (150, 200)),
             (104, (5, 5), (0, 0)), (105, (15, 25), (80, 100))]
    return poses.pack([poses.make_pose(s, a, b) for s, a, b in specs])


def test_ragged_bf16_stride2(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(desc, 7)
    batch = _ragged_batch()
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512, keep_stages=True)
    got = m.score(batch)
    for p in range(len(batch["n_lig"])):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        _layers_in_isolation(F, m, desc, W, p)
        g = O.radius_graph(xyz, 1.6, 4.5)
        rp, col = split_csr(m.fetch(F.STAGE_EDGES_NC, p), len(xyz))
        np.testing.assert_array_equal(col, g["nc"][1])
        exp = O.score_pose(desc, W, xyz, feat, n_lig)
        assert abs(float(got[p]) - exp) <= BF16_AFFINITY_TOL, (p, got[p], exp)
    alone = m.score(poses.subset(batch, [2]))
    assert alone[0] == got[2]


def test_full_size_bf16(F):
    desc = configs.model("fusion-48grid-c64", dtype="bf16")
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
        assert abs(float(got[int(k)]) - v["affinity"]) <= BF16_AFFINITY_TOL, (k, got[int(k)], v["affinity"])
    # the residual 7^3 layer and the stride-2 layer of one pose, in isolation
    _layers_in_isolation(F, m, desc, W, 0, layers={1, 3})
    # against the FP32 path on all 64 poses
    d32 = configs.model("fusion-48grid-c64", dtype="f32")
    m32 = F.Model(d32, weights.to_blob(d32, W), max_poses=64, max_atoms=1200)
    ref32 = m32.score(batch)
    delta = np.abs(got - ref32)
    print(f"bf16 vs f32 over 64 poses: mean |d| {delta.mean():.4f}, max |d| {delta.max():.4f}")
    assert delta.max() <= BF16_AFFINITY_TOL
