"""GPU parity of the FP32 path against the FP64 oracle, through the C ABI.

* edges: bit-exact CSR (both sides evaluate the float32 edge rule);
* grid origin: bit-exact (float32 rule on both sides);
* voxel grid, conv maps, latents: FP32 rounding tolerances;
* affinity: <= 1e-4 absolute (the FP32 target);
at the small single-pose model, a ragged 20^3 model over a mixed batch (tiles
and a ragged tail), and the full-size model on the 64-pose batch (every pose
against stored oracle values, edges of every pose, grids of sampled poses).
"""

import numpy as np
import pytest

from gpu_common import F32_AFFINITY_TOL, golden, require_gpu, split_csr
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _edges_equal(F, m, p, xyz, cut_cov, cut_nc):
    g = O.radius_graph(xyz, cut_cov, cut_nc)
    n = len(xyz)
    for stage, name in ((F.STAGE_EDGES_COV, "cov"), (F.STAGE_EDGES_NC, "nc")):
        rp, col = split_csr(m.fetch(stage, p), n)
        np.testing.assert_array_equal(rp, g[name][0], err_msg=f"pose {p} {name} row_ptr")
        np.testing.assert_array_equal(col, g[name][1], err_msg=f"pose {p} {name} col")


def test_tiny_pose_all_stages(F):
    desc = configs.model("fusion-24grid-c32")
    W = weights.init_weights(desc, 0)
    batch = poses.make_batch(configs.WORKLOADS["pose1-lig24-pocket200"])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=512, keep_stages=True)
    got = m.score(batch)
    st = {}
    xyz, feat, n_lig = poses.pose_slice(batch, 0)
    exp = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
    np.testing.assert_array_equal(m.fetch(F.STAGE_ORIGIN, 0), st["origin"])
    G = m.fetch(F.STAGE_GRID, 0).reshape(st["grid"].shape)
    np.testing.assert_allclose(G, st["grid"], rtol=1e-5, atol=2e-6)
    for i in range(len(desc["conv"])):
        c = m.fetch(F.STAGE_CONV, (i << 16) | 0).reshape(st[f"conv{i}"].shape)
        np.testing.assert_allclose(c, st[f"conv{i}"], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(m.fetch(F.STAGE_POOL, 0).reshape(st["pool"].shape), st["pool"], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(m.fetch(F.STAGE_CNN_LATENT, 0), st["cnn_latent"], rtol=1e-4, atol=1e-5)
    _edges_equal(F, m, 0, xyz, desc["cut_cov"], desc["cut_nc"])
    np.testing.assert_allclose(m.fetch(F.STAGE_SG_STATE, 0).reshape(-1, 32), st["sg0.step1"], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(m.fetch(F.STAGE_SG_LATENT, 0), st["sg_latent"], rtol=1e-4, atol=1e-4)
    assert abs(float(got[0]) - exp) <= F32_AFFINITY_TOL, (got[0], exp)
    g = golden("tiny1_w0.json")
    assert g["input_digest"] == poses.digest(batch)
    assert abs(float(got[0]) - g["poses"]["0"]["affinity"]) <= F32_AFFINITY_TOL


def _ragged_batch():
    specs = [(101, (20, 30), (60, 120)), (102, (8, 12), (20, 40)), (103, (30, 40), (150, 200)),
             (104, (5, 5), (0, 0)), (105, (15, 25), (80, 100))]
    return poses.pack([poses.make_pose(s, a, b) for s, a, b in specs])


def test_ragged_model_mixed_batch(F):
    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 7)
    batch = _ragged_batch()
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512, keep_stages=True)
    got = m.score(batch)
    for p in range(len(batch["n_lig"])):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        st = {}
        exp = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
        G = m.fetch(F.STAGE_GRID, p).reshape(st["grid"].shape)
        np.testing.assert_allclose(G, st["grid"], rtol=1e-5, atol=2e-6, err_msg=f"grid pose {p}")
        for i in range(len(desc["conv"])):
            c = m.fetch(F.STAGE_CONV, (i << 16) | p).reshape(st[f"conv{i}"].shape)
            np.testing.assert_allclose(c, st[f"conv{i}"], rtol=1e-4, atol=1e-5, err_msg=f"conv{i} pose {p}")
        _edges_equal(F, m, p, xyz, desc["cut_cov"], desc["cut_nc"])
        np.testing.assert_allclose(m.fetch(F.STAGE_SG_LATENT, p), st["sg_latent"], rtol=1e-4, atol=1e-4)
        assert abs(float(got[p]) - exp) <= F32_AFFINITY_TOL, (p, got[p], exp)


def test_full_size_batch64_sampled(F):
    desc = configs.model("fusion-48grid-c64")
    W = weights.init_weights(desc, 0)
    batch = poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"])
    g = golden("full64_w0.json")
    assert g["input_digest"] == poses.digest(batch), "generated inputs differ from the stored ones"
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=64, max_atoms=1200)
    got = m.score(batch)
    assert np.all(np.isfinite(got))
    idx = [int(k) for k in g["poses"]]
    d_or = np.abs(got[idx] - np.array([g["poses"][str(i)]["affinity"] for i in idx]))
    print(f"f32 vs the FP64 oracle over {len(idx)} stored poses: mean |d| {d_or.mean():.2e}, max |d| {d_or.max():.2e}")
    for k, v in g["poses"].items():
        p = int(k)
        np.testing.assert_allclose(m.fetch(F.STAGE_CNN_LATENT, p), v["cnn_latent"], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(m.fetch(F.STAGE_SG_LATENT, p), v["sg_latent"], rtol=1e-4, atol=1e-4)
        assert abs(float(got[p]) - v["affinity"]) <= F32_AFFINITY_TOL, (p, got[p], v["affinity"])
    # every pose's edges, two poses' grids
    for p in range(64):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        _edges_equal(F, m, p, xyz, desc["cut_cov"], desc["cut_nc"])
    for p in (5, 50):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        o = O.grid_origin(xyz[:n_lig], 48, 1.0)
        np.testing.assert_array_equal(m.fetch(F.STAGE_ORIGIN, p), o)
        G = O.voxelize(xyz, feat, o, 48, 1.0, 1.0, 3)
        np.testing.assert_allclose(m.fetch(F.STAGE_GRID, p).reshape(G.shape), G, rtol=1e-5, atol=2e-6)
    # spread of the random-init affinities (the tolerance is meaningful only if O(0.1..10))
    assert 0.05 < float(np.std(got)) < 50.0


def test_pose_alone_equals_pose_in_batch(F):
    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 7)
    batch = _ragged_batch()
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512)
    full = m.score(batch).copy()
    for p in (0, 2, 4):
        alone = m.score(poses.subset(batch, [p]))
        assert alone[0] == full[p]
    rev = m.score(poses.subset(batch, [4, 3, 2, 1, 0]))
    np.testing.assert_array_equal(rev, full[::-1])


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_device_pointer_path_matches_host_path(F, dtype):
    """Device pointers: the atom count is read on the device and the kernels are launched for the capacity
    (the tensor-core graph kernels' persistent CTAs then skip the tiles past the count); scores equal the
    host path's bit for bit."""
    import torch
    desc = configs.model("fusion-20grid-ragged", dtype=dtype)
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 7)
    batch = _ragged_batch()
    stream = torch.cuda.current_stream()
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512, stream=stream.cuda_stream)
    host = m.score(batch).copy()
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in batch.items()}
    out = torch.empty(len(batch["n_lig"]), dtype=torch.float32, device="cuda")
    m.score(dev, out=out, on_device=True)
    np.testing.assert_array_equal(out.cpu().numpy(), host)
