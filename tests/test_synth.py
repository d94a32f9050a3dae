"""The seeded generators: deterministic, within the stated ranges, and free of
atom pairs within 1e-5 A^2 of a squared edge cutoff."""

import numpy as np

from synth import configs, poses, weights


def test_pose_is_deterministic_and_in_range():
    a = poses.make_pose(17, (20, 50), (300, 600))
    b = poses.make_pose(17, (20, 50), (300, 600))
    assert all(np.array_equal(x, y) for x, y in zip(a[:2], b[:2])) and a[2] == b[2]
    xyz, feat, n_lig = a
    assert 20 <= n_lig <= 50 and 300 <= len(xyz) - n_lig <= 600
    assert xyz.dtype == np.float32 and feat.shape == (len(xyz), 19)
    assert np.all(feat[:n_lig, 13] == 1.0) and np.all(feat[n_lig:, 13] == -1.0)
    # one element per atom
    assert np.all(feat[:, :9].sum(axis=1) == 1.0)


def test_tiny_pose_recipe():
    b = poses.make_batch(configs.WORKLOADS["pose1-lig24-pocket200"])
    assert b["atom_off"].tolist() == [0, 224] and b["n_lig"].tolist() == [24]
    xyz = b["xyz"].astype(np.float64)
    lig, poc = xyz[:24], xyz[24:]
    c = lig.mean(axis=0)
    r = np.linalg.norm(poc - c, axis=1)
    assert r.min() >= 4.0 - 1e-3 and r.max() <= 11.0 + 1e-3
    d = np.linalg.norm(xyz[:, None] - xyz[None], axis=2) + np.eye(224) * 100
    assert d.min() >= 1.2 - 0.02
    # ligand bonds
    dl = d[:24, :24]
    assert ((dl > 1.32) & (dl < 1.56)).sum() // 2 >= 24


def test_no_pairs_near_cutoffs():
    xyz, _, _ = poses.make_pose(3, (20, 50), (300, 600))
    assert poses._near_cutoff_pairs(xyz) == []


def test_blob_layout_size_and_order():
    d = configs.model("fusion-24grid-c32")
    W = weights.init_weights(d, 0)
    blob = weights.to_blob(d, W)
    assert len(blob) == weights.blob_size(d)
    first = np.frombuffer(blob[:4 * W["conv0.w"].size], dtype="<f4")
    assert np.array_equal(first, W["conv0.w"].reshape(-1))
    assert weights.cnn_out_shape(configs.model("fusion-48grid-c64")) == (128, 12)
