"""The seeded generators: deterministic, within the stated ranges, and free of
atom pairs within 1e-5 A^2 of a squared edge cutoff; the uneven pools' pose
groups are one ligand moved rigidly (plus jitter) in one pocket, with ligand
and pocket sizes distributed as stated; the random-init weights follow the
stated bounds (restated from each tensor's shape) with uniform moments."""

import numpy as np
import pytest

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


def _kabsch_rmsd(a, b):
    """RMSD of b onto a after the best rigid superposition (Kabsch: SVD of the covariance)."""
    a = a - a.mean(axis=0)
    b = b - b.mean(axis=0)
    u, _, vt = np.linalg.svd(b.T @ a)
    d = np.sign(np.linalg.det(u @ vt))
    r = u @ np.diag([1.0, 1.0, d]) @ vt
    return float(np.sqrt(((b @ r - a) ** 2).sum(axis=1).mean()))


def test_pose_group_is_one_ligand_rigidly_moved_in_one_pocket():
    """The uneven pools' recipe: the n_rot poses of a group share the ligand size, the features and the pocket;
    each ligand is the same rigid body up to the per-atom jitter (about 0.5 A per axis: the RMSD between two
    poses after superposition is about 0.5 sqrt(3) sqrt(2) = 1.2 A), turned by a different rotation."""
    group = poses.make_pose_group(500123, 4)
    again = poses.make_pose_group(500123, 4)
    assert all(np.array_equal(p[0], q[0]) and np.array_equal(p[1], q[1]) for p, q in zip(group, again))
    n_lig = group[0][2]
    assert 8 <= n_lig <= 90 and 150 <= len(group[0][0]) - n_lig <= 1000
    lig0 = group[0][0][:n_lig].astype(np.float64)
    for xyz, feat, nl in group[1:]:
        assert nl == n_lig and np.array_equal(feat, group[0][1])
        # the pocket stays put (up to the 0.01 A nudges that clear near-cutoff pairs)
        assert np.abs(xyz[n_lig:] - group[0][0][n_lig:]).max() < 0.1
        lig = xyz[:n_lig].astype(np.float64)
        assert 0.6 < _kabsch_rmsd(lig0, lig) < 1.8
        # a different orientation: without superposition the ligands are far apart
        c = lig0.mean(axis=0) - lig.mean(axis=0)
        assert np.sqrt((((lig + c) - lig0) ** 2).sum(axis=1).mean()) > 2.0
        assert poses._near_cutoff_pairs(xyz) == []


def test_uneven_pool_size_distribution():
    """Ligand sizes log-normal around a median of 32 atoms (clipped to 8..90), pockets uniform in 150..1000."""
    pool = poses.make_uneven_pool(80, 1)
    n_lig = np.array([p[2] for p in pool])
    n_poc = np.array([len(p[0]) - p[2] for p in pool])
    assert n_lig.min() >= 8 and n_lig.max() <= 90
    assert 27 <= np.median(n_lig) <= 39
    assert 0.3 <= np.std(np.log(n_lig)) <= 0.6
    assert n_poc.min() >= 150 and n_poc.max() <= 1000
    assert 450 <= n_poc.mean() <= 700


def _expected_bound(name, W, desc):
    """The init rule of the weights module, restated from each tensor's shape: Kaiming-uniform sqrt(6 / fan_in)
    for ReLU layers (convs, CNN dense), U(+-1/sqrt(fan_in)) for biases, message transforms, gates, the gather
    and the last head layer, U(+-1/sqrt(H)) for the GRU, LeCun-uniform sqrt(3 / fan_in) for SELU head layers."""
    H = desc["sg_hidden"]
    if ".gru." in name:
        return 1.0 / np.sqrt(H)
    layer, kind = name.rsplit(".", 1)
    w = W[layer + ".w"] if kind == "b" else W[name]
    fan = int(np.prod(w.shape[1:]))
    if kind == "b":
        return 1.0 / np.sqrt(fan)
    if name.startswith("conv") or name == "cnn_dense.w":
        return np.sqrt(6.0 / fan)
    if name.startswith("head"):
        last = int(layer[4:]) == len(desc["head"]) - 1
        return 1.0 / np.sqrt(fan) if last else np.sqrt(3.0 / fan)
    return 1.0 / np.sqrt(fan)


def test_weight_init_bounds_and_moments():
    desc = configs.model("fusion-48grid-c64")
    W = weights.init_weights(desc, 0)
    names = [n for n, _s, _k, _f in weights.layout(desc)]
    assert sorted(names) == sorted(W)
    for name in names:
        w = W[name].astype(np.float64)
        b = _expected_bound(name, W, desc)
        assert np.abs(w).max() <= b * (1 + 1e-6), name
        if w.size >= 4096:   # enough draws to see the whole range and the uniform moments
            assert np.abs(w).max() >= 0.99 * b, name
            assert abs(w.mean()) < 0.05 * b, name
            assert w.var() == pytest.approx(b * b / 3.0, rel=0.05), name
