"""A pose at the atom capacity (max_atoms = 4096) through the C ABI.

One pose: a 60-atom ligand from the generator plus 4036 further atoms drawn
uniformly in a 36 A cube around it (0.087 atoms per cubic A, the density of a
protein), features drawn at random.  On the 20^3 model, FP32 and BF16: the
covalent and non-covalent edge lists must equal the oracle's bit for bit, and
the affinity must be within 1e-4 (FP32) / 0.05 (BF16) of the FP64 oracle.  The
cell lists, the per-atom edge capacity, the graph steps over 4096 nodes and the
voxelization of atoms far outside the grid all run at their largest sizes.
"""

import numpy as np
import pytest

from gpu_common import F32_AFFINITY_TOL, require_gpu, split_csr
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu

N_MAX = 4096


def _big_pose():
    xyz_l, feat_l, n_lig = poses.make_pose(77, (60, 60), (0, 0))
    rng = np.random.default_rng(78)
    n_p = N_MAX - n_lig
    c = xyz_l.mean(axis=0)
    xyz_p = (c + rng.uniform(-18.0, 18.0, (n_p, 3))).astype(np.float32)
    feat_p = (rng.random((n_p, 19)) * (rng.random((n_p, 19)) < 0.3)).astype(np.float32)
    return (np.concatenate([xyz_l, xyz_p]).astype(np.float32), np.concatenate([feat_l, feat_p]).astype(np.float32),
            n_lig)


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.fixture(scope="module")
def case():
    xyz, feat, n_lig = _big_pose()
    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 13)
    st = {}
    exp = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
    return xyz, feat, n_lig, W, exp, st["graph"]


@pytest.mark.parametrize("dtype,tol", [("f32", F32_AFFINITY_TOL), ("bf16", 0.05)])
def test_pose_at_atom_capacity(F, case, dtype, tol):
    xyz, feat, n_lig, W, exp, graph = case
    assert len(xyz) == N_MAX
    desc = configs.model("fusion-20grid-ragged", dtype=dtype)
    batch = poses.pack([(xyz, feat, n_lig)])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=1, max_atoms=N_MAX, max_degree=64, keep_stages=True)
    got = float(m.score(batch)[0])
    for stage, name in ((F.STAGE_EDGES_COV, "cov"), (F.STAGE_EDGES_NC, "nc")):
        rp, col = split_csr(m.fetch(stage, 0), N_MAX)
        np.testing.assert_array_equal(rp, graph[name][0], err_msg=f"{name} row_ptr")
        np.testing.assert_array_equal(col, graph[name][1], err_msg=f"{name} col")
    m.close()
    assert np.isfinite(got) and abs(got - exp) <= tol, (got, exp)
