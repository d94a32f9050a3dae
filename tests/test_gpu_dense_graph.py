"""Radius graph on a pose far denser than a protein, through the C ABI.

400 atoms drawn uniformly in a 7 A cube (1.17 atoms per cubic A, about 13x a
protein's density): 175 non-covalent neighbours within 4.5 A per atom on
average and up to 328, 16 covalent ones within 1.6 A on average and up to 32.
Rows longer than 128 take the fill pass's single-lane sort, shorter ones the
warp's rank sort; the cell list collapses to a few cells.  Both edge lists must
equal the oracle's bit for bit (the float32 edge rule on both sides), on the
20^3 model with max_degree 1024 (capacity N x 1024 holds the ~76,000 edges).
A second pose of the same batch, built by the usual generator, must keep its
own edges too.
"""

import numpy as np
import pytest

from gpu_common import require_gpu, split_csr
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _dense_pose(seed, n=400, side=7.0):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, side, (n, 3)).astype(np.float32)
    feat = (rng.random((n, 19)) * (rng.random((n, 19)) < 0.3)).astype(np.float32)
    return xyz, feat, 40


def test_dense_pose_edges_bit_exact(F):
    desc = configs.model("fusion-20grid-ragged", dtype="f32")
    dense = _dense_pose(91)
    normal = poses.make_pose(92, (20, 30), (100, 150))
    batch = poses.pack([dense, normal])
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 3)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=2, max_atoms=512, max_degree=1024, keep_stages=True)
    m.score(batch)
    longest = 0
    for p in range(2):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        g = O.radius_graph(xyz, desc["cut_cov"], desc["cut_nc"])
        for stage, name in ((F.STAGE_EDGES_COV, "cov"), (F.STAGE_EDGES_NC, "nc")):
            rp, col = split_csr(m.fetch(stage, p), len(xyz))
            np.testing.assert_array_equal(rp, g[name][0], err_msg=f"pose {p} {name} row_ptr")
            np.testing.assert_array_equal(col, g[name][1], err_msg=f"pose {p} {name} col")
            longest = max(longest, int(np.diff(rp).max()))
    m.close()
    assert longest > 128, longest      # the long-row sort ran
