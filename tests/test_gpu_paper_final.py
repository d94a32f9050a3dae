"""The paper-final architecture (Tables II, III and V) through the C ABI.

The `fusion-paper-final` preset: 3D-CNN 19->32 5^3, residual 32 5^3, 32->64 3^3 stride 2, residual 64 3^3
(the 24^3 layer after the stride-2 one reads its input channel-blocked, as the stride-2 layer's epilogue
writes it), dense 128; SG-CNN with 6 covalent then 3 mixed gated steps, covalent cutoff 2.24 A and
non-covalent 5.22 A; head 128 -> 64 -> 24 -> 1.  Four poses of the 64-pose workload, weights seed 1
(affinity spread 0.53):

* FP32: every edge list bit-exact, affinities of two poses within 1e-4 of the FP64 oracle;
* BF16 and FP8: each conv layer of a pose in isolation (the GPU's own input map convolved in float64),
  affinity within 0.05 of the oracle, and a pose alone scores as in the batch.
"""

import numpy as np
import pytest

from gpu_common import (F32_AFFINITY_TOL, check_layer_bf16, check_layer_fp8, layers_in_isolation, require_gpu,
                        split_csr)
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu

NAME = "fusion-paper-final"


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.fixture(scope="module")
def case():
    batch = poses.subset(poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"]), [0, 1, 2, 3])
    W = weights.init_weights(configs.model(NAME), 1)
    exp = [O.score_pose(configs.model(NAME), W, *poses.pose_slice(batch, p)) for p in (0, 1)]
    return batch, W, exp


def test_paper_final_f32(F, case):
    batch, W, exp = case
    desc = configs.model(NAME, dtype="f32")
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=1200, keep_stages=True)
    got = m.score(batch).copy()
    for p in range(4):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        g = O.radius_graph(xyz, desc["cut_cov"], desc["cut_nc"])
        for stage, name in ((F.STAGE_EDGES_COV, "cov"), (F.STAGE_EDGES_NC, "nc")):
            rp, col = split_csr(m.fetch(stage, p), len(xyz))
            np.testing.assert_array_equal(rp, g[name][0], err_msg=f"pose {p} {name} row_ptr")
            np.testing.assert_array_equal(col, g[name][1], err_msg=f"pose {p} {name} col")
    m.close()
    for p in (0, 1):
        assert abs(float(got[p]) - exp[p]) <= F32_AFFINITY_TOL, (p, got[p], exp[p])


@pytest.mark.parametrize("dtype,check", [("bf16", check_layer_bf16), ("fp8", check_layer_fp8)])
def test_paper_final_tensor_cores(F, case, dtype, check):
    batch, W, exp = case
    desc = configs.model(NAME, dtype=dtype)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=1200, keep_stages=True)
    got = m.score(batch).copy()
    layers_in_isolation(F, m, desc, W, 0, check)
    alone = m.score(poses.subset(batch, [2]))[0]
    m.close()
    for p in (0, 1):
        assert np.isfinite(got[p]) and abs(float(got[p]) - exp[p]) <= 0.05, (p, got[p], exp[p])
    assert alone == got[2]
