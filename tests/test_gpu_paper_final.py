"""The paper-final architecture (Tables II, III and V) through the C ABI.

The `fusion-paper-final` preset: 3D-CNN 19->32 5^3, residual 32 5^3, 32->64 3^3 stride 2, residual 64 3^3
(the 24^3 layer after the stride-2 one reads its input channel-blocked, as the stride-2 layer's epilogue
writes it), dense 128 then 64 (the CNN latent); SG-CNN with 6 covalent steps at the 19 feature channels,
the gate to the covalent gather width 24, then 3 mixed steps at width 24 (covalent cutoff 2.24 A,
non-covalent 5.22 A), gated gather to 128; head 128 -> 64 -> 24 -> 1.  The graph kernels carry both stages
at width 32 with the extra channels held at zero.  Four poses of the 64-pose workload, weights seed 1:

* FP32: every edge list bit-exact; the CNN latent (second dense layer), the SG latent and the affinities
  of two poses against the FP64 oracle (1e-4); the last node states equal the oracle's 24 channels and
  hold exact zeros in the padding channels;
* BF16 and FP8: each conv layer of a pose in isolation (the GPU's own input map convolved in float64),
  affinity within 0.05 of the oracle, and a pose alone scores as in the batch;
* the Late and Mid-level Fusion forms on the same branches (the SG-CNN's own 128 -> 85 -> 42 -> 1 stack
  in Late Fusion): FP32 affinities against the oracle head on the oracle's latents (1e-4), BF16 within 0.05.
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
    stages = []
    for p in (0, 1):
        st = {}
        O.score_pose(configs.model(NAME), W, *poses.pose_slice(batch, p), stages=st)
        stages.append(st)
    return batch, W, stages


def test_paper_final_f32(F, case):
    batch, W, stages = case
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
    for p in (0, 1):
        st = stages[p]
        cnn = m.fetch(F.STAGE_CNN_LATENT, p)
        assert cnn.shape == (64,)
        np.testing.assert_allclose(cnn, st["cnn_latent"], rtol=1e-4, atol=1e-5)
        np.testing.assert_allclose(m.fetch(F.STAGE_SG_LATENT, p), st["sg_latent"], rtol=1e-4, atol=1e-4)
        h = m.fetch(F.STAGE_SG_STATE, p).reshape(-1, 32)
        np.testing.assert_allclose(h[:, :24], st["sg1.step2"], rtol=1e-4, atol=1e-5)
        assert np.all(h[:, 24:] == 0.0)
        assert abs(float(got[p]) - st["affinity"]) <= F32_AFFINITY_TOL, (p, got[p], st["affinity"])
    m.close()


@pytest.mark.parametrize("dtype,check", [("bf16", check_layer_bf16), ("fp8", check_layer_fp8)])
def test_paper_final_tensor_cores(F, case, dtype, check):
    batch, W, stages = case
    desc = configs.model(NAME, dtype=dtype)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=1200, keep_stages=True)
    got = m.score(batch).copy()
    layers_in_isolation(F, m, desc, W, 0, check)
    alone = m.score(poses.subset(batch, [2]))[0]
    m.close()
    for p in (0, 1):
        exp = stages[p]["affinity"]
        assert np.isfinite(got[p]) and abs(float(got[p]) - exp) <= 0.05, (p, got[p], exp)
    assert alone == got[2]


@pytest.mark.parametrize("form", ["late", "mid"])
@pytest.mark.parametrize("dtype,tol", [("f32", F32_AFFINITY_TOL), ("bf16", 0.05)])
def test_paper_final_fusion_forms(F, case, form, dtype, tol):
    """The forms share the branches' weights (the same seed draws the same branch tensors first), so the
    oracle's latents of the coherent model serve; the form's own head is the oracle's."""
    batch, _, stages = case
    name = f"{NAME}-{form}"
    W = weights.init_weights(configs.model(name), 1)
    desc = configs.model(name, dtype=dtype)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=1200)
    got = m.score(batch).copy()
    alone = m.score(poses.subset(batch, [1]))[0]
    m.close()
    for p in (0, 1):
        exp = O.head(configs.model(name), W, stages[p]["cnn_latent"], stages[p]["sg_latent"])
        assert np.isfinite(got[p]) and abs(float(got[p]) - exp) <= tol, (form, dtype, p, got[p], exp)
    assert alone == got[1]
