"""Mid-level and Late Fusion heads (Section 2.2) through the C ABI.

* small model (24^3 grid, one pose): the GPU affinity against the FP64 oracle's
  whole forward pass, FP32 within 1e-4, BF16 and FP8 within 0.05;
* full-size model (48^3 grid, 8 poses of the 64-pose workload, FP32 and BF16):
  the oracle head applied to the GPU's own CNN and SG latents (fetched stage
  outputs) against the GPU affinity, within 1e-4 of the affinity scale, so the
  head kernel is checked at the real widths (mid-level: a 576-wide first
  fusion layer and residual layers; late: two branch stacks) without the
  oracle's minute-long full-size CNN;
* a pose scores the same alone and in the batch.
"""

import numpy as np
import pytest

from gpu_common import F32_AFFINITY_TOL, require_gpu
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.mark.parametrize("form", ["mid", "late"])
@pytest.mark.parametrize("dtype,tol", [("f32", F32_AFFINITY_TOL), ("bf16", 0.05), ("fp8", 0.05)])
def test_small_model_against_oracle(F, form, dtype, tol):
    name = f"fusion-24grid-c32-{form}"
    W = weights.init_weights(configs.model(name), 0)
    desc = configs.model(name, dtype=dtype)
    batch = poses.make_batch(configs.WORKLOADS["pose1-lig24-pocket200"])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=1, max_atoms=512)
    got = float(m.score(batch)[0])
    m.close()
    exp = O.score_pose(configs.model(name), W, *poses.pose_slice(batch, 0))
    assert np.isfinite(got) and abs(got - exp) <= tol, (got, exp)


@pytest.mark.parametrize("form", ["mid", "late"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_full_size_head_on_gpu_latents(F, form, dtype):
    name = f"fusion-48grid-c64-{form}"
    W = weights.init_weights(configs.model(name), 1)
    desc = configs.model(name, dtype=dtype)
    batch = poses.subset(poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"]), list(range(8)))
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=1200, keep_stages=True)
    got = m.score(batch).copy()
    for p in range(8):
        cnn = m.fetch(F.STAGE_CNN_LATENT, p).astype(np.float64)
        sg = m.fetch(F.STAGE_SG_LATENT, p).astype(np.float64)
        exp = O.head(configs.model(name), W, cnn, sg)
        assert abs(float(got[p]) - exp) <= 1e-4 * max(1.0, abs(exp)), (p, got[p], exp)
    alone = m.score(poses.subset(batch, [5]))
    assert alone[0] == got[5]
    assert np.std(got) > 0.0
    m.close()
