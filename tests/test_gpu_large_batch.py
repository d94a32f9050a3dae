"""A 512-pose call of the full-size model through the C ABI.

The persistent convolutions run one CTA per SM over all tiles of the call, so
at 512 poses each CTA processes about 364 tiles (55,296 tiles of the
residual layers): the tile loop, the per-tile deadlines and the barrier phases
must hold over that many tiles.  The affinities of the 512-pose call must equal,
bit for bit, those of the same poses scored 64 at a time (BF16 and FP8), and
all be finite.
"""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_512_poses_equal_64_pose_calls(F, dtype):
    wl = dict(configs.WORKLOADS["batch64-lig20to50-pocket300to600"])
    wl["seeds"] = list(range(3001, 3513))
    batch = poses.make_batch(wl)
    desc = configs.model("fusion-48grid-c64", dtype=dtype)
    blob = weights.to_blob(desc, weights.init_weights(configs.model("fusion-48grid-c64"), 0))
    big = F.Model(desc, blob, max_poses=512, max_atoms=1200)
    got = big.score(batch).copy()
    big.close()
    small = F.Model(desc, blob, max_poses=64, max_atoms=1200)
    ref = np.concatenate([small.score(poses.subset(batch, list(range(i, i + 64)))) for i in range(0, 512, 64)])
    small.close()
    assert np.all(np.isfinite(got))
    np.testing.assert_array_equal(got, ref)
