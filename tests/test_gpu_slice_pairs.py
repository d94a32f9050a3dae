"""Slice-paired tensor-core convolutions (two adjacent output slices per MMA,
N = 2 x output channels) against the one-slice-per-MMA form, through the C ABI.

Both forms sum every output element in the same order (the paired form adds
exact zeros for the offsets outside the kernel), so the conv layer outputs and
the affinities must be bit-identical, on the full-size model (stride-1 64-
channel layers and the stride-2 128-channel layer, forced paired too) and on
the 20^3 model with ragged z tails, for BF16 and FP8.
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
@pytest.mark.parametrize("model,workload,n", [
    ("fusion-48grid-c64", "batch64-lig20to50-pocket300to600", 6),
    ("fusion-20grid-ragged", "batch64-lig20to50-pocket300to600", 5),
])
def test_pairs_match_single_slices(F, dtype, model, workload, n):
    desc = configs.model(model, dtype=dtype)
    W = weights.init_weights(configs.model(model), 0)
    batch = poses.subset(poses.make_batch(configs.WORKLOADS[workload]), list(range(n)))
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=n, max_atoms=1200, keep_stages=True)
    res = {}
    for mode in (-1, 0, 1):
        m.conv_slice_pairs(mode)
        tiles = m.conv_tiles()
        if mode >= 0:
            assert all(t["slice_pairs"] == bool(mode) for t in tiles)
        else:
            assert [t["slice_pairs"] for t in tiles] == [
                cv["stride"] == 1 and cv["c_out"] <= 64 for cv in desc["conv"]]
        aff = m.score(batch).copy()
        convs = [m.fetch(F.STAGE_CONV, (i << 16) | (n - 1)).copy() for i in range(len(desc["conv"]))]
        res[mode] = (aff, convs)
    m.close()
    for mode in (0, 1):
        np.testing.assert_array_equal(res[mode][0], res[-1][0])
        for a, b in zip(res[mode][1], res[-1][1]):
            np.testing.assert_array_equal(a, b)
    assert np.all(np.isfinite(res[-1][0]))


def test_pair_option_rejects_bad_values_and_fp32(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    m = F.Model(desc, weights.to_blob(desc, weights.init_weights(configs.model("fusion-20grid-ragged"), 0)),
                max_poses=1, max_atoms=1200)
    with pytest.raises(F.FusionError) as e:
        m.conv_slice_pairs(2)
    assert e.value.code == F.FUSION_EINVAL
    m.close()
    d32 = configs.model("fusion-20grid-ragged", dtype="f32")
    m = F.Model(d32, weights.to_blob(d32, weights.init_weights(configs.model("fusion-20grid-ragged"), 0)),
                max_poses=1, max_atoms=1200)
    with pytest.raises(F.FusionError) as e:
        m.conv_slice_pairs(1)
    assert e.value.code == F.FUSION_EUNSUPPORTED
    m.close()
