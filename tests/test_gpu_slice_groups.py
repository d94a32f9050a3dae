"""Slice-grouped tensor-core convolutions (one MMA serving 1, 2, 4 or 8 adjacent
output slices, N = slices x output channels) against each other, through the
C ABI.

Every grouping adds each output element's terms in the same order (kernel
offset groups in (ty, tx) order, z offset ascending), so the conv layer outputs
and the affinities must be bit-identical across groupings: on the full-size
model (stride-1 64-channel layers with up to 4 slices per MMA, the stride-2
128-channel layer with up to 2), on the 20^3 model (32-channel layers,
ragged z tails, a stride-2 layer with one z offset in some phases) and on the
paper-final model (32-channel layers at 16 slices per CTA, up to 8 per MMA),
for BF16 and FP8.  Where a grouping does not fit a layer, the option must fail with
FUSION_EUNSUPPORTED and leave the previous plans in place.
"""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _fits(cv, T, G):
    # 8 slices per MMA only with 16 slices per CTA (two slice groups, two MMA issuers)
    return T % G == 0 and G * cv["c_out"] <= 256 and (G != 8 or T // G >= 2)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("model,n", [("fusion-48grid-c64", 6), ("fusion-20grid-ragged", 5), ("fusion-paper-final", 2)])
def test_slice_groups_match(F, dtype, model, n):
    desc = configs.model(model, dtype=dtype)
    W = weights.init_weights(configs.model(model), 0)
    batch = poses.subset(poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"]), list(range(n)))
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=n, max_atoms=1200, keep_stages=True)
    res = {}
    for mode in (-1, 1, 2, 4, 8):
        tiles = m.conv_tiles()
        fits = all(_fits(cv, t["slices_per_cta"], mode) for cv, t in zip(desc["conv"], tiles)) if mode > 0 else True
        if not fits:
            before = [t["slices_per_mma"] for t in tiles]
            with pytest.raises(F.FusionError) as e:
                m.conv_slices_per_mma(mode)
            assert e.value.code == F.FUSION_EUNSUPPORTED
            assert [t["slices_per_mma"] for t in m.conv_tiles()] == before
            continue
        m.conv_slices_per_mma(mode)
        tiles = m.conv_tiles()
        if mode > 0:
            assert all(t["slices_per_mma"] == mode for t in tiles)
        else:
            for cv, t in zip(desc["conv"], tiles):
                T = t["slices_per_cta"]
                want = 1 if cv["stride"] != 1 else 8 if T == 16 and _fits(cv, T, 8) else \
                    max(G for G in (1, 2, 4) if _fits(cv, T, G))
                assert t["slices_per_mma"] == want
        aff = m.score(batch).copy()
        convs = [m.fetch(F.STAGE_CONV, (i << 16) | (n - 1)).copy() for i in range(len(desc["conv"]))]
        res[mode] = (aff, convs)
    m.close()
    assert len(res) >= 3
    for mode in res:
        np.testing.assert_array_equal(res[mode][0], res[-1][0])
        for a, b in zip(res[mode][1], res[-1][1]):
            np.testing.assert_array_equal(a, b)
    assert np.all(np.isfinite(res[-1][0]))


def test_slice_group_option_rejects_bad_values_and_fp32(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 0)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=1, max_atoms=1200)
    for bad in (0, 3, 16):
        with pytest.raises(F.FusionError) as e:
            m.conv_slices_per_mma(bad)
        assert e.value.code == F.FUSION_EINVAL
    # 8 slices per MMA needs 16 slices per CTA (32-channel layers whose z extent suits it): not this model,
    # whose layers keep their plans
    before = m.conv_tiles()
    with pytest.raises(F.FusionError) as e:
        m.conv_slices_per_mma(8)
    assert e.value.code == F.FUSION_EUNSUPPORTED
    assert m.conv_tiles() == before
    m.close()
    d32 = configs.model("fusion-20grid-ragged", dtype="f32")
    m = F.Model(d32, weights.to_blob(d32, W), max_poses=1, max_atoms=1200)
    with pytest.raises(F.FusionError) as e:
        m.conv_slices_per_mma(1)
    assert e.value.code == F.FUSION_EUNSUPPORTED
    m.close()
