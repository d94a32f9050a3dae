"""Parity-split inputs of the stride-2 tensor-core convolutions (FUSION_OPT_CONV_STRIDE2_SPLIT), through
the C ABI.

A stride-2 layer (Section 3.3.1, Table III) reads input voxel 2 o + p - pad for output o and kernel offset
p.  With the option on (the default) the previous layer's epilogue, or the FP8 quantizer, stores its map as
the 8 sub-grids of one coordinate parity, so each parity phase's halo is one plain TMA box; with it off
the layer reads NDHWC through the TMA element stride.  The halo in shared memory holds the same values in
both modes and the MMAs run in the same order, so every conv map and affinity must be bit-identical:
checked on the full-size model (conv3: 64 -> 128, 5^3, 48^3 in), the 20^3 model (conv2: 32 -> 64, 3^3,
20^3 in, ragged tiles) and the paper-final model (conv2: 32 -> 64, 3^3, 48^3 in), BF16 and FP8.  The
layers' values themselves are checked against float64 products of their own inputs in test_gpu_bf16.py and
test_gpu_fp8.py (layers in isolation), which run in the default mode.
"""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _run(F, m, batch, n_conv, n):
    aff = m.score(batch).copy()
    convs = [[m.fetch(F.STAGE_CONV, (i << 16) | p).copy() for i in range(n_conv)] for p in range(n)]
    return aff, convs


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("model,n", [("fusion-48grid-c64", 3), ("fusion-20grid-ragged", 5), ("fusion-paper-final", 2)])
def test_split_and_strided_inputs_match(F, dtype, model, n):
    desc = configs.model(model, dtype=dtype)
    W = weights.init_weights(configs.model(model), 0)
    batch = poses.subset(poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"]), list(range(n)))
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=n, max_atoms=1200, keep_stages=True)
    nc = len(desc["conv"])
    def tiles():   # the buffer layouts' byte rounding differs, the tile shapes do not
        return [{k: v for k, v in t.items() if k != "smem_bytes"} for t in m.conv_tiles()]
    t0 = tiles()
    split = _run(F, m, batch, nc, n)
    m.conv_stride2_split(0)
    assert tiles() == t0
    strided = _run(F, m, batch, nc, n)
    m.conv_stride2_split(-1)
    again = _run(F, m, batch, nc, n)
    m.close()
    for a, b in ((split, strided), (split, again)):
        np.testing.assert_array_equal(a[0], b[0])
        for p in range(n):
            for i in range(nc):
                np.testing.assert_array_equal(a[1][p][i], b[1][p][i], err_msg=f"pose {p} conv {i}")
    assert np.all(np.isfinite(split[0]))


def test_split_option_rejects_bad_values_and_fp32(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 0)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=1, max_atoms=1200)
    for bad in (2, -2):
        with pytest.raises(F.FusionError) as e:
            m.conv_stride2_split(bad)
        assert e.value.code == F.FUSION_EINVAL
    m.close()
    d32 = configs.model("fusion-20grid-ragged", dtype="f32")
    m32 = F.Model(d32, weights.to_blob(d32, W), max_poses=1, max_atoms=1200)
    with pytest.raises(F.FusionError) as e:
        m32.conv_stride2_split(0)
    assert e.value.code == F.FUSION_EUNSUPPORTED
    m32.close()
