"""The dense layer entry point that allocates nothing (fixed library scratch)
must give the same result as the dense layer inside fusion_score.

It serves callers that cannot allocate device memory: code that runs under a
device-memory budget owned by someone else, or a request loop that cannot take
the synchronisation and latency of cudaMalloc / cudaFree.  The test scores two
different batches with fusion_score, feeds each batch's pooled CNN map to the
no-allocation entry point in two calls in a row, and compares with the dense
output fusion_score produced.  It builds everything it needs, so it passes in a
fresh process as well as after the other tests.
"""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


def _dense_weights_dhwc(desc, W):
    """The blob's dense matrix with its input reordered from (C, D, H, W) to (D, H, W, C)."""
    from synth.weights import cnn_out_shape
    c, n = cnn_out_shape(desc)
    w = W["cnn_dense.w"].reshape(-1, c, n * n * n)
    return np.ascontiguousarray(w.transpose(0, 2, 1).reshape(w.shape[0], -1))


def test_dense_noalloc_matches_fusion_score_dense():
    F = require_gpu()
    import torch

    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 11)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=256)
    wd = torch.from_numpy(_dense_weights_dhwc(desc, W)).cuda()
    bias = torch.from_numpy(W["cnn_dense.b"]).cuda()
    N, K = wd.shape
    batches = [poses.pack([poses.make_pose(s, (10, 25), (40, 90)) for s in (21, 22, 23, 24, 25)]),
               poses.pack([poses.make_pose(s, (12, 30), (50, 100)) for s in (31, 32, 33)])]
    stream = torch.cuda.current_stream()
    for batch in batches:
        B = len(batch["n_lig"])
        m.score(batch)
        pooled = np.stack([m.fetch(F.STAGE_POOL, p) for p in range(B)])
        expect = np.stack([m.fetch(F.STAGE_CNN_LATENT, p) for p in range(B)])
        x = torch.from_numpy(pooled).cuda()
        y = torch.full((B, N), float("nan"), device="cuda")
        F.fusion_cnn_dense_noalloc(x, wd, bias, B, N, K, True, y, stream.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_allclose(y.cpu().numpy(), expect, rtol=1e-5, atol=1e-5)
    m.close()


def test_dense_noalloc_rejects_sizes_beyond_its_scratch():
    F = require_gpu()
    import torch

    x = torch.zeros(8, device="cuda")
    K = 221184                                  # 108 splits
    B, N = 64, 512                              # 108 * 64 * 512 partials > 2^21
    with pytest.raises(F.FusionError) as e:
        F.fusion_cnn_dense_noalloc(x, x, x, B, N, K, True, x)
    assert e.value.code == F.FUSION_EINVAL and "scratch" in str(e.value)
