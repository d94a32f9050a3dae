"""The dense layer entry point that allocates nothing (fixed library scratch)
must give the dense layer's result: against the dense layer inside
fusion_score, and against a float64 product computed on the host.

It serves callers that cannot allocate device memory: code that runs under a
device-memory budget owned by someone else, or a request loop that cannot take
the synchronisation and latency of cudaMalloc / cudaFree.  The first test
scores two different batches with fusion_score, feeds each batch's pooled CNN
map to the no-allocation entry point in two calls in a row, and compares with
the dense output fusion_score produced and with x @ W.T + b in float64.  The
second covers sizes that cross the kernel's 64-row pose and output tiles, many
K splits with an empty last split, and no activation.  Every test builds what
it needs, so the file passes in a fresh process as well as after the other
tests.
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


def _host_dense(x, w, b, relu):
    """float64 y = act(x W^T + b) on the host."""
    y = np.asarray(x, np.float64) @ np.asarray(w, np.float64).T + np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def _assert_close(got, ref):
    """FP32 split-K sums against float64: 1e-5 relative plus 1e-5 of the largest |output|."""
    scale = float(np.abs(ref).max()) + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= 1e-5 * np.abs(ref) + 1e-5 * scale), (float(err.max()), scale)


def test_dense_noalloc_matches_fusion_score_dense():
    F = require_gpu()
    import torch

    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 11)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=256)
    wd_h = _dense_weights_dhwc(desc, W)
    wd = torch.from_numpy(wd_h).cuda()
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
        got = y.cpu().numpy()
        np.testing.assert_allclose(got, expect, rtol=1e-5, atol=1e-5)
        _assert_close(got, _host_dense(pooled, wd_h, W["cnn_dense.b"], True))
    m.close()


@pytest.mark.parametrize("B,N,K,relu", [
    (65, 70, 8000, False),        # one pose row and six outputs past a 64-row tile, 3 splits, no activation
    (3, 129, 262152, True),       # 128 splits; the last split's K range is empty (2080 x 127 > K)
    (130, 1, 2048, False),        # one split, one output, three pose tiles
])
def test_dense_noalloc_sizes_against_float64(B, N, K, relu):
    F = require_gpu()
    import torch

    rng = np.random.default_rng(B * 1000 + N)
    x = rng.uniform(0.0, 1.0, (B, K)).astype(np.float32)
    w = rng.uniform(-1.0, 1.0, (N, K)).astype(np.float32) / np.float32(np.sqrt(K))
    b = rng.uniform(-0.5, 0.5, N).astype(np.float32)
    xd, wd, bd = (torch.from_numpy(a).cuda() for a in (x, w, b))
    ref = _host_dense(x, w, b, relu)
    for _ in range(2):                                   # two calls in a row share the scratch
        y = torch.full((B, N), float("nan"), device="cuda")
        F.fusion_cnn_dense_noalloc(xd, wd, bd, B, N, K, relu, y)
        torch.cuda.synchronize()
        _assert_close(y.cpu().numpy(), ref)


def test_dense_noalloc_rejects_sizes_beyond_its_scratch():
    F = require_gpu()
    import torch

    x = torch.zeros(8, device="cuda")
    K = 221184                                  # 108 splits
    B, N = 64, 512                              # 108 * 64 * 512 partials > 2^21
    with pytest.raises(F.FusionError) as e:
        F.fusion_cnn_dense_noalloc(x, x, x, B, N, K, True, x)
    assert e.value.code == F.FUSION_EINVAL and "scratch" in str(e.value)


def test_dense_noalloc_rejects_misaligned_operands():
    """An offset view of x or w (not 16-byte aligned) is refused on the host; nothing is launched."""
    F = require_gpu()
    import torch

    B, N, K = 2, 4, 64
    buf = torch.zeros(B * K + 1, device="cuda")
    w = torch.zeros(N * K, device="cuda")
    b = torch.zeros(N, device="cuda")
    y = torch.zeros(B * N, device="cuda")
    for xs, ws in ((buf[1:], w), (buf[:-1], buf[1:])):
        with pytest.raises(F.FusionError) as e:
            F.fusion_cnn_dense_noalloc(xs, ws, b, B, N, K, True, y)
        assert e.value.code == F.FUSION_EINVAL and "aligned" in str(e.value)
    # the aligned call still works afterwards
    F.fusion_cnn_dense_noalloc(buf[:-1], w, b, B, N, K, True, y)
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0
