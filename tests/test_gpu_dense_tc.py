"""The CNN dense layer on the tensor cores (BF16 / FP8 models, Section 3.3.1: flatten -> dense + ReLU) against
a float64 product of its own inputs.

`dense_tc_kernel` multiplies the pooled map (stored in bf16) by the dense matrix rounded to bf16 (round to
nearest even) with FP32 accumulation: split-K partials of 16-wide MMA steps, reduced in a fixed split order,
then bias and ReLU.  The same product is computed here in float64 from the fetched pooled map and the
host-rounded matrix.  FP32 accumulation over K terms errs by at most about (K / 16 + splits) x 2^-24 of the
sum of |terms| (8e-4 for K = 221,184, the full-size model) and in practice by far less: measured 4.5e-8.  The
bound used, 2e-6 of each output's sum of |terms|, keeps 40x room over that, while a dropped 64-wide K slice
(about 3e-4 of the sum at this K), a wrong tile or a transposed operand moves outputs by far more.

* full-size model (221,184 -> 256), 4 poses of the 64-pose workload, BF16 and FP8 models (the FP8 model
  keeps this layer in BF16);
* the paper-final model (110,592 -> 128, then the second dense layer 128 -> 64 in FP32): its latent against
  ReLU(b2 + W2 y1) with y1 the float64 first layer.
"""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights
from synth.weights import cnn_out_shape

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _dense_dhwc(desc, w):
    """A dense matrix whose input is the (C, D, H, W) flatten, reordered to the GPU's (D, H, W, C) flatten."""
    c, n = cnn_out_shape(desc)
    w = w.reshape(w.shape[0], c, n * n * n)
    return np.ascontiguousarray(w.transpose(0, 2, 1).reshape(w.shape[0], -1))


def _check(got, x, w, b, relu=True):
    terms = np.abs(x) @ np.abs(w).T                       # each output's sum of |terms|
    ref = x @ w.T + b
    if relu:
        ref = np.maximum(ref, 0.0)
    err = np.abs(got - ref)
    # ReLU can only shrink a difference, so the pre-activation bound holds after it
    ok = err <= 2e-6 * terms + 1e-7
    assert np.all(ok), (float(err.max()), float((err / (terms + 1e-30)).max()))
    return float((err / (terms + 1e-30)).max())


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_full_size_dense_tc(F, dtype):
    name = "fusion-48grid-c64"
    W = weights.init_weights(configs.model(name), 0)
    desc = configs.model(name, dtype=dtype)
    batch = poses.subset(poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"]), [0, 9, 33, 63])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=1200, keep_stages=True)
    m.score(batch)
    x = np.stack([m.fetch(F.STAGE_POOL, p) for p in range(4)]).astype(np.float64)
    got = np.stack([m.fetch(F.STAGE_CNN_LATENT, p) for p in range(4)]).astype(np.float64)
    m.close()
    w = _bf16(_dense_dhwc(desc, W["cnn_dense.w"]))
    worst = _check(got, x, w, W["cnn_dense.b"].astype(np.float64))
    print(f"dense on tensor cores ({dtype}): max |error| / sum |terms| = {worst:.2e}")


def test_paper_final_dense_layers(F):
    name = "fusion-paper-final"
    W = weights.init_weights(configs.model(name), 1)
    desc = configs.model(name, dtype="bf16")
    batch = poses.subset(poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"]), [2, 40])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=2, max_atoms=1200, keep_stages=True)
    m.score(batch)
    x = np.stack([m.fetch(F.STAGE_POOL, p) for p in range(2)]).astype(np.float64)
    got = np.stack([m.fetch(F.STAGE_CNN_LATENT, p) for p in range(2)]).astype(np.float64)
    m.close()
    w1 = _bf16(_dense_dhwc(desc, W["cnn_dense.w"]))
    y1 = np.maximum(x @ w1.T + W["cnn_dense.b"].astype(np.float64), 0.0)
    w2 = W["cnn_dense2.w"].astype(np.float64)
    # the second layer's inputs carry the first layer's FP32 error: bound it through |W2|
    terms1 = np.abs(x) @ np.abs(w1).T
    ref = np.maximum(y1 @ w2.T + W["cnn_dense2.b"].astype(np.float64), 0.0)
    bound = 2e-6 * (terms1 @ np.abs(w2).T) + 1e-5 * (np.abs(y1) @ np.abs(w2).T) + 1e-7
    err = np.abs(got - ref)
    assert np.all(err <= bound), (float(err.max()), float(bound.min()))
