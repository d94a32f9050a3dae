"""Pins of the oracle's 3D-CNN pieces against torch's float64 CPU library routines
and special cases with closed forms (1^3 kernel = matrix product, delta kernel = identity)."""

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import fusion_oracle as O


def _torch_conv(x, w, b, stride):
    k = w.shape[2]
    xt = torch.from_numpy(x).permute(3, 0, 1, 2)[None]
    y = F.conv3d(xt, torch.from_numpy(w), torch.from_numpy(b), stride=stride, padding=k // 2)
    return y[0].permute(1, 2, 3, 0).numpy()


@pytest.mark.parametrize("n,ci,co,k,s", [(6, 2, 3, 3, 1), (6, 2, 3, 5, 1), (7, 3, 4, 3, 2),
                                         (9, 4, 2, 5, 2), (5, 1, 1, 7, 1)])
def test_conv3d_matches_torch_float64(n, ci, co, k, s):
    rng = np.random.default_rng(n * 100 + k)
    x = rng.normal(size=(n, n, n, ci))
    w = rng.normal(size=(co, ci, k, k, k))
    b = rng.normal(size=co)
    np.testing.assert_allclose(O.conv3d(x, w, b, s), _torch_conv(x, w, b, s), rtol=1e-12, atol=1e-12)


def test_conv3d_unit_kernel_is_matmul():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(4, 5, 6, 3))
    w = rng.normal(size=(2, 3, 1, 1, 1))
    b = rng.normal(size=2)
    np.testing.assert_allclose(O.conv3d(x, w, b), x @ w[:, :, 0, 0, 0].T + b, rtol=1e-13, atol=1e-13)


def test_conv3d_delta_kernel_is_identity():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(6, 6, 6, 3))
    w = np.zeros((3, 3, 5, 5, 5))
    for c in range(3):
        w[c, c, 2, 2, 2] = 1.0
    np.testing.assert_array_equal(O.conv3d(x, w, np.zeros(3)), x)


def test_conv3d_offcentre_delta_shifts_with_zero_padding():
    x = np.arange(5 * 5 * 5, dtype=np.float64).reshape(5, 5, 5, 1)
    w = np.zeros((1, 1, 3, 3, 3))
    w[0, 0, 2, 1, 0] = 1.0          # reads x[z+1][y][x-1]
    y = O.conv3d(x, w, np.zeros(1))
    exp = np.zeros_like(x)
    exp[:4, :, 1:] = x[1:, :, :4]
    np.testing.assert_array_equal(y, exp)


def test_maxpool_matches_torch():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, 7, 7, 3))
    ref = F.max_pool3d(torch.from_numpy(x).permute(3, 0, 1, 2)[None], 2)[0].permute(1, 2, 3, 0).numpy()
    np.testing.assert_array_equal(O.maxpool3d(x, 2), ref)


@pytest.mark.parametrize("dense2", [0, 16])
def test_cnn_branch_matches_torch_restatement(dense2):
    """The CNN branch, and with a second dense layer (Section 3.3.1) whose output is the latent."""
    from synth import configs, weights
    desc = configs.model("fusion-20grid-ragged")
    desc["cnn_dense2"] = dense2
    W = weights.init_weights(desc, 4)
    rng = np.random.default_rng(4)
    G = np.abs(rng.normal(size=(20, 20, 20, 19))) * 0.1
    got = O.cnn_branch(desc, W, G)
    x = torch.from_numpy(G).permute(3, 0, 1, 2)[None]
    for i, cv in enumerate(desc["conv"]):
        y = F.relu(F.conv3d(x, torch.from_numpy(W[f"conv{i}.w"]).double(), torch.from_numpy(W[f"conv{i}.b"]).double(),
                            stride=cv["stride"], padding=cv["k"] // 2))
        x = x + y if cv["residual"] else y
    x = F.max_pool3d(x, 2)
    exp = F.relu(F.linear(x.reshape(-1), torch.from_numpy(W["cnn_dense.w"]).double(),
                          torch.from_numpy(W["cnn_dense.b"]).double()))
    if dense2:
        exp = F.relu(F.linear(exp, torch.from_numpy(W["cnn_dense2.w"]).double(),
                              torch.from_numpy(W["cnn_dense2.b"]).double()))
    np.testing.assert_allclose(got, exp.numpy(), rtol=1e-10, atol=1e-12)
