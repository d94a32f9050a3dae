"""The error of the three-term BF16 product that the tensor-core graph step uses (CPU).

x = x_hi + x_lo + r_x with x_hi = bf16(x), x_lo = bf16(x - x_hi) (round to nearest even, 8 significant
bits), so |x_lo| <= 2^-8 |x| and |r_x| <= 2^-16 |x|.  Then x y - (x_lo y_hi + x_hi y_lo + x_hi y_hi) =
x_hi r_y + r_x y_hi + x_lo y_lo + smaller terms, at most about 3 * 2^-16 |x y| (4.6e-5), and in a dot product
the independent rounding errors mostly cancel.  Checked here on node-state and weight values of the graph
step's shapes and ranges (states in [-1, 1], weights U(+-1/8)): the elementwise bound, a K = 64 dot product
within 1e-5 of the sum of its |terms|, and the figure the GPU tolerance relies on: dropping any one of the
three terms, or plain BF16 products, errs by over 100x more.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def split(a):
    a = np.asarray(a, dtype=np.float32)
    hi = bf16(a)
    lo = bf16((a.astype(np.float64) - hi).astype(np.float32))
    return hi, lo


def test_three_term_product_error_bound():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(128, 64)).astype(np.float32)
    w = (rng.uniform(-1, 1, size=(192, 64)) / 8.0).astype(np.float32)
    xh, xl = split(x)
    wh, wl = split(w)
    xd, wd = x.astype(np.float64), w.astype(np.float64)
    # elementwise products of every (node, output, input) triple
    exact = xd[:, None, :] * wd[None, :, :]
    three = xl[:, None, :] * wh[None, :, :] + xh[:, None, :] * wl[None, :, :] + xh[:, None, :] * wh[None, :, :]
    err3 = np.abs(three - exact)
    assert np.all(err3 <= 3.0 * 2.0 ** -16 * np.abs(exact))
    # a K = 64 dot product: within 1e-5 of the sum of its |terms|
    dot_err = np.abs(three.sum(-1) - exact.sum(-1))
    scale = np.abs(exact).sum(-1)
    rel3 = (dot_err / scale).max()
    assert rel3 <= 1e-5
    # one term dropped, or plain BF16: over 100x the three-term error
    variants = {
        "no lo*hi": xh[:, None, :] * wl[None, :, :] + xh[:, None, :] * wh[None, :, :],
        "no hi*lo": xl[:, None, :] * wh[None, :, :] + xh[:, None, :] * wh[None, :, :],
        "plain bf16": xh[:, None, :] * wh[None, :, :],
    }
    for name, v in variants.items():
        rel = (np.abs(v.sum(-1) - exact.sum(-1)) / scale).max()
        assert rel > 100 * rel3, (name, rel, rel3)
