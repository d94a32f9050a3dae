"""Pins of the oracle's Mid-level and Late Fusion heads (Section 2.2) against
facts that do not come from the oracle itself:

* Late Fusion is the plain mean of two independent affinity stacks: each stack
  restated with torch float64 Linear/ReLU layers, and a stack whose last layer
  has zero weights returns exactly its bias (so the mean's 1/2 is pinned);
* Mid-level Fusion with zero branch weights and biases feeds SELU(0) = 0 into
  the appended columns, so it equals a coherent head on the first (cnn + sg)
  columns of its first layer: this pins the concatenation order [cnn, sg,
  branch outputs];
* a residual hidden fusion layer with zero weights and bias is the identity
  (x + SELU(0) = x), and without the residual flag it maps to zero;
* the Mid-level head restated with torch float64 layers.
"""

import numpy as np
import pytest

from oracle import fusion_oracle as O
from synth import configs, weights

torch = pytest.importorskip("torch")


def _latents(desc, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(desc["cnn_dense"]), rng.standard_normal(desc["sg_gather_width"])


def _torch_stack(W, prefix, widths, x, act_between, act_last):
    v = torch.from_numpy(np.asarray(x, dtype=np.float64))
    for l in range(len(widths)):
        lin = torch.nn.Linear(v.shape[0], widths[l]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W[f"{prefix}{l}.w"].astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(W[f"{prefix}{l}.b"].astype(np.float64)))
        v = lin(v)
        last = l + 1 == len(widths)
        act = act_last if last else act_between
        if act == "relu":
            v = torch.relu(v)
        elif act == "selu":
            v = torch.nn.functional.selu(v)
    return v.detach().numpy()


@pytest.mark.parametrize("name", ["fusion-24grid-c32-late", "fusion-48grid-c64-late"])
def test_late_fusion_is_mean_of_torch_stacks(name):
    desc = configs.model(name)
    W = weights.init_weights(desc, 3)
    c, s = _latents(desc, 4)
    ac = _torch_stack(W, "cnn_out", desc["cnn_out"], c, "relu", None)[0]
    as_ = _torch_stack(W, "sg_out", desc["sg_out"], s, "relu", None)[0]
    assert abs(O.head(desc, W, c, s) - 0.5 * (ac + as_)) <= 1e-12 * (1 + abs(ac) + abs(as_))


def test_late_fusion_constant_branch_pins_the_mean():
    desc = configs.model("fusion-24grid-c32-late")
    W = weights.init_weights(desc, 5)
    c, s = _latents(desc, 6)
    last = len(desc["cnn_out"]) - 1
    W[f"cnn_out{last}.w"][:] = 0.0
    W[f"cnn_out{last}.b"][:] = np.float32(2.5)
    as_ = _torch_stack(W, "sg_out", desc["sg_out"], s, "relu", None)[0]
    assert O.head(desc, W, c, s) == pytest.approx(0.5 * (2.5 + as_), abs=1e-12)


@pytest.mark.parametrize("name", ["fusion-24grid-c32-mid", "fusion-48grid-c64-mid"])
def test_mid_fusion_zero_branches_equal_coherent_head_on_leading_columns(name):
    desc = configs.model(name)
    W = weights.init_weights(desc, 7)
    for br in ("cnn_out", "sg_out"):
        for l in range(len(desc[br])):
            W[f"{br}{l}.w"][:] = 0.0
            W[f"{br}{l}.b"][:] = 0.0
    c, s = _latents(desc, 8)
    coh = configs.model(name)
    coh.update(fusion="coherent", cnn_out=[], sg_out=[])
    Wc = dict(W)
    Wc["head0.w"] = W["head0.w"][:, :desc["cnn_dense"] + desc["sg_gather_width"]].copy()
    assert O.head(desc, W, c, s) == pytest.approx(O.head(coh, Wc, c, s), abs=1e-12)


def test_mid_fusion_matches_torch_restatement():
    desc = configs.model("fusion-24grid-c32-mid")
    W = weights.init_weights(desc, 9)
    c, s = _latents(desc, 10)
    dc = _torch_stack(W, "cnn_out", desc["cnn_out"], c, "selu", "selu")
    ds = _torch_stack(W, "sg_out", desc["sg_out"], s, "selu", "selu")
    v = torch.from_numpy(np.concatenate([c, s, dc, ds]))
    L = len(desc["head"])
    for l in range(L):
        lin = torch.nn.Linear(v.shape[0], desc["head"][l]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W[f"head{l}.w"].astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(W[f"head{l}.b"].astype(np.float64)))
        u = lin(v)
        if l + 1 < L:
            u = torch.nn.functional.selu(u)
            if u.shape == v.shape:          # the preset has head_residual = 1
                u = u + v
        v = u
    assert O.head(desc, W, c, s) == pytest.approx(float(v.detach()[0]), abs=1e-10)


def test_residual_zero_layer_is_identity():
    desc = configs.model("fusion-24grid-c32-mid")          # head [96, 96, 1], residual on
    W = weights.init_weights(desc, 11)
    c, s = _latents(desc, 12)
    W["head1.w"][:] = 0.0
    W["head1.b"][:] = 0.0
    # with layer 1 the identity, the head is layer 0 (SELU) then the last layer applied to its output
    W2 = dict(W)
    W2["head1.w"] = W["head2.w"]
    W2["head1.b"] = W["head2.b"]
    short = configs.model("fusion-24grid-c32-mid")
    short["head"] = [96, 1]
    assert O.head(desc, W, c, s) == pytest.approx(O.head(short, W2, c, s), abs=1e-12)
    # without the residual, the zero layer maps everything to SELU(0) = 0 and the output is the last bias
    plain = configs.model("fusion-24grid-c32-mid")
    plain["head_residual"] = 0
    assert O.head(plain, W, c, s) == pytest.approx(float(W["head2.b"][0]), abs=1e-12)
