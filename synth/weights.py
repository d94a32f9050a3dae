"""Seeded random-init weights and the little-endian float32 weights blob.

No trained checkpoint exists, so weights are drawn from
``numpy.random.default_rng(seed)`` in the order of ``layout(desc)``:

* conv and dense layers followed by ReLU: Kaiming-uniform with ReLU gain,
  bound sqrt(6 / fan_in), fan_in = C_in k^3 (or the input width);
* biases, message transforms, gates and the last head layer:
  U(+-1/sqrt(fan_in));
* GRU matrices and biases: U(+-1/sqrt(w)) with w the stage's node-state width
  (the usual GRU init);
* SELU head layers: LeCun-uniform, bound sqrt(3 / fan_in).

The blob is every tensor of ``layout(desc)`` in order, each row-major
float32 little-endian, with no header or padding.  Tensor shapes follow the
PyTorch conventions: conv ``[C_out][C_in][kd][kh][kw]``, linear ``[out][in]``,
GRU ``w_ih``/``w_hh`` ``[3H][H]`` with gate rows in (reset, update, new)
order.  The CNN dense layer's input index is the (C, D, H, W) flattening of
the pooled map.  A model with a second CNN dense layer (``cnn_dense2``) has
it right after the first; SG-CNN stages of their own widths (``sg_width``)
have matrices of those widths, the gate between stages mapping
[h (w_0), h0 (w_0)] to w_1.
"""

from __future__ import annotations

import numpy as np

from .configs import EDGE_COV, EDGE_NC


def cnn_out_shape(desc):
    """(channels, side) of the 3D-CNN feature map after the convs and pool."""
    n = desc["grid_n"]
    c = desc["n_feat"]
    for cv in desc["conv"]:
        p = cv["k"] // 2
        n = (n + 2 * p - cv["k"]) // cv["stride"] + 1
        c = cv["c_out"]
    if desc["pool"] and desc["pool"] > 1:
        n = n // desc["pool"]
    return c, n


def stage_widths(desc):
    """Node-state width of each SG-CNN stage: sg_width[s] when given (nonzero), else sg_hidden."""
    H = desc["sg_hidden"]
    w = list(desc.get("sg_width") or [])
    return [w[s] if s < len(w) and w[s] else H for s in range(len(desc["sg_stages"]))]


def edge_types(mask):
    out = []
    if mask & EDGE_COV:
        out.append("cov")
    if mask & EDGE_NC:
        out.append("nc")
    return out


def layout(desc):
    """[(name, shape, init_kind, fan_in)] in blob order."""
    L = []
    c_prev = desc["n_feat"]
    for i, cv in enumerate(desc["conv"]):
        fan = cv["c_in"] * cv["k"] ** 3
        L.append((f"conv{i}.w", (cv["c_out"], cv["c_in"], cv["k"], cv["k"], cv["k"]), "kaiming", fan))
        L.append((f"conv{i}.b", (cv["c_out"],), "bias", fan))
        c_prev = cv["c_out"]
    c, n = cnn_out_shape(desc)
    flat = c * n ** 3
    L.append(("cnn_dense.w", (desc["cnn_dense"], flat), "kaiming", flat))
    L.append(("cnn_dense.b", (desc["cnn_dense"],), "bias", flat))
    d2 = desc.get("cnn_dense2", 0)
    if d2:
        L.append(("cnn_dense2.w", (d2, desc["cnn_dense"]), "kaiming", desc["cnn_dense"]))
        L.append(("cnn_dense2.b", (d2,), "bias", desc["cnn_dense"]))
    cnn_latent = d2 or desc["cnn_dense"]
    wid = stage_widths(desc)
    for s, st in enumerate(desc["sg_stages"]):
        H = wid[s]
        for e in edge_types(st["edges"]):
            L.append((f"sg{s}.{e}.w", (H, H), "bias", H))
            L.append((f"sg{s}.{e}.b", (H,), "bias", H))
        L.append((f"sg{s}.gru.w_ih", (3 * H, H), "gru", H))
        L.append((f"sg{s}.gru.w_hh", (3 * H, H), "gru", H))
        L.append((f"sg{s}.gru.b_ih", (3 * H,), "gru", H))
        L.append((f"sg{s}.gru.b_hh", (3 * H,), "gru", H))
        if desc["sg_gate"] and s + 1 < len(desc["sg_stages"]):
            Hn = wid[s + 1]
            L.append((f"sg{s}.gate.wi", (Hn, H + wid[0]), "bias", H + wid[0]))
            L.append((f"sg{s}.gate.bi", (Hn,), "bias", H + wid[0]))
            L.append((f"sg{s}.gate.wj", (Hn, H), "bias", H))
            L.append((f"sg{s}.gate.bj", (Hn,), "bias", H))
    G = desc["sg_gather_width"]
    H = wid[-1]
    if desc["sg_gather"] == "gated":
        L.append(("gather.wg", (G, 2 * H), "bias", 2 * H))
        L.append(("gather.bg", (G,), "bias", 2 * H))
        L.append(("gather.wo", (G, H), "bias", H))
        L.append(("gather.bo", (G,), "bias", H))
    else:
        L.append(("gather.w", (G, H), "bias", H))
        L.append(("gather.b", (G,), "bias", H))
    mode = desc.get("fusion", "coherent")
    # branch output layers: Late Fusion's own affinity stacks (ReLU between), Mid-level's dense layers (SELU)
    for br, fin in (("cnn_out", cnn_latent), ("sg_out", G)):
        widths = desc.get(br, [])
        for l, w in enumerate(widths):
            last = l + 1 == len(widths)
            kind = "lecun" if mode == "mid" else ("bias" if last else "kaiming")
            L.append((f"{br}{l}.w", (w, fin), kind, fin))
            L.append((f"{br}{l}.b", (w,), "bias", fin))
            fin = w
    fin = cnn_latent + G
    if mode == "mid":
        fin += desc["cnn_out"][-1] + desc["sg_out"][-1]
    for l, w in enumerate(desc["head"]):
        last = l + 1 == len(desc["head"])
        L.append((f"head{l}.w", (w, fin), "bias" if last else "lecun", fin))
        L.append((f"head{l}.b", (w,), "bias", fin))
        fin = w
    return L


def init_weights(desc, seed: int):
    """Dict name -> float32 array, drawn in ``layout`` order from one generator."""
    rng = np.random.default_rng(seed)
    W = {}
    for name, shape, kind, fan in layout(desc):
        if kind == "kaiming":
            bound = np.sqrt(6.0 / fan)
        elif kind == "lecun":
            bound = np.sqrt(3.0 / fan)
        else:                                          # bias-style, and GRU (fan = the stage's width)
            bound = 1.0 / np.sqrt(fan)
        W[name] = ((rng.random(shape, dtype=np.float32) * 2.0 - 1.0) * np.float32(bound)).astype(np.float32)
    return W


def to_blob(desc, W) -> bytes:
    parts = []
    for name, shape, _k, _f in layout(desc):
        a = np.ascontiguousarray(W[name], dtype="<f4")
        assert a.shape == tuple(shape), (name, a.shape, shape)
        parts.append(a.tobytes())
    return b"".join(parts)


def blob_size(desc) -> int:
    return 4 * sum(int(np.prod(s)) for _n, s, _k, _f in layout(desc))
