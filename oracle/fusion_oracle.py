"""Plain FP64 CPU oracle for Coherent Fusion pose scoring.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (the CUDA library and its binding) never calls it and
shares no code with it.

It evaluates the forward pass of the model the paper describes, written out as
its definition, in float64 (except where the method fixes float32: the grid
origin and containing voxel, and the distance-cutoff edge test):

* voxelization of atoms into a C-channel density grid (Section 1, Section 3.3:
  a voxelized representation of atoms in a 3D grid);
* the 3D-CNN: convolutions with bias and ReLU, residual blocks, max-pool and a
  dense layer (Section 3.3.1, Table III, Fig. 1);
* the spatial graph with covalent and non-covalent edge types chosen by
  distance thresholds (Section 1, Table I, Table II);
* PotentialNet gated graph convolution: GRU-updated message passing, a
  per-node gate between stages and a gated sum over ligand atoms (Section
  3.3.1, citing PotentialNet and Gated Graph Sequence Neural Networks);
* the fusion head: concatenated latents through dense layers with SELU
  (Section 3.3.3, Table V); dropout is the identity at inference;
* the output is the predicted affinity in pK units (Eq. 1).

The paper defers the exact voxel kernel, grid placement and layer equations to
the earlier FAST work, which is not available; the readings used here are:

* grid centre = ligand centroid, summed left to right in float32 and divided
  by the ligand atom count in float32; origin = centre - (n h / 2) in float32;
* the containing voxel of an atom on axis d is floor(fl32(fl32(x_d - o_d) / h));
* each atom spreads its features with the voxel-integrated isotropic Gaussian
  w = prod_d 1/2 [erf((u_d + h - x_d) / (sigma sqrt 2)) - erf((u_d - x_d) / (sigma sqrt 2))]
  (u_d = lower voxel edge) over the cube of voxels within +-k of its
  containing voxel; voxels outside the grid are dropped, never renormalised;
* conv: same padding k // 2, bias, ReLU; residual block y = x + ReLU(conv(x));
  pool 2^3 stride 2; flatten in (C, D, H, W) order; dense + ReLU (and, when the
  model has one, a second dense + ReLU whose output is the CNN latent);
* edges (exact float32, no fused multiply-add): s = fl(fl(fl(dx dx) + fl(dy dy)) + fl(dz dz))
  with dx = fl(x_i - x_j); covalent iff s < fl(c_cov c_cov); non-covalent iff
  not covalent and s < fl(c_nc c_nc); i != j;
* h0 = features zero-padded to the first stage's width (the hidden width H
  unless a stage width is given); message
  m_i = sum over edge types e and neighbours j of (W_e h_j + b_e);
  h <- GRU(m, h); gate between stages h <- sigmoid(W_i [h, h0] + b_i) * (W_j h + b_j),
  which maps to the next stage's width;
* gather over ligand atoms i < n_lig: gated sum
  sum_i sigmoid(W_g [h_i, x_i] + b_g) * (W_o h_i + b_o), x_i = the input of the
  last stage, or the linear sum sum_i (W h_i + b);
* head: Linear -> SELU -> ... -> Linear, concatenation order [cnn, sg].
"""

from __future__ import annotations

import math

import numpy as np

EDGE_COV = 1
EDGE_NC = 2

SELU_ALPHA = 1.6732632423543772848170429916717
SELU_SCALE = 1.0507009873554804934193349852946

_erf = np.vectorize(math.erf, otypes=[np.float64])


# ---------------------------------------------------------------- voxelize --

def grid_origin(xyz_lig, n, h):
    """Grid origin (float32 [3]) from the ligand atoms (Section 3.3 grid placement reading).

    Centroid summed left to right in float32, divided in float32; the origin
    sits half a grid edge below it.
    """
    xyz_lig = np.asarray(xyz_lig, dtype=np.float32)
    s = np.zeros(3, dtype=np.float32)
    for a in range(len(xyz_lig)):
        s = (s + xyz_lig[a]).astype(np.float32)
    c = (s / np.float32(len(xyz_lig))).astype(np.float32)
    half = np.float32(np.float32(n) * np.float32(h)) * np.float32(0.5)
    return (c - half).astype(np.float32)


def containing_voxel(x, origin, h):
    """Integer voxel index per axis: floor(fl32(fl32(x - o) / h))."""
    t = (np.float32(x) - np.float32(origin)).astype(np.float32)
    q = (t / np.float32(h)).astype(np.float32)
    return np.floor(q).astype(np.int64)


def axis_weights(x, origin, ci, h, sigma, k):
    """1D voxel-integrated Gaussian weights for voxels ci-k..ci+k on one axis (float64)."""
    d = float(np.float64(x) - np.float64(origin))      # exact for float32 inputs
    idx = np.arange(ci - k, ci + k + 1, dtype=np.float64)
    lo = idx * h - d
    s2 = sigma * math.sqrt(2.0)
    return 0.5 * (_erf((lo + h) / s2) - _erf(lo / s2))


def voxelize(xyz, feat, origin, n, h, sigma, k):
    """Density grid G[z][y][x][c] (float64): G = sum_a feat[a][c] w(a, v) (Section 3.3 reading)."""
    xyz = np.asarray(xyz, dtype=np.float32)
    feat = np.asarray(feat, dtype=np.float32).astype(np.float64)
    C = feat.shape[1]
    G = np.zeros((n, n, n, C), dtype=np.float64)
    for a in range(len(xyz)):
        ci = [int(containing_voxel(xyz[a, d], origin[d], h)) for d in range(3)]
        w = [axis_weights(xyz[a, d], origin[d], ci[d], h, sigma, k) for d in range(3)]
        sl = []
        ws = []
        skip = False
        for d in range(3):
            lo, hi = ci[d] - k, ci[d] + k + 1
            clo, chi = max(lo, 0), min(hi, n)
            if clo >= chi:
                skip = True
                break
            sl.append(slice(clo, chi))
            ws.append(w[d][clo - lo: chi - lo])
        if skip:
            continue
        wx, wy, wz = ws
        sx, sy, sz = sl
        block = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
        G[sz, sy, sx, :] += block[..., None] * feat[a][None, None, None, :]
    return G


# ------------------------------------------------------------------ 3D-CNN --

def conv3d(x, w, b, stride=1):
    """y[z][o] = b[o] + sum_{i, delta} W[o][i][delta] x_pad[z*s + delta][i] (Section 3.3.1).

    x: [D][H][W][C_in] float64; w: [C_out][C_in][k][k][k]; same padding k // 2.
    The sum over input channels for each kernel offset is a matrix product.
    """
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    k = w.shape[2]
    p = k // 2
    D, Hh, Ww, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((D + 2 * p, Hh + 2 * p, Ww + 2 * p, Ci))
    xp[p:p + D, p:p + Hh, p:p + Ww] = x
    Do = (D + 2 * p - k) // stride + 1
    Ho = (Hh + 2 * p - k) // stride + 1
    Wo = (Ww + 2 * p - k) // stride + 1
    y = np.zeros((Do, Ho, Wo, Co)) + np.asarray(b, dtype=np.float64)
    for kd in range(k):
        for kh in range(k):
            for kw in range(k):
                xs = xp[kd:kd + stride * (Do - 1) + 1:stride,
                        kh:kh + stride * (Ho - 1) + 1:stride,
                        kw:kw + stride * (Wo - 1) + 1:stride, :]
                y += np.ascontiguousarray(xs).reshape(-1, Ci).dot(w[:, :, kd, kh, kw].T).reshape(Do, Ho, Wo, Co)
    return y


def relu(x):
    return np.maximum(x, 0.0)


def maxpool3d(x, p=2):
    """Max over non-overlapping p^3 windows, floor of the side (Fig. 1 pool)."""
    D = x.shape[0] // p
    x = x[:D * p, :D * p, :D * p]
    C = x.shape[3]
    return x.reshape(D, p, D, p, D, p, C).max(axis=(1, 3, 5))


def cnn_branch(desc, W, G, stages=None):
    """3D-CNN latent from the grid (Section 3.3.1, Table III)."""
    x = G
    for i, cv in enumerate(desc["conv"]):
        y = relu(conv3d(x, W[f"conv{i}.w"], W[f"conv{i}.b"], cv["stride"]))
        if cv["residual"]:
            y = x + y
        x = y
        if stages is not None:
            stages[f"conv{i}"] = x
    if desc["pool"] and desc["pool"] > 1:
        x = maxpool3d(x, desc["pool"])
        if stages is not None:
            stages["pool"] = x
    v = x.transpose(3, 0, 1, 2).reshape(-1)
    out = relu(W["cnn_dense.w"].astype(np.float64) @ v + W["cnn_dense.b"])
    if desc.get("cnn_dense2"):
        # a second dense layer (Section 3.3.1: the second dense layer is the first reduced by a factor of 2);
        # the latent the fusion layers read is the last hidden layer, Layer^{M-1} (Section 2.2)
        if stages is not None:
            stages["cnn_dense1"] = out
        out = relu(W["cnn_dense2.w"].astype(np.float64) @ out + W["cnn_dense2.b"])
    if stages is not None:
        stages["cnn_latent"] = out
    return out


# ------------------------------------------------------------------- graph --

def radius_graph(xyz, cut_cov, cut_nc):
    """Covalent and non-covalent edge sets (Section 1, Table II) under the float32 rule.

    Returns {"cov": (row_ptr, col), "nc": (row_ptr, col)} with local indices,
    rows sorted by neighbour index.
    """
    x = np.asarray(xyz, dtype=np.float32)
    n = len(x)
    dx = (x[:, None, 0] - x[None, :, 0]).astype(np.float32)
    dy = (x[:, None, 1] - x[None, :, 1]).astype(np.float32)
    dz = (x[:, None, 2] - x[None, :, 2]).astype(np.float32)
    s = ((dx * dx + dy * dy).astype(np.float32) + dz * dz).astype(np.float32)
    c2 = np.float32(np.float32(cut_cov) * np.float32(cut_cov))
    n2 = np.float32(np.float32(cut_nc) * np.float32(cut_nc))
    off = ~np.eye(n, dtype=bool)
    cov = (s < c2) & off
    nc = (~cov) & (s < n2) & off
    out = {}
    for name, m in (("cov", cov), ("nc", nc)):
        deg = m.sum(axis=1)
        rp = np.zeros(n + 1, dtype=np.int64)
        rp[1:] = np.cumsum(deg)
        col = np.nonzero(m)[1].astype(np.int32)   # row-major: sorted by j within a row
        out[name] = (rp, col)
    return out


# ------------------------------------------------------------------ SG-CNN --

def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def gru_cell(m, h, w_ih, w_hh, b_ih, b_hh):
    """Gated recurrent unit update (Gated Graph Sequence Neural Networks, cited in Section 3.3.1).

    Gate rows in (reset, update, new) order:
    r = sigmoid(W_ir m + b_ir + W_hr h + b_hr), z = sigmoid(W_iz m + b_iz + W_hz h + b_hz),
    n = tanh(W_in m + b_in + r * (W_hn h + b_hn)), h' = (1 - z) * n + z * h.
    """
    H = h.shape[1]
    gi = m @ w_ih.T + b_ih
    gh = h @ w_hh.T + b_hh
    r = sigmoid(gi[:, :H] + gh[:, :H])
    z = sigmoid(gi[:, H:2 * H] + gh[:, H:2 * H])
    nn = np.tanh(gi[:, 2 * H:] + r * gh[:, 2 * H:])
    return (1.0 - z) * nn + z * h


def _edge_names(mask):
    out = []
    if mask & EDGE_COV:
        out.append("cov")
    if mask & EDGE_NC:
        out.append("nc")
    return out


def stage_widths(desc):
    """Node-state width of each SG-CNN stage: sg_width[s] when given (nonzero), else sg_hidden."""
    H = desc["sg_hidden"]
    w = list(desc.get("sg_width") or [])
    return [w[s] if s < len(w) and w[s] else H for s in range(len(desc["sg_stages"]))]


def sg_branch(desc, W, feat, n_lig, graph, stages=None):
    """SG-CNN latent (Section 3.3.1, Table II): gated graph conv stages + ligand gather.

    Stage s keeps node states of its own width w_s (the first stage at least the feature count); the gate
    between stages maps [h, h0] to the next stage's width (the covalent gather width of Table II)."""
    W = {k: v.astype(np.float64) for k, v in W.items() if k.startswith(("sg", "gather"))}
    widths = stage_widths(desc)
    N = len(feat)
    h0 = np.zeros((N, widths[0]))
    h0[:, :feat.shape[1]] = np.asarray(feat, dtype=np.float64)
    h = h0
    x_in = h0
    nst = len(desc["sg_stages"])
    for s, st in enumerate(desc["sg_stages"]):
        x_in = h
        H = widths[s]
        for step in range(st["steps"]):
            m = np.zeros((N, H))
            for e in _edge_names(st["edges"]):
                T = h @ W[f"sg{s}.{e}.w"].T + W[f"sg{s}.{e}.b"]
                rp, col = graph[e]
                rows = np.repeat(np.arange(N), np.diff(rp))
                np.add.at(m, rows, T[col])
            h = gru_cell(m, h, W[f"sg{s}.gru.w_ih"], W[f"sg{s}.gru.w_hh"],
                         W[f"sg{s}.gru.b_ih"], W[f"sg{s}.gru.b_hh"])
            if stages is not None:
                stages[f"sg{s}.step{step}"] = h
        if desc["sg_gate"] and s + 1 < nst:
            hh = np.concatenate([h, h0], axis=1)
            h = sigmoid(hh @ W[f"sg{s}.gate.wi"].T + W[f"sg{s}.gate.bi"]) * \
                (h @ W[f"sg{s}.gate.wj"].T + W[f"sg{s}.gate.bj"])
            if stages is not None:
                stages[f"sg{s}.gate"] = h
    hl = h[:n_lig]
    if desc["sg_gather"] == "gated":
        xl = x_in[:n_lig]
        g = sigmoid(np.concatenate([hl, xl], axis=1) @ W["gather.wg"].T + W["gather.bg"])
        v = g * (hl @ W["gather.wo"].T + W["gather.bo"])
    else:
        v = hl @ W["gather.w"].T + W["gather.b"]
    out = v.sum(axis=0)
    if stages is not None:
        stages["sg_latent"] = out
    return out


# -------------------------------------------------------------------- head --

def selu(x):
    """SELU with the constants of Klambauer et al. (cited in Table V)."""
    return SELU_SCALE * np.where(x > 0, x, SELU_ALPHA * (np.exp(np.minimum(x, 0.0)) - 1.0))


def _dense(W, name, v):
    return W[f"{name}.w"].astype(np.float64) @ v + W[f"{name}.b"].astype(np.float64)


def head(desc, W, cnn, sg):
    """Affinity from the two latents.

    Coherent Fusion (Section 3.3.3, Table V): the concatenated latents through
    the fusion layers, Linear -> SELU ... -> Linear.  Mid-level Fusion (Section
    2.2, Table IV): each latent first through its model-specific dense layers
    (Linear -> SELU each), those outputs concatenated after the two latents,
    then the fusion layers.  Late Fusion (Section 2.2): the unweighted mean of
    the two branches' own affinities, each branch a stack Linear -> ReLU ... ->
    Linear of final width 1.  With head_residual, a hidden fusion layer whose
    input and output widths match returns x + SELU(W x + b).
    """
    mode = desc.get("fusion", "coherent")
    cnn = np.asarray(cnn, dtype=np.float64)
    sg = np.asarray(sg, dtype=np.float64)
    if mode == "late":
        out = []
        for br, v in (("cnn_out", cnn), ("sg_out", sg)):
            n = len(desc[br])
            for l in range(n):
                v = _dense(W, f"{br}{l}", v)
                if l + 1 < n:
                    v = relu(v)
            out.append(float(v[0]))
        return 0.5 * (out[0] + out[1])
    v = np.concatenate([cnn, sg])
    if mode == "mid":
        parts = [cnn, sg]
        for br, u in (("cnn_out", cnn), ("sg_out", sg)):
            for l in range(len(desc[br])):
                u = selu(_dense(W, f"{br}{l}", u))
            parts.append(u)
        v = np.concatenate(parts)
    L = len(desc["head"])
    for l in range(L):
        u = _dense(W, f"head{l}", v)
        if l + 1 < L:
            u = selu(u)
            if desc.get("head_residual", 0) and u.shape == v.shape:
                u = v + u
        v = u
    return float(v[0])


# ------------------------------------------------------------------- whole --

def score_pose(desc, W, xyz, feat, n_lig, stages=None, origin=None):
    """Predicted affinity (pK, Eq. 1) of one pose."""
    n, h = desc["grid_n"], desc["grid_h"]
    if origin is None:
        origin = grid_origin(xyz[:n_lig], n, h)
    G = voxelize(xyz, feat, origin, n, h, desc["sigma"], desc["support"])
    if stages is not None:
        stages["origin"] = origin
        stages["grid"] = G
    cnn = cnn_branch(desc, W, G, stages)
    graph = radius_graph(xyz, desc["cut_cov"], desc["cut_nc"])
    if stages is not None:
        stages["graph"] = graph
    sg = sg_branch(desc, W, feat, n_lig, graph, stages)
    a = head(desc, W, cnn, sg)
    if stages is not None:
        stages["affinity"] = a
    return a

