"""Pins of the oracle's SG-CNN, head and whole network:

* GRU update = torch.nn.GRUCell (float64, same weights);
* sigmoid and SELU = torch's;
* the SG branch equals a dense-adjacency restatement built on torch modules;
* the SG latent is invariant to atom order within the ligand and the pocket;
* zero message-passing steps with a linear gather has a closed form;
* the whole tiny network equals a torch restatement (F.conv3d, GRUCell, ...).
"""

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import fusion_oracle as O
from synth import configs, poses, weights


def test_gru_matches_torch_grucell():
    rng = np.random.default_rng(0)
    H = 16
    cell = torch.nn.GRUCell(H, H).double()
    m = rng.normal(size=(7, H))
    h = rng.normal(size=(7, H))
    exp = cell(torch.from_numpy(m), torch.from_numpy(h)).detach().numpy()
    got = O.gru_cell(m, h, cell.weight_ih.detach().numpy(), cell.weight_hh.detach().numpy(),
                     cell.bias_ih.detach().numpy(), cell.bias_hh.detach().numpy())
    np.testing.assert_allclose(got, exp, rtol=1e-13, atol=1e-14)


def test_activations_match_torch():
    x = np.linspace(-8, 8, 101)
    np.testing.assert_allclose(O.selu(x), F.selu(torch.from_numpy(x)).numpy(), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(O.sigmoid(x), torch.sigmoid(torch.from_numpy(x)).numpy(), rtol=1e-14)


def _widths(desc):
    w = list(desc.get("sg_width") or [])
    return [w[s] if s < len(w) and w[s] else desc["sg_hidden"] for s in range(len(desc["sg_stages"]))]


def _torch_sg(desc, W, feat, n_lig, graph):
    """Dense-adjacency restatement with torch modules (a GRUCell and Linear layers of each stage's width)."""
    T = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float64))
    widths = _widths(desc)
    H = widths[0]
    N = len(feat)
    A = {}
    for e, (rp, col) in graph.items():
        M = torch.zeros(N, N, dtype=torch.float64)
        for i in range(N):
            M[i, col[rp[i]:rp[i + 1]]] = 1.0
        A[e] = M
    h0 = torch.zeros(N, H, dtype=torch.float64)
    h0[:, :feat.shape[1]] = T(feat)
    h = h0
    x_in = h0
    for s, st in enumerate(desc["sg_stages"]):
        x_in = h
        H = widths[s]
        cell = torch.nn.GRUCell(H, H).double()
        with torch.no_grad():
            cell.weight_ih.copy_(T(W[f"sg{s}.gru.w_ih"]))
            cell.weight_hh.copy_(T(W[f"sg{s}.gru.w_hh"]))
            cell.bias_ih.copy_(T(W[f"sg{s}.gru.b_ih"]))
            cell.bias_hh.copy_(T(W[f"sg{s}.gru.b_hh"]))
        names = [n for n, bit in (("cov", 1), ("nc", 2)) if st["edges"] & bit]
        for _ in range(st["steps"]):
            m = sum(A[e] @ F.linear(h, T(W[f"sg{s}.{e}.w"]), T(W[f"sg{s}.{e}.b"])) for e in names)
            h = cell(m, h).detach()
        if desc["sg_gate"] and s + 1 < len(desc["sg_stages"]):
            g = torch.sigmoid(F.linear(torch.cat([h, h0], 1), T(W[f"sg{s}.gate.wi"]), T(W[f"sg{s}.gate.bi"])))
            h = g * F.linear(h, T(W[f"sg{s}.gate.wj"]), T(W[f"sg{s}.gate.bj"]))
    hl = h[:n_lig]
    if desc["sg_gather"] == "gated":
        g = torch.sigmoid(F.linear(torch.cat([hl, x_in[:n_lig]], 1), T(W["gather.wg"]), T(W["gather.bg"])))
        v = g * F.linear(hl, T(W["gather.wo"]), T(W["gather.bo"]))
    else:
        v = F.linear(hl, T(W["gather.w"]), T(W["gather.b"]))
    return v.sum(0).numpy()


@pytest.mark.parametrize("name", ["fusion-24grid-c32", "fusion-20grid-ragged", "fusion-paper-final"])
def test_sg_branch_matches_dense_adjacency_torch(name):
    """Includes the paper-final SG-CNN: stage widths 19 then 24 (Table II's covalent gather width)."""
    desc = configs.model(name)
    W = weights.init_weights(desc, 2)
    xyz, feat, n_lig = poses.make_pose(5, (20, 30), (60, 90))
    g = O.radius_graph(xyz, desc["cut_cov"], desc["cut_nc"])
    got = O.sg_branch(desc, W, feat, n_lig, g)
    exp = _torch_sg(desc, W, feat, n_lig, g)
    np.testing.assert_allclose(got, exp, rtol=1e-10, atol=1e-10)


def test_sg_latent_invariant_to_atom_order():
    desc = configs.model("fusion-48grid-c64")
    W = weights.init_weights(desc, 3)
    xyz, feat, n_lig = poses.make_pose(8, (20, 30), (80, 120))
    N = len(xyz)
    rng = np.random.default_rng(0)
    perm = np.concatenate([rng.permutation(n_lig), n_lig + rng.permutation(N - n_lig)])
    a = O.sg_branch(desc, W, feat, n_lig, O.radius_graph(xyz, 1.6, 4.5))
    b = O.sg_branch(desc, W, feat[perm], n_lig, O.radius_graph(xyz[perm], 1.6, 4.5))
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-11)


def test_zero_steps_linear_gather_closed_form():
    desc = configs.model("fusion-24grid-c32")
    desc["sg_stages"] = [dict(steps=0, edges=3)]
    W = weights.init_weights(desc, 1)
    xyz, feat, n_lig = poses.make_pose(2, (10, 10), (20, 20))
    got = O.sg_branch(desc, W, feat, n_lig, O.radius_graph(xyz, 1.6, 4.5))
    fs = feat[:n_lig].astype(np.float64).sum(axis=0)
    exp = W["gather.w"][:, :19].astype(np.float64) @ fs + n_lig * W["gather.b"].astype(np.float64)
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-12)


def test_isolated_node_gets_zero_message():
    desc = configs.model("fusion-24grid-c32")
    W = weights.init_weights(desc, 1)
    xyz = np.array([[0, 0, 0], [50, 0, 0]], dtype=np.float32)
    feat = np.random.default_rng(0).normal(size=(2, 19)).astype(np.float32)
    st = {}
    O.sg_branch(desc, W, feat, 1, O.radius_graph(xyz, 1.6, 4.5), st)
    h0 = np.zeros((2, 32))
    h0[:, :19] = feat
    Wd = {k: v.astype(np.float64) for k, v in W.items()}
    exp = O.gru_cell(np.zeros((2, 32)), h0, Wd["sg0.gru.w_ih"], Wd["sg0.gru.w_hh"], Wd["sg0.gru.b_ih"], Wd["sg0.gru.b_hh"])
    np.testing.assert_allclose(st["sg0.step0"], exp, rtol=1e-14)


def test_head_matches_torch():
    desc = configs.model("fusion-48grid-c64")
    W = weights.init_weights(desc, 5)
    rng = np.random.default_rng(5)
    cnn, sg = rng.normal(size=256), rng.normal(size=128)
    v = torch.from_numpy(np.concatenate([cnn, sg]))
    for l in range(3):
        v = F.linear(v, torch.from_numpy(W[f"head{l}.w"]).double(), torch.from_numpy(W[f"head{l}.b"]).double())
        if l < 2:
            v = F.selu(v)
    np.testing.assert_allclose(O.head(desc, W, cnn, sg), float(v[0]), rtol=1e-12)


def test_tiny_network_end_to_end_matches_torch_restatement():
    desc = configs.model("fusion-24grid-c32")
    W = weights.init_weights(desc, 0)
    b = poses.make_batch(configs.WORKLOADS["pose1-lig24-pocket200"])
    xyz, feat, n_lig = poses.pose_slice(b, 0)
    st = {}
    a = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
    # restate the CNN with torch on the oracle's (separately pinned) grid
    x = torch.from_numpy(st["grid"]).permute(3, 0, 1, 2)[None]
    for i, cv in enumerate(desc["conv"]):
        y = F.relu(F.conv3d(x, torch.from_numpy(W[f"conv{i}.w"]).double(), torch.from_numpy(W[f"conv{i}.b"]).double(),
                            padding=cv["k"] // 2))
        x = x + y if cv["residual"] else y
    x = F.max_pool3d(x, 2)
    cnn = F.relu(F.linear(x.reshape(-1), torch.from_numpy(W["cnn_dense.w"]).double(),
                          torch.from_numpy(W["cnn_dense.b"]).double()))
    sg = torch.from_numpy(_torch_sg(desc, W, feat, n_lig, st["graph"]))
    v = torch.cat([cnn, sg])
    v = F.selu(F.linear(v, torch.from_numpy(W["head0.w"]).double(), torch.from_numpy(W["head0.b"]).double()))
    v = F.linear(v, torch.from_numpy(W["head1.w"]).double(), torch.from_numpy(W["head1.b"]).double())
    np.testing.assert_allclose(a, float(v[0]), rtol=1e-10, atol=1e-10)
