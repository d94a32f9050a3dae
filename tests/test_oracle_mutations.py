"""The oracle's pins catch plausible mistakes (CPU).

Each case plants one mistake in a copy of the oracle's source (a sign, an index, an order, a constant, a
missing factor or term), puts the mutated functions in place of the oracle's for the duration of the test,
runs the pins that should notice, and requires at least one of them to fail.  The pins themselves are the
tests of `test_oracle_*.py`, called with one of their parameter sets.
"""

import inspect

import pytest

import test_oracle_cnn as cnn_pins
import test_oracle_fusion_forms as forms_pins
import test_oracle_graph as graph_pins
import test_oracle_sgcnn as sg_pins
import test_oracle_voxelize as vox_pins
from oracle import fusion_oracle as O

pytest.importorskip("torch")
pytest.importorskip("scipy")

# (name, [(text in the oracle, replacement)], pins: callables that should fail)
MUTATIONS = [
    ("erf difference with the wrong sign",
     [("return 0.5 * (_erf((lo + h) / s2) - _erf(lo / s2))", "return 0.5 * (_erf((lo + h) / s2) + _erf(lo / s2))")],
     [vox_pins.test_single_atom_at_voxel_centre_matches_quadrature,
      vox_pins.test_mass_equals_cdf_product_for_in_grid_supports]),
    ("voxel edges shifted by half a voxel",
     [("lo = idx * h - d", "lo = (idx + 0.5) * h - d")],
     [vox_pins.test_single_atom_at_voxel_centre_matches_quadrature,
      lambda: vox_pins.test_off_centre_atom_general_spacing(0.5, 1.5, 5)]),
    ("Gaussian width sigma instead of sigma sqrt 2",
     [("s2 = sigma * math.sqrt(2.0)", "s2 = sigma")],
     [vox_pins.test_single_atom_at_voxel_centre_matches_quadrature,
      vox_pins.test_mass_equals_cdf_product_for_in_grid_supports]),
    ("containing voxel rounded instead of floored",
     [("return np.floor(q).astype(np.int64)", "return np.round(q).astype(np.int64)")],
     [vox_pins.test_containing_voxel_on_boundary_and_centroid_rule,
      vox_pins.test_single_atom_at_voxel_centre_matches_quadrature]),
    ("convolution kernel flipped along z",
     [("dot(w[:, :, kd, kh, kw].T)", "dot(w[:, :, k - 1 - kd, kh, kw].T)")],
     [lambda: cnn_pins.test_conv3d_matches_torch_float64(6, 2, 3, 3, 1),
      cnn_pins.test_conv3d_offcentre_delta_shifts_with_zero_padding]),
    ("weights used transposed (input and output channels swapped)",
     [("dot(w[:, :, kd, kh, kw].T)", "dot(w[:, :, kd, kh, kw].T[::-1, ::-1])")],
     [lambda: cnn_pins.test_conv3d_matches_torch_float64(6, 2, 3, 3, 1),
      cnn_pins.test_conv3d_unit_kernel_is_matmul]),
    ("average pooling instead of max",
     [(".max(axis=(1, 3, 5))", ".mean(axis=(1, 3, 5))")],
     [cnn_pins.test_maxpool_matches_torch, lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(0)]),
    ("ReLU after the residual add",
     [("        y = relu(conv3d(x, W[f\"conv{i}.w\"], W[f\"conv{i}.b\"], cv[\"stride\"]))\n        if cv[\"residual\"]:\n            y = x + y",
       "        y = conv3d(x, W[f\"conv{i}.w\"], W[f\"conv{i}.b\"], cv[\"stride\"])\n        if cv[\"residual\"]:\n            y = x + y\n        y = relu(y)")],
     [lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(0)]),
    ("non-strict cutoff",
     [("cov = (s < c2) & off", "cov = (s <= c2) & off"), ("nc = (~cov) & (s < n2) & off", "nc = (~cov) & (s <= n2) & off")],
     [graph_pins.test_boundary_pairs_use_strict_inequality]),
    ("self loops kept",
     [("off = ~np.eye(n, dtype=bool)", "off = np.ones((n, n), dtype=bool)")],
     [graph_pins.test_graph_structure, lambda: graph_pins.test_edges_match_kdtree(0)]),
    ("GRU reset and update gates swapped",
     [("r = sigmoid(gi[:, :H] + gh[:, :H])", "r = sigmoid(gi[:, H:2 * H] + gh[:, H:2 * H])"),
      ("z = sigmoid(gi[:, H:2 * H] + gh[:, H:2 * H])", "z = sigmoid(gi[:, :H] + gh[:, :H])")],
     [sg_pins.test_gru_matches_torch_grucell]),
    ("GRU candidate without the reset gate",
     [("nn = np.tanh(gi[:, 2 * H:] + r * gh[:, 2 * H:])", "nn = np.tanh(gi[:, 2 * H:] + gh[:, 2 * H:])")],
     [sg_pins.test_gru_matches_torch_grucell]),
    ("messages over one edge type only",
     [("for e in _edge_names(st[\"edges\"]):", "for e in _edge_names(st[\"edges\"])[:1]:")],
     [lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-20grid-ragged")]),
    ("gather without its gate",
     [("v = g * (hl @ W[\"gather.wo\"].T + W[\"gather.bo\"])", "v = hl @ W[\"gather.wo\"].T + W[\"gather.bo\"]")],
     [lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-20grid-ragged"),
      sg_pins.test_tiny_network_end_to_end_matches_torch_restatement]),
    ("SELU alpha of another activation",
     [("SELU_ALPHA = 1.6732632423543772848170429916717", "SELU_ALPHA = 1.0")],
     [sg_pins.test_activations_match_torch, sg_pins.test_head_matches_torch]),
    ("Late Fusion summing the two affinities instead of averaging",
     [("return 0.5 * (out[0] + out[1])", "return out[0] + out[1]")],
     [lambda: forms_pins.test_late_fusion_is_mean_of_torch_stacks("fusion-24grid-c32-late"),
      forms_pins.test_late_fusion_constant_branch_pins_the_mean]),
    ("Late Fusion stacks without their ReLU",
     [("                if l + 1 < n:\n                    v = relu(v)", "                pass")],
     [lambda: forms_pins.test_late_fusion_is_mean_of_torch_stacks("fusion-24grid-c32-late")]),
    ("Mid-level branch outputs in front of the latents",
     [("parts = [cnn, sg]", "parts = []"), ("        v = np.concatenate(parts)", "        v = np.concatenate(parts + [cnn, sg])")],
     [lambda: forms_pins.test_mid_fusion_zero_branches_equal_coherent_head_on_leading_columns("fusion-24grid-c32-mid"),
      forms_pins.test_mid_fusion_matches_torch_restatement]),
    ("residual fusion layer without its add",
     [("u = v + u", "u = u")],
     [forms_pins.test_residual_zero_layer_is_identity, forms_pins.test_mid_fusion_matches_torch_restatement]),
    ("latents concatenated in the other order",
     [("    v = np.concatenate([cnn, sg])\n", "    v = np.concatenate([sg, cnn])\n")],
     [sg_pins.test_head_matches_torch, sg_pins.test_tiny_network_end_to_end_matches_torch_restatement]),
    ("convolution without its bias",
     [("y = np.zeros((Do, Ho, Wo, Co)) + np.asarray(b, dtype=np.float64)", "y = np.zeros((Do, Ho, Wo, Co))")],
     [lambda: cnn_pins.test_conv3d_matches_torch_float64(6, 2, 3, 3, 1),
      lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(0)]),
    ("flatten in (D, H, W, C) order instead of (C, D, H, W)",
     [("v = x.transpose(3, 0, 1, 2).reshape(-1)", "v = x.reshape(-1)")],
     [lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(0)]),
    ("stage gate reading h twice instead of [h, h0]",
     [("hh = np.concatenate([h, h0], axis=1)", "hh = np.concatenate([h, h], axis=1)")],
     [lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-20grid-ragged")]),
    ("messages without the edge-transform bias",
     [("T = h @ W[f\"sg{s}.{e}.w\"].T + W[f\"sg{s}.{e}.b\"]", "T = h @ W[f\"sg{s}.{e}.w\"].T")],
     [lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-24grid-c32"),
      sg_pins.test_tiny_network_end_to_end_matches_torch_restatement]),
    ("second CNN dense layer without its ReLU",
     [("out = relu(W[\"cnn_dense2.w\"].astype(np.float64) @ out + W[\"cnn_dense2.b\"])",
       "out = W[\"cnn_dense2.w\"].astype(np.float64) @ out + W[\"cnn_dense2.b\"]")],
     [lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(16)]),
    ("CNN latent taken before the second dense layer",
     [("out = relu(W[\"cnn_dense2.w\"].astype(np.float64) @ out + W[\"cnn_dense2.b\"])", "pass")],
     [lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(16)]),
    ("stage gate reading the padded features in place of the stage's own states",
     [("hh = np.concatenate([h, h0], axis=1)", "hh = np.concatenate([h0, h0], axis=1)")],
     [lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-paper-final")]),
    ("gather over every atom, not only the ligand's",
     [("hl = h[:n_lig]", "hl = h"), ("xl = x_in[:n_lig]", "xl = x_in")],
     [sg_pins.test_zero_steps_linear_gather_closed_form,
      lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-20grid-ragged")]),
    ("gated gather reading the first stage's input instead of the last",
     [("        x_in = h\n        H = widths[s]\n", "        H = widths[s]\n")],
     [lambda: sg_pins.test_sg_branch_matches_dense_adjacency_torch("fusion-20grid-ragged")]),
    ("GRU blend with z and 1 - z swapped",
     [("return (1.0 - z) * nn + z * h", "return z * nn + (1.0 - z) * h")],
     [sg_pins.test_gru_matches_torch_grucell]),
    ("SELU without its scale",
     [("return SELU_SCALE * np.where(x > 0, x,", "return np.where(x > 0, x,")],
     [sg_pins.test_activations_match_torch, sg_pins.test_head_matches_torch]),
    ("non-covalent set also holding the covalent pairs",
     [("nc = (~cov) & (s < n2) & off", "nc = (s < n2) & off")],
     [graph_pins.test_graph_structure, lambda: graph_pins.test_edges_match_kdtree(0)]),
    ("grid centred on the origin instead of on the ligand centroid",
     [("return (c - half).astype(np.float32)", "return c.astype(np.float32)")],
     [vox_pins.test_containing_voxel_on_boundary_and_centroid_rule]),
    ("max-pool window of the first voxel only",
     [(".max(axis=(1, 3, 5))", "[:, 0, :, 0, :, 0]")],
     [cnn_pins.test_maxpool_matches_torch, lambda: cnn_pins.test_cnn_branch_matches_torch_restatement(0)]),
]


def _mutant(subs):
    src = inspect.getsource(O)
    for old, new in subs:
        assert src.count(old) == 1, f"mutation anchor not found exactly once: {old!r}"
        src = src.replace(old, new)
    ns = {"__name__": "oracle_mutant"}
    exec(compile(src, "oracle_mutant", "exec"), ns)
    return ns


@pytest.mark.parametrize("name,subs,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(monkeypatch, name, subs, pins):
    ns = _mutant(subs)
    for key, val in ns.items():
        if key.startswith("__") or not hasattr(O, key):
            continue
        monkeypatch.setattr(O, key, val)
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught >= 1, f"no pin noticed: {name}"


def test_unmutated_oracle_passes_the_same_pins():
    for _, _, pins in MUTATIONS:
        for pin in pins:
            pin()
