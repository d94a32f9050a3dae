"""Model descriptions and workload recipes for Coherent Fusion pose scoring.

A model description is a plain dict; the CUDA path converts it to the C
struct ``fusion_model_desc`` and the oracle reads it directly.  Nothing here
computes any part of the method.

Architecture readings (the paper gives the components, Fig. 1 and Tables
I-V, but defers voxel sizing, atom propagation and layer equations to the
earlier FAST work):

* 3D-CNN: same-padded convolutions with bias and ReLU, optional residual
  blocks y = x + ReLU(conv(x)), a 2^3 max-pool and one dense layer + ReLU
  (Section 3.3.1, Table III; no batch norm).
* SG-CNN: PotentialNet-style gated graph convolution (Section 3.3.1, Table II):
  GRU-updated message passing over covalent and non-covalent edges found by
  distance cutoff, optional per-node gate between stages, and a sum over
  ligand atoms.
* Fusion head: concatenated latents through dense layers with SELU
  (Section 3.3.3, Table V); dropout is the identity at inference.
* Fusion variants (Section 2.2): "coherent" (the head above), "mid" (Mid-level
  Fusion: model-specific dense layers with SELU on each latent, concatenated
  with the latents themselves, then the fusion layers) and "late" (Late Fusion:
  the mean of the two branches' own affinity outputs, each a dense stack with
  ReLU between layers and a linear last layer of width 1).  ``head_residual``:
  a hidden fusion layer whose input and output widths match adds its input,
  y = x + SELU(W x + b) (the Mid-level model's residual fusion layers, Table IV).
"""

from __future__ import annotations

import copy

EDGE_COV = 1
EDGE_NC = 2

N_FEAT = 19


def _conv(c_in, c_out, k, stride=1, residual=0):
    return dict(c_in=c_in, c_out=c_out, k=k, stride=stride, residual=residual)


# Small single-pose model: 24^3 grid, conv 19->32 (5^3), one residual 32->32
# (5^3) block, 2^3 max-pool, dense 64; two gated graph steps (hidden 32) over
# both edge types, ligand sum-pool to 64; head 128 -> 64 -> 1.
FUSION_TINY = dict(
    name="fusion-24grid-c32",
    n_feat=N_FEAT,
    grid_n=24, grid_h=1.0, sigma=1.0, support=3,
    conv=[_conv(19, 32, 5), _conv(32, 32, 5, residual=1)],
    pool=2,
    cnn_dense=64,
    sg_hidden=32,
    sg_stages=[dict(steps=2, edges=EDGE_COV | EDGE_NC)],
    sg_gate=0,
    sg_gather="linear",
    sg_gather_width=64,
    cut_cov=1.6, cut_nc=4.5,
    head=[64, 1],
    fusion="coherent", cnn_out=[], sg_out=[], head_residual=0,
    dtype="f32",
)

# Full-size model: 48^3 x 19 grid at 1 A; conv 19->64 (7^3), two residual
# 64-channel 7^3 blocks, conv 64->128 (5^3, stride 2), 2^3 pool, dense 256;
# 3 covalent gated steps, per-node gate, 3 covalent+non-covalent steps at
# hidden 64, gated ligand pooling to 128; head 384 -> 256 -> 64 -> 1.
FUSION_FULL = dict(
    name="fusion-48grid-c64",
    n_feat=N_FEAT,
    grid_n=48, grid_h=1.0, sigma=1.0, support=3,
    conv=[_conv(19, 64, 7), _conv(64, 64, 7, residual=1),
          _conv(64, 64, 7, residual=1), _conv(64, 128, 5, stride=2)],
    pool=2,
    cnn_dense=256,
    sg_hidden=64,
    sg_stages=[dict(steps=3, edges=EDGE_COV), dict(steps=3, edges=EDGE_COV | EDGE_NC)],
    sg_gate=1,
    sg_gather="gated",
    sg_gather_width=128,
    cut_cov=1.6, cut_nc=4.5,
    head=[256, 64, 1],
    fusion="coherent", cnn_out=[], sg_out=[], head_residual=0,
    dtype="f32",
)

# Same structure as the full-size model at a size the oracle finishes in a
# second: a 20^3 grid (not a multiple of any tile edge), 3^3 kernels, a
# strided conv, a stage gate and gated gather.  Used for ragged-tail parity.
FUSION_RAGGED = dict(
    name="fusion-20grid-ragged",
    n_feat=N_FEAT,
    grid_n=20, grid_h=1.0, sigma=1.0, support=3,
    conv=[_conv(19, 32, 3), _conv(32, 32, 3, residual=1), _conv(32, 64, 3, stride=2)],
    pool=2,
    cnn_dense=32,
    sg_hidden=32,
    sg_stages=[dict(steps=2, edges=EDGE_COV), dict(steps=1, edges=EDGE_COV | EDGE_NC)],
    sg_gate=1,
    sg_gather="gated",
    sg_gather_width=24,
    cut_cov=1.6, cut_nc=4.5,
    head=[32, 16, 1],
    fusion="coherent", cnn_out=[], sg_out=[], head_residual=0,
    dtype="f32",
)

# The architecture of the final models in Tables II, III and V: 3D-CNN with
# 32 then 64 filters, 5^3 then 3^3 kernels, residual option 2, dense 128 then
# 128 / 2 = 64 (Section 3.3.1), whose output is the CNN latent (Layer^{M-1},
# Section 2.2); SG-CNN (PotentialNet): a covalent stage of K=6 steps at 2.24 A
# on the 19 atom features, gated to the covalent gather width 24, then a
# non-covalent stage of K=3 steps at 5.22 A at width 24 over both edge types,
# gated and summed over the ligand to the non-covalent gather width 128 (the SG
# latent, Layer^{N-3}); four SELU fusion layers.  Grid 48^3 at 1 A.  The graph
# kernels carry both stages at width 32.
FUSION_PAPER = dict(
    name="fusion-paper-final",
    n_feat=N_FEAT,
    grid_n=48, grid_h=1.0, sigma=1.0, support=3,
    conv=[_conv(19, 32, 5), _conv(32, 32, 5, residual=1),
          _conv(32, 64, 3, stride=2), _conv(64, 64, 3, residual=1)],
    pool=2,
    cnn_dense=128,
    cnn_dense2=64,
    sg_hidden=32,
    sg_width=[19, 24],
    sg_stages=[dict(steps=6, edges=EDGE_COV), dict(steps=3, edges=EDGE_COV | EDGE_NC)],
    sg_gate=1,
    sg_gather="gated",
    sg_gather_width=128,
    cut_cov=2.24, cut_nc=5.22,
    head=[128, 64, 24, 1],
    fusion="coherent", cnn_out=[], sg_out=[], head_residual=0,
    dtype="f32",
)


def _variant(base: dict, name: str, **kw) -> dict:
    d = copy.deepcopy(base)
    d.update(name=name, **kw)
    return d


# The earlier fusion forms on the same branches: Mid-level Fusion (model-specific dense layers, their
# outputs concatenated with the latents, residual fusion layers; Table IV has 5 fusion layers) and
# Late Fusion (mean of the two branches' own outputs).
FUSION_TINY_MID = _variant(FUSION_TINY, "fusion-24grid-c32-mid", fusion="mid", cnn_out=[32], sg_out=[32],
                           head=[96, 96, 1], head_residual=1)
FUSION_TINY_LATE = _variant(FUSION_TINY, "fusion-24grid-c32-late", fusion="late", cnn_out=[32, 1],
                            sg_out=[32, 1], head=[])
FUSION_FULL_MID = _variant(FUSION_FULL, "fusion-48grid-c64-mid", fusion="mid", cnn_out=[128], sg_out=[64],
                           head=[256, 256, 128, 128, 1], head_residual=1)
FUSION_FULL_LATE = _variant(FUSION_FULL, "fusion-48grid-c64-late", fusion="late", cnn_out=[64, 1],
                            sg_out=[64, 1], head=[])

# The paper-final branches in the earlier fusion forms.  Late Fusion: each model's own output layers on its
# latent, the 3D-CNN's output layer (64 -> 1) and the SG-CNN's dense layers reduced from the gather width by a
# factor of 1.5 and then 2 (128 -> 85 -> 42, Section 3.3.1) before its output layer.  Mid-level Fusion (Table
# IV): model-specific dense layers, their outputs concatenated after the latents, five residual fusion layers
# (the widths are not given in the paper; chosen here).
FUSION_PAPER_LATE = _variant(FUSION_PAPER, "fusion-paper-final-late", fusion="late", cnn_out=[1],
                             sg_out=[85, 42, 1], head=[])
FUSION_PAPER_MID = _variant(FUSION_PAPER, "fusion-paper-final-mid", fusion="mid", cnn_out=[32], sg_out=[64],
                            head=[288, 288, 128, 128, 1], head_residual=1)

MODELS = {m["name"]: m for m in (FUSION_TINY, FUSION_FULL, FUSION_RAGGED, FUSION_PAPER, FUSION_TINY_MID,
                                 FUSION_TINY_LATE, FUSION_FULL_MID, FUSION_FULL_LATE, FUSION_PAPER_LATE,
                                 FUSION_PAPER_MID)}


def model(name: str, dtype: str | None = None) -> dict:
    """A deep copy of a preset, optionally with another compute dtype."""
    d = copy.deepcopy(MODELS[name])
    if dtype is not None:
        d["dtype"] = dtype
    return d


# Workload recipes.  Each pose p is generated from its own seed; atom counts
# are drawn from that pose's generator inside the stated ranges.
WORKLOADS = {
    # one pose, seed 0: 24 ligand atoms (2 rings) and 200 pocket atoms
    "pose1-lig24-pocket200": dict(seeds=[0], n_lig=(24, 24), n_pocket=(200, 200), rings=2),
    # batch of 64 poses, seeds 1..64, ligands 20-50, pockets 300-600
    "batch64-lig20to50-pocket300to600": dict(seeds=list(range(1, 65)), n_lig=(20, 50),
                                             n_pocket=(300, 600), rings=None),
    # batch of 256 poses, ligands 15-60, pockets 250-800
    "batch256-lig15to60-pocket250to800": dict(seeds=list(range(1001, 1257)), n_lig=(15, 60),
                                              n_pocket=(250, 800), rings=None),
}
