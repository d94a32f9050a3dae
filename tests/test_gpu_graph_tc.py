"""Gated graph convolution on the tensor cores (FUSION_OPT_GRAPH_TENSOR_CORES, Section 3.3.1's gated graph
convolution).

The stage gate, the GRU updates and the edge transforms run as three BF16 MMAs per product: each operand x is
split into x_hi = bf16(x) and x_lo = bf16(x - x_hi), and x y = x_lo y_hi + x_hi y_lo + x_hi y_hi with FP32
accumulation.  What is dropped (x_lo y_lo and the remainders of both splits) is at most about 3 * 2^-16
(4.6e-5) of |x y| per term, and a dot product over K <= 64 inputs errs by a few 1e-6 of the sum of its
|terms| (the rounding errors cancel).  Node states are bounded by 1 (a GRU's h' is a convex mix of tanh and
h); the message sums add up to ~60 transforms and the errors carry through the stage gate and up to 9
steps.  Measured worst node-state deviations from the FP32 CUDA-core graph: 1.4e-4 (full-size model, 6
steps) and 9.0e-4 (paper-final model, 9 steps, 160 poses); STATE_TOL = 2e-3 keeps 2x room.  A product with
a term missing, or plain BF16 products, errs by over 100x more per dot product (tests/test_split_bf16.py
checks both figures on the CPU), and a gate out of order or a missing bias moves states by far more.

* FP32 full-size model (H = 64) on the 64-pose workload with the graph on the tensor cores: every pose's
  SG latent against the stored FP64 oracle values, the affinities within 1e-3 of them; the same batch on
  the FP32 CUDA-core graph: node states within STATE_TOL, CNN latents bit-identical (the branches are
  independent);
* the ragged model (H = 32, gate, gated gather) on a mixed batch: SG latent against the oracle per pose;
* the paper-final model at 160 poses (more 128-node tiles than the kernel's persistent CTAs, so CTAs loop):
  node states within STATE_TOL of the CUDA-core graph's, and a pose alone scores as in the batch;
* option values.
"""

import numpy as np
import pytest

from gpu_common import golden, require_gpu
from oracle import fusion_oracle as O
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu

STATE_TOL = 2e-3      # node states (|h| <= 1), tensor-core graph against the FP32 CUDA-core graph
LATENT_TOL = 1e-3     # SG latent (a sum over up to 60 ligand atoms) against the FP64 oracle, abs + rel
AFF_TOL = 1e-3


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _states(F, m, n):
    return [m.fetch(F.STAGE_SG_STATE, p).copy() for p in range(n)]


def test_full_size_f32_on_tensor_cores(F):
    desc = configs.model("fusion-48grid-c64")
    W = weights.init_weights(desc, 0)
    batch = poses.make_batch(configs.WORKLOADS["batch64-lig20to50-pocket300to600"])
    g = golden("full64_w0.json")
    assert g["input_digest"] == poses.digest(batch)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=64, max_atoms=1200, keep_stages=True)
    ref = m.score(batch).copy()
    ref_state = _states(F, m, 64)
    ref_cnn = [m.fetch(F.STAGE_CNN_LATENT, p).copy() for p in range(64)]
    m.graph_tensor_cores(1)
    got = m.score(batch).copy()
    state = _states(F, m, 64)
    d_state = max(float(np.abs(state[p] - ref_state[p]).max()) for p in range(64))
    idx = [int(k) for k in g["poses"]]
    lat_err = []
    for k, v in g["poses"].items():
        p = int(k)
        sg = m.fetch(F.STAGE_SG_LATENT, p)
        np.testing.assert_allclose(sg, v["sg_latent"], rtol=LATENT_TOL, atol=LATENT_TOL, err_msg=f"pose {p}")
        lat_err.append(float(np.abs(sg - np.asarray(v["sg_latent"])).max()))
        np.testing.assert_array_equal(m.fetch(F.STAGE_CNN_LATENT, p), ref_cnn[p])
    d_aff = np.abs(got[idx] - np.array([g["poses"][str(i)]["affinity"] for i in idx]))
    print(f"graph on tensor cores, H=64: max |d state| vs CUDA cores {d_state:.2e}; SG latent vs FP64 oracle "
          f"max {max(lat_err):.2e}; affinity vs oracle mean {d_aff.mean():.2e} max {d_aff.max():.2e}; "
          f"vs CUDA-core graph max {np.abs(got - ref).max():.2e}")
    assert d_state <= STATE_TOL
    assert d_aff.max() <= AFF_TOL
    m.close()


def test_ragged_model_on_tensor_cores(F):
    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 7)
    specs = [(101, (20, 30), (60, 120)), (102, (8, 12), (20, 40)), (103, (30, 40), (150, 200)),
             (104, (5, 5), (0, 0)), (105, (15, 25), (80, 100))]
    batch = poses.pack([poses.make_pose(s, a, b) for s, a, b in specs])
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512, keep_stages=True)
    m.graph_tensor_cores(1)
    got = m.score(batch).copy()
    worst = 0.0
    for p in range(len(specs)):
        xyz, feat, n_lig = poses.pose_slice(batch, p)
        st = {}
        exp = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
        sg = m.fetch(F.STAGE_SG_LATENT, p)
        np.testing.assert_allclose(sg, st["sg_latent"], rtol=LATENT_TOL, atol=LATENT_TOL, err_msg=f"pose {p}")
        worst = max(worst, float(np.abs(sg - st["sg_latent"]).max()))
        assert abs(float(got[p]) - exp) <= AFF_TOL, (p, got[p], exp)
    print(f"graph on tensor cores, H=32 ragged: SG latent vs FP64 oracle max {worst:.2e}")
    m.close()


def test_paper_final_many_tiles(F):
    desc = configs.model("fusion-paper-final", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-paper-final"), 1)
    wl = dict(configs.WORKLOADS["batch256-lig15to60-pocket250to800"])
    wl["seeds"] = wl["seeds"][:160]
    batch = poses.make_batch(wl)
    A = int(batch["atom_off"][-1]) if "atom_off" in batch else None
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=160, max_atoms=1200, keep_stages=True)
    tc = m.score(batch).copy()
    tc_state = _states(F, m, 160)
    alone = m.score(poses.subset(batch, [117]))[0]
    m.graph_tensor_cores(0)
    simt = m.score(batch).copy()
    simt_state = _states(F, m, 160)
    m.close()
    d_state = max(float(np.abs(tc_state[p] - simt_state[p]).max()) for p in range(160))
    print(f"paper-final, 160 poses ({A} atoms): max |d state| {d_state:.2e}, "
          f"max |d affinity| {np.abs(tc - simt).max():.2e}")
    assert d_state <= STATE_TOL
    assert np.abs(tc - simt).max() <= AFF_TOL
    assert alone == tc[117]


def test_option_values(F):
    desc = configs.model("fusion-24grid-c32", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-24grid-c32"), 0)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=2, max_atoms=256)
    for v in (-1, 0, 1):
        m.graph_tensor_cores(v)
    for bad in (2, -2):
        with pytest.raises(F.FusionError):
            m.graph_tensor_cores(bad)
    m.close()
