"""The stored oracle values the GPU tests compare against are current (CPU).

Each file under ``tests/golden/`` was written by ``make_golden.py`` from the
oracle and the seeded generators.  Its inputs must still be the ones the
generators make here (same digest), and the single-pose file is recomputed
with the oracle and must match to rounding.  Without that, an oracle change
that was not followed by regenerating the files would leave the GPU parity
tests checking against stale numbers.  The full-size files take about a
minute per pose in the oracle, so only their inputs are checked here.
"""

import json
import os

import numpy as np
import pytest

from oracle import fusion_oracle as O
from synth import configs, poses, weights

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")

pytest.importorskip("scipy")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(GOLDEN) if f.endswith(".json")))
def test_stored_inputs_are_the_generators_current_output(name):
    g = _load(name)
    assert g["model"] in configs.MODELS and g["workload"] in configs.WORKLOADS
    batch = poses.make_batch(configs.WORKLOADS[g["workload"]])
    assert g["input_digest"] == poses.digest(batch), f"{name}: regenerate with tests/golden/make_golden.py"
    n = len(batch["n_lig"])
    assert all(0 <= int(p) < n for p in g["poses"])


def test_single_pose_values_match_the_oracle_as_it_stands():
    g = _load("tiny1_w0.json")
    desc = configs.model(g["model"])
    W = weights.init_weights(desc, g["weights_seed"])
    batch = poses.make_batch(configs.WORKLOADS[g["workload"]])
    for p, want in g["poses"].items():
        st = {}
        xyz, feat, n_lig = poses.pose_slice(batch, int(p))
        got = O.score_pose(desc, W, xyz, feat, n_lig, stages=st)
        assert got == pytest.approx(want["affinity"], abs=1e-12, rel=1e-12)
        np.testing.assert_allclose(st["cnn_latent"], want["cnn_latent"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(st["sg_latent"], want["sg_latent"], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(np.asarray(st["origin"], dtype=np.float64), want["origin"])
