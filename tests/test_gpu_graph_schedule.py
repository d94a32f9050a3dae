"""Graph-convolution schedules: 1, 2, 4 or 8 nodes per warp (FUSION_OPT_GRAPH_NODES_PER_WARP).

Each node's sums keep the order of a warp per node whatever the schedule, so on the FP32 and BF16 paths
the affinities and the final node states of a mixed batch must be bit-identical across the four values;
the autotuner must pick one of them and leave the scores unchanged.
"""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


def _batch():
    specs = [(201, (20, 30), (60, 120)), (202, (8, 12), (20, 40)), (203, (30, 40), (150, 200)),
             (204, (5, 5), (0, 0)), (205, (15, 25), (80, 100))]
    return poses.pack([poses.make_pose(s, a, b) for s, a, b in specs])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_nodes_per_warp_bit_identical(F, dtype):
    desc = configs.model("fusion-20grid-ragged", dtype=dtype)
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 4)
    batch = _batch()
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512, keep_stages=True)
    ref, ref_state = None, None
    for npw in (1, 2, 4, 8):
        assert m.graph_nodes_per_warp(npw) == npw
        got = m.score(batch).copy()
        state = [m.fetch(F.STAGE_SG_STATE, p).copy() for p in range(len(batch["n_lig"]))]
        if ref is None:
            ref, ref_state = got, state
        else:
            np.testing.assert_array_equal(got, ref, err_msg=f"{npw} nodes per warp")
            for p in range(len(state)):
                np.testing.assert_array_equal(state[p], ref_state[p], err_msg=f"pose {p}, {npw} nodes per warp")
    # the default: 2 with the graph on the tensor cores (BF16), 4 on the CUDA cores (FP32); it follows the
    # graph mode while the caller has not chosen a value
    assert m.graph_nodes_per_warp(-1) == (2 if dtype == "bf16" else 4)
    m.graph_tensor_cores(0 if dtype == "bf16" else 1)
    assert m.graph_nodes_per_warp() == (4 if dtype == "bf16" else 2)
    m.graph_tensor_cores(-1)
    assert m.graph_nodes_per_warp() == (2 if dtype == "bf16" else 4)
    with pytest.raises(F.FusionError):
        m.graph_nodes_per_warp(3)
    m.close()


def test_autotune_picks_a_schedule(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 4)
    batch = _batch()
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=8, max_atoms=512)
    before = m.score(batch).copy()
    m.autotune(batch)
    assert m.graph_nodes_per_warp() in (1, 2, 4, 8)
    np.testing.assert_array_equal(m.score(batch), before)
    m.close()
