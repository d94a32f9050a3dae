"""CUDA-graph replay and the conv tile autotuner give bit-identical results to
plain launches (same kernels, same per-output reduction order), for each
dtype, several batch sizes (graph cache hits and misses) and device inputs."""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.fixture(scope="module")
def pool():
    return poses.make_uneven_pool(2, 6, seed0=4242)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_graph_replay_matches_plain_launches(F, pool, dtype):
    import torch
    desc = configs.model("fusion-20grid-ragged", dtype=dtype)
    blob = weights.to_blob(desc, weights.init_weights(desc, 9))
    m = F.Model(desc, blob, max_poses=8, max_atoms=1200)
    batches = [poses.pack(pool[0:5]), poses.pack(pool[5:8]), poses.pack(pool[8:12]), poses.pack(pool[0:5])]
    plain = [m.score(b).copy() for b in batches]
    m.use_cuda_graphs(True)
    graph = [m.score(b).copy() for b in batches]
    for a, b in zip(plain, graph):
        np.testing.assert_array_equal(a, b)
    assert m.timings()["total"] > 0.0
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in batches[1].items()}
    out = torch.empty(3, device="cuda")
    m.score(dev, n_poses=3, out=out, on_device=True)
    np.testing.assert_array_equal(out.cpu().numpy(), plain[1])
    m.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_autotune_keeps_results(F, pool, dtype):
    desc = configs.model("fusion-20grid-ragged", dtype=dtype)
    blob = weights.to_blob(desc, weights.init_weights(desc, 9))
    m = F.Model(desc, blob, max_poses=8, max_atoms=1200)
    b = poses.pack(pool[:8])
    before = m.score(b).copy()
    m.autotune(b)
    tiles = m.conv_tiles()
    assert all(t["slices_per_cta"] in (2, 4, 8) and t["stages"] >= 2 and t["smem_bytes"] <= 227 * 1024
               for t in tiles)
    np.testing.assert_array_equal(m.score(b), before)
    m.use_cuda_graphs(True)
    np.testing.assert_array_equal(m.score(b), before)
    m.close()


def test_autotune_rejects_fp32(F, pool):
    desc = configs.model("fusion-20grid-ragged", dtype="f32")
    blob = weights.to_blob(desc, weights.init_weights(desc, 9))
    m = F.Model(desc, blob, max_poses=8, max_atoms=1200)
    with pytest.raises(F.FusionError) as e:
        m.autotune(poses.pack(pool[:2]))
    assert e.value.code == F.FUSION_EUNSUPPORTED
    m.close()
