"""Error paths through the C ABI on the GPU: bad inputs are rejected with
status codes (host checks, or device flags read back after the call), the
output is left untouched, and the model keeps working afterwards.  Nothing here
faults, traps or hangs the GPU: every failure is a flag or a host check."""

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.fixture(scope="module")
def setup(F):
    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 3)
    blob = weights.to_blob(desc, W)
    m = F.Model(desc, blob, max_poses=4, max_atoms=256, max_degree=64)
    batch = poses.pack([poses.make_pose(s, (10, 20), (40, 80)) for s in (1, 2, 3)])
    ref = m.score(batch).copy()
    return desc, blob, m, batch, ref


def _expect(F, code, fn):
    with pytest.raises(F.FusionError) as e:
        fn()
    assert e.value.code == code, str(e.value)


def test_host_validation(F, setup):
    desc, blob, m, batch, ref = setup
    out = np.full(3, 7.0, dtype=np.float32)
    bad = {k: v.copy() for k, v in batch.items()}
    bad["xyz"][5, 1] = np.nan
    _expect(F, F.FUSION_EINVAL, lambda: m.score(bad, out=out))
    bad = {k: v.copy() for k, v in batch.items()}
    bad["n_lig"][1] = 10_000
    _expect(F, F.FUSION_EINVAL, lambda: m.score(bad, out=out))
    bad = {k: v.copy() for k, v in batch.items()}
    bad["n_lig"][0] = 0
    _expect(F, F.FUSION_EINVAL, lambda: m.score(bad, out=out))
    big = poses.pack([poses.make_pose(9, (30, 30), (300, 300))])
    _expect(F, F.FUSION_EINVAL, lambda: m.score(big, out=np.zeros(1, np.float32)))
    five = poses.pack([poses.make_pose(s, (5, 8), (5, 10)) for s in range(5)])
    _expect(F, F.FUSION_EINVAL, lambda: m.score(five, out=np.zeros(5, np.float32)))
    assert np.all(out == 7.0)
    np.testing.assert_array_equal(m.score(batch), ref)


def test_device_flags(F, setup):
    import torch
    desc, blob, m, batch, ref = setup
    bad = {k: v.copy() for k, v in batch.items()}
    bad["xyz"][7, 2] = np.inf
    bad["n_lig"][2] = 999
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in bad.items()}
    out = torch.full((3,), 7.0, device="cuda")
    _expect(F, F.FUSION_EINVAL, lambda: m.score(dev, out=out, on_device=True))
    assert torch.all(out == 7.0)
    np.testing.assert_array_equal(m.score(batch), ref)


def test_edge_capacity_flag(F, setup):
    desc, blob, m, batch, ref = setup
    small = F.Model(desc, blob, max_poses=4, max_atoms=256, max_degree=2)
    _expect(F, F.FUSION_ECAPACITY, lambda: small.score(batch))
    small.close()


def test_create_errors(F, setup):
    desc, blob, m, batch, ref = setup
    _expect(F, F.FUSION_EWEIGHTS, lambda: F.Model(desc, blob[:-4], max_poses=2))
    d2 = configs.model("fusion-20grid-ragged")
    d2["conv"][0]["c_out"] = 48
    with pytest.raises(F.FusionError) as e:
        F.Model(d2, blob, max_poses=2)
    assert e.value.code == F.FUSION_EINVAL


def test_empty_batch_is_noop(F, setup):
    desc, blob, m, batch, ref = setup
    empty = dict(atom_off=np.zeros(1, np.int32), n_lig=np.zeros(0, np.int32),
                 xyz=np.zeros((0, 3), np.float32), feat=np.zeros((0, 19), np.float32))
    out = m.score(empty, n_poses=0, out=np.zeros(0, np.float32))
    assert out.shape == (0,)
    np.testing.assert_array_equal(m.score(batch), ref)


def test_atoms_outside_grid_and_single_atom_ligand(F):
    from oracle import fusion_oracle as O
    desc = configs.model("fusion-20grid-ragged")
    W = weights.init_weights(desc, 3)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=256)
    xyz, feat, n_lig = poses.make_pose(4, (12, 12), (60, 60))
    far = xyz.copy()
    far[n_lig:] += np.float32(60.0)          # pocket far outside the grid
    one = (xyz[:1].copy(), feat[:1].copy(), 1)  # a single-atom ligand, no pocket
    b = poses.pack([(far, feat, n_lig), one])
    got = m.score(b)
    for p in range(2):
        x, f, nl = poses.pose_slice(b, p)
        exp = O.score_pose(desc, W, x, f, nl)
        assert abs(float(got[p]) - exp) <= 1e-4, (p, got[p], exp)


def test_bounded_wait_runs_out_and_model_recovers(F):
    """Failure detection without a fault: the first conv launch of the next call is armed to load
    nothing, so its bounded waits run out; the call returns FUSION_ETIMEOUT within a few seconds, the
    output is untouched, and the next call gives the normal result."""
    import time
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 3)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=256)
    batch = poses.pack([poses.make_pose(s, (10, 20), (40, 80)) for s in (1, 2, 3)])
    ref = m.score(batch).copy()
    F.fusion_set_option(m.handle, F.FUSION_OPT_TEST_WAIT_TIMEOUT, 1)
    out = np.full(3, 7.0, dtype=np.float32)
    t0 = time.perf_counter()
    _expect(F, F.FUSION_ETIMEOUT, lambda: m.score(batch, out=out))
    assert time.perf_counter() - t0 < 10.0
    assert np.all(out == 7.0)
    np.testing.assert_array_equal(m.score(batch), ref)
    m.use_cuda_graphs(True)
    _expect(F, F.FUSION_EUNSUPPORTED, lambda: F.fusion_set_option(m.handle, F.FUSION_OPT_TEST_WAIT_TIMEOUT, 1))
    m.close()


def test_graph_bounded_wait_runs_out_and_model_recovers(F):
    """The same for the tensor-core graph convolution: the next call's first graph launch issues no weight
    copy, its bounded wait runs out and sets the timeout flag (the later graph launches see the flag and give
    up at once); the call returns FUSION_ETIMEOUT with the output untouched and the next call is normal."""
    import time
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(configs.model("fusion-20grid-ragged"), 3)
    m = F.Model(desc, weights.to_blob(desc, W), max_poses=4, max_atoms=256)
    batch = poses.pack([poses.make_pose(s, (10, 20), (40, 80)) for s in (1, 2, 3)])
    ref = m.score(batch).copy()
    F.fusion_set_option(m.handle, F.FUSION_OPT_TEST_WAIT_TIMEOUT, 2)
    # an armed test keeps CUDA graphs off (a capture would replay the stalled launch)
    _expect(F, F.FUSION_EUNSUPPORTED, lambda: m.use_cuda_graphs(True))
    out = np.full(3, 7.0, dtype=np.float32)
    t0 = time.perf_counter()
    _expect(F, F.FUSION_ETIMEOUT, lambda: m.score(batch, out=out))
    assert time.perf_counter() - t0 < 10.0
    assert np.all(out == 7.0)
    np.testing.assert_array_equal(m.score(batch), ref)
    _expect(F, F.FUSION_EINVAL, lambda: F.fusion_set_option(m.handle, F.FUSION_OPT_TEST_WAIT_TIMEOUT, 3))
    m.graph_tensor_cores(0)
    _expect(F, F.FUSION_EUNSUPPORTED, lambda: F.fusion_set_option(m.handle, F.FUSION_OPT_TEST_WAIT_TIMEOUT, 2))
    m.close()
