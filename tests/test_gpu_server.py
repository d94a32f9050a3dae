"""Continuous-batching server through the C ABI: every pose's result is the
same as scoring that pose alone, whatever mix of uneven poses (and, in a
server with BF16 and FP8 slots, of dtypes) it was batched with; bad poses are
rejected at submission; a full queue answers EAGAIN; a result is collected
once; the HBM budget limits the slots."""

import time

import numpy as np
import pytest

from gpu_common import require_gpu
from synth import configs, poses, weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    return require_gpu()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_results_same_alone_and_in_the_mix(F, dtype):
    desc = configs.model("fusion-20grid-ragged", dtype=dtype)
    W = weights.init_weights(desc, 5)
    blob = weights.to_blob(desc, W)
    pool = poses.make_uneven_pool(3, 8, seed0=777)
    srv = F.Server(desc, blob, max_batch=8, slots=2, batch_window_us=500.0, max_atoms=1200)
    rng = np.random.default_rng(0)
    tickets = []
    for i, (x, f, nl) in enumerate(pool):
        tickets.append(srv.submit(x, f, nl))
        if rng.random() < 0.3:
            time.sleep(rng.random() * 0.003)     # ragged arrivals -> varied batch mixes
    srv.drain()
    got = []
    for t in tickets:
        r = srv.poll(t)
        assert r is not None
        got.append(r[0])
    st = srv.stats()
    assert st["completed"] == len(pool) and st["failed"] == 0 and st["batches"] >= 3
    srv.close()
    m = F.Model(desc, blob, max_poses=1, max_atoms=1200)
    alone = np.array([m.score(poses.pack([p]))[0] for p in pool])
    np.testing.assert_array_equal(np.array(got, dtype=np.float32), alone)


def test_mixed_dtype_server_results_same_alone(F):
    """One server with BF16 and FP8 slots (the serving workload mixes the two): each request names its dtype,
    and every result equals that pose scored alone by a model of that dtype, bit for bit."""
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(desc, 5)
    blob = weights.to_blob(desc, W)
    pool = poses.make_uneven_pool(3, 8, seed0=778)
    srv = F.Server(desc, blob, max_batch=8, slots=4, batch_window_us=500.0, max_atoms=1200, dtypes=("fp8",))
    st = srv.stats()
    assert st["slots"] == 4 and st["slots_by_dtype"] == {"f32": 0, "bf16": 2, "fp8": 2}
    with pytest.raises(F.FusionError) as e:
        srv.submit(*pool[0], dtype="f32")            # no FP32 slots in this server
    assert e.value.code == F.FUSION_EINVAL
    rng = np.random.default_rng(1)
    order = [(i, "bf16" if rng.random() < 0.5 else "fp8") for i in range(len(pool))]
    order += [(i, "fp8" if dt == "bf16" else "bf16") for i, dt in order[::3]]   # some poses in both dtypes
    tickets = []
    for i, dt in order:
        tickets.append(srv.submit(*pool[i], dtype=dt))
        if rng.random() < 0.3:
            time.sleep(rng.random() * 0.003)
    srv.drain()
    got = [srv.poll(t)[0] for t in tickets]
    assert srv.stats()["completed"] == len(order)
    srv.close()
    alone = {}
    for dt in ("bf16", "fp8"):
        d = configs.model("fusion-20grid-ragged", dtype=dt)
        m = F.Model(d, weights.to_blob(d, W), max_poses=1, max_atoms=1200)
        alone[dt] = [float(m.score(poses.pack([p]))[0]) for p in pool]
        m.close()
    for (i, dt), g in zip(order, got):
        assert np.float32(g) == np.float32(alone[dt][i]), (i, dt, g, alone[dt][i])


def test_rejections_and_queue_capacity(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    W = weights.init_weights(desc, 5)
    blob = weights.to_blob(desc, W)
    srv = F.Server(desc, blob, max_batch=64, slots=1, batch_window_us=3e6, queue_capacity=3, max_atoms=300)
    x, f, nl = poses.make_pose(3, (10, 12), (40, 60))
    bad = x.copy()
    bad[2, 0] = np.nan
    with pytest.raises(F.FusionError) as e:
        srv.submit(bad, f, nl)
    assert e.value.code == F.FUSION_EINVAL
    with pytest.raises(F.FusionError):
        srv.submit(x, f, len(x) + 1)
    big = poses.make_pose(4, (20, 20), (400, 400))
    with pytest.raises(F.FusionError):
        srv.submit(*big)
    t = [srv.submit(x, f, nl) for _ in range(3)]
    assert all(v is not None for v in t)
    assert srv.submit(x, f, nl) is None          # queue full while the slot waits to fill its batch
    srv.drain(timeout_s=30.0)
    vals = [srv.poll(v)[0] for v in t]
    assert vals[0] == vals[1] == vals[2]
    # a result is handed out once: polling a collected ticket again is an error, not a pending result
    with pytest.raises(F.FusionError) as e:
        srv.poll(t[0])
    assert e.value.code == F.FUSION_EINVAL and "already collected" in str(e.value)
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_hbm_budget_limits_slots(F):
    desc = configs.model("fusion-20grid-ragged", dtype="bf16")
    blob = weights.to_blob(desc, weights.init_weights(desc, 5))
    one = F.Server(desc, blob, max_batch=8, slots=4, max_atoms=300)
    per_slot = one.stats()["slot_bytes"]
    assert one.stats()["slots"] == 4 and per_slot > 0
    one.close()
    two = F.Server(desc, blob, max_batch=8, slots=4, hbm_budget_bytes=int(2.5 * per_slot), max_atoms=300)
    assert two.stats()["slots"] == 2
    two.close()
    with pytest.raises(F.FusionError) as e:
        F.Server(desc, blob, max_batch=8, slots=1, hbm_budget_bytes=per_slot // 4, max_atoms=300)
    assert e.value.code == F.FUSION_ENOMEM
