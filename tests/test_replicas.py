"""Replica sharding and the end-of-job gather, on CPU with 2 gloo ranks."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2104_04547_gb300.replicas import shard_range


@pytest.mark.parametrize("n,world", [(64, 1), (64, 2), (7, 3), (2, 4), (0, 2), (1000, 8)])
def test_shards_cover_everything_once(n, world):
    seen = []
    sizes = []
    for r in range(world):
        b, e = shard_range(n, r, world)
        seen.extend(range(b, e))
        sizes.append(e - b)
    assert seen == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    import torch.distributed as dist

    from paper_2104_04547_gb300.replicas import gather_affinities, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = shard_range(n, rank, world)
    # each rank "scores" its shard: affinity of pose i = i * 0.5 (a stand-in for the GPU call)
    local = np.arange(b, e, dtype=np.float32) * 0.5
    out = gather_affinities(local, n)
    q.put((rank, out.tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [64, 13])
def test_gather_two_gloo_ranks(n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = (np.arange(n, dtype=np.float32) * 0.5).tolist()
    assert res[0] == expect and res[1] == expect
