"""Replica bookkeeping across ranks on CPU (gloo, world size 2): item
sharding, the C_eff gather on rank 0 and the maximum of the timed region.
The solves themselves need a GPU; here each rank fills its slice with a
value that identifies the item."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2412_11566_gb300.replicas import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_ceff(i):
    return np.full((6, 6), float(i)) + np.eye(6) * 0.5


def _worker(rank, world, port, n_items, q):
    import torch.distributed as dist
    from paper_2412_11566_gb300.replicas import gather_ceff, max_over_ranks, shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = sh(n_items, rank, world)
        local = np.stack([_fake_ceff(i) for i in mine]) if len(mine) else np.zeros((0, 6, 6))
        full = gather_ceff(local, n_items, rank, world)
        tmax = max_over_ranks(1.0 + rank, world)
        q.put((rank, None if full is None else full.tolist(), tmax))
    finally:
        dist.destroy_process_group()


def test_shard_covers_items_once():
    for n in (0, 1, 5, 64):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


@pytest.mark.parametrize("n_items", [5, 1])
def test_gather_and_max_two_ranks(n_items):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_items, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, full, tmax = q.get(timeout=120)
        res[rank] = (full, tmax)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full0, t0 = res[0]
    assert res[1][0] is None
    assert np.array_equal(np.asarray(full0), np.stack([_fake_ceff(i) for i in range(n_items)]))
    assert t0 == 2.0 and res[1][1] == 2.0
