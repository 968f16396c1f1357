"""The multi-GPU host path on CPU: two gloo ranks split one job by the
longest-first greedy partition (rt_shard_assign, the partition every rank of
a sharded batch plan computes), each "traces" its own items with a host
stand-in, and the partial maps and gradient grids are gathered by the sum
over ranks (paper_2606_02413_gb300.shard.gather_sum, the collective the GPU
path uses).  The gathered results must equal one rank doing the whole job,
bit for bit: the stand-ins produce integer values, so only a wrong
partition (an item traced twice or never) or a wrong reduction can differ.
The bench's max-time / summed-work reduction is checked too."""
import os
import socket

import numpy as np
import pytest

NF, NY, NX, CHUNK = 3, 17, 23, 64
GRID = (5, 6, 7)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _items():
    """(frequency, first pixel, count) chunks of one job and their costs."""
    npix = NX * NY
    items = [(f, p0, min(CHUNK, npix - p0)) for f in range(NF) for p0 in range(0, npix, CHUNK)]
    cost = np.random.default_rng(7).uniform(1.0, 50.0, size=len(items))
    return items, cost


def _stand_in(items, owner, rank):
    """Host stand-in for tracing: integer-valued T_b per ray, and each ray's
    integer-valued gradient contribution scattered to a node grid."""
    tb = np.zeros((NF, NY * NX), np.float32)
    grad = np.zeros(int(np.prod(GRID)), np.float32)
    for (f, p0, n), o in zip(items, owner):
        if rank is not None and o != rank:
            continue
        pix = np.arange(p0, p0 + n)
        tb[f, pix] = (f * 7919 + pix * 13) % 65536
        np.add.at(grad, (pix * 31 + f * 5) % grad.size, 1.0 + (pix % 3))
    return tb, grad


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    from paper_2606_02413_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items, cost = _items()
        owner = shard.assign(cost, world)
        all_owners = [torch.zeros(len(items), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(all_owners, torch.from_numpy(owner))
        same = all(torch.equal(a, all_owners[0]) for a in all_owners)
        tb, grad = _stand_in(items, owner, rank)
        tb_t, grad_t = torch.from_numpy(tb), torch.from_numpy(grad)
        shard.gather_sum(tb_t)
        shard.gather_sum(grad_t)
        loads = [float(cost[owner == r].sum()) for r in range(world)]
        ms, steps = bench.reduce_over_ranks(100.0 + 10.0 * rank, 1000.0 * (rank + 1), world)
        out.put((rank, same, owner.tolist(), tb_t.numpy().tobytes(), grad_t.numpy().tobytes(), loads, ms, steps))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_gather_and_reduce():
    import torch.multiprocessing as mp

    from paper_2606_02413_gb300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    items, cost = _items()
    owner = np.array(res[0][2])
    assert res[0][1] and res[1][1] and res[0][2] == res[1][2]   # every rank computed the same partition
    assert set(owner.tolist()) == {0, 1}                          # both ranks have work
    assert np.array_equal(owner, shard.assign(cost, 2))
    # longest-first greedy bound: no rank exceeds the mean load by more than the largest item
    loads = res[0][5]
    assert max(loads) <= sum(loads) / 2 + cost.max()
    tb1, grad1 = _stand_in(items, owner, None)                   # one rank doing the whole job
    for r in res:
        assert r[3] == tb1.tobytes() and r[4] == grad1.tobytes()
        assert r[6] == 110.0 and r[7] == 3000.0                   # slowest rank's time, summed work


def test_shard_assign_edge_cases():
    from paper_2606_02413_gb300 import _abi, shard
    assert shard.assign(np.zeros(0), 3).size == 0
    assert shard.assign([4.0, 1.0], 1).tolist() == [0, 0]
    assert sorted(shard.assign([1.0, 1.0, 1.0], 8).tolist()) == [0, 1, 2]  # more ranks than items
    with pytest.raises(_abi.RtError, match="RT_ERR_ARG"):
        shard.assign([1.0, -2.0], 2)
    with pytest.raises(_abi.RtError, match="RT_ERR_ARG"):
        shard.assign([1.0], 0)
