"""The N > 1 host path of bench.py on CPU: two gloo ranks shard the work by
observer longitude (independent problems) and reduce (max time, summed
work) after the timed region; no collective touches the data path."""
import math
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import corona_synth as cs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.shard_views(cs.View(0.1, 0.2, 8, 6), world, rank)
        # rank r pretends to have taken 100 + 10 r ms for 1000 (r + 1) ray-steps
        ms, steps = bench.reduce_over_ranks(100.0 + 10.0 * rank, 1000.0 * (rank + 1), world)
        out.put((rank, v.lon_rad, v.lat_rad, v.nx, v.ny, ms, steps))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, lon0, lat0, nx0, ny0, ms0, st0), (r1, lon1, lat1, nx1, ny1, ms1, st1) = res
    assert (r0, r1) == (0, 1)
    assert lon0 == pytest.approx(0.1) and lon1 == pytest.approx(0.1 + math.pi)  # distinct problems
    assert (lat0, nx0, ny0) == (lat1, nx1, ny1) == (0.2, 8, 6)                 # same shape per rank
    assert ms0 == ms1 == 110.0                                                  # the slowest rank
    assert st0 == st1 == 3000.0                                                 # the job's work
