"""The multi-GPU partition on one GPU: the shard plans of every rank of a
world, run one after another (no rank waits on another), must together trace
every ray exactly once with the single-GPU arithmetic (their summed maps
equal rt_trace_image's bit for bit), and the per-rank adjoints (weights
zeroed outside each rank's rays) must sum to the single-GPU gradient."""
import numpy as np
import pytest

import corona_synth as cs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_02413_gb300 import build
    build.build()
    import paper_2606_02413_gb300 as rt
    return rt


@pytest.mark.parametrize("world", [2, 3, 5])
def test_shards_cover_every_ray_once(rt, world):
    import torch
    from paper_2606_02413_gb300 import shard
    ctx = rt.Context(0)
    g, _, _ = cs.tiny_workload()
    grid = ctx.load(g)
    v = cs.View(0.4, 0.1, 41, 37, -2.6, 2.4, -2.5, 2.7)
    f = np.array([55e6, 180e6, 640e6])
    o = rt.options(precision=1)
    ref = ctx.trace_image(grid, v, f, o)
    total = torch.zeros_like(ref)
    owned = torch.zeros(ref.shape, dtype=torch.int32, device=ref.device)
    for r in range(world):
        tb, d = shard.trace_image(ctx, grid, v, f, o, r, world, diag=True)
        total += tb
        owned += (d[..., 6] != 0).to(torch.int32)
    torch.cuda.synchronize()
    assert bool((owned == 1).all())          # every ray traced by exactly one rank
    assert torch.equal(total, ref)           # with the single-GPU arithmetic


def test_sharded_adjoint_sums_to_single_gpu(rt):
    import torch
    from paper_2606_02413_gb300 import shard
    ctx = rt.Context(0)
    g = cs.newkirk_grid(24, 16, 24, 4.0)
    grid = ctx.load(g)
    v = cs.View(0.3, 0.1, 7, 6, -1.8, 1.8, -1.6, 1.6)
    f = [70e6, 240e6]
    o = rt.options(precision=1, dtau=1e-2)
    w = np.random.default_rng(5).normal(size=(len(f), v.ny, v.nx))
    ref_ne, ref_te = ctx.backward(grid, v, f, w, o)
    sum_ne, sum_te = torch.zeros_like(ref_ne), torch.zeros_like(ref_te)
    for r in range(3):
        dne, dte = shard.backward(ctx, grid, v, f, w, o, r, 3)
        sum_ne += dne
        sum_te += dte
    torch.cuda.synchronize()
    for a, b in ((sum_ne, ref_ne), (sum_te, ref_te)):   # equal up to the order of the float atomics
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * b.abs().max().item())
