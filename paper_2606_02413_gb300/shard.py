"""Multi-GPU partition of one tracing job: one process per GPU.

Every (pixel, frequency) ray is independent (Sec. 3.2), so one job splits
into the (request, frequency, 64-pixel chunk) items of the batch plan.  Every
rank computes the same longest-first greedy partition of those items
(``rt_shard_assign`` over the plan's path-length estimates), traces only its
own with a replicated grid, and the maps are gathered by a sum over ranks
(each pixel is written by exactly one rank, the others hold zero, so the sum
is exact).  The adjoint splits the same way: each rank zeroes the weights
dL/dT_b of the rays it does not own (rt_backward then skips them in every
pass) and the two gradient grids are summed over the ranks, the method's one
exchange step.

Collectives go through ``torch.distributed`` (NCCL between GPUs, gloo on CPU
for the host-side tests); nothing here computes any of the method.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi


def assign(costs, world_size: int) -> np.ndarray:
    """rt_shard_assign on the host: the owning rank of every item."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    out = np.zeros(c.size, dtype=np.int32)
    _abi.check(_abi.lib().rt_shard_assign(c.ctypes.data_as(C.POINTER(C.c_double)), c.size, int(world_size),
                                          out.ctypes.data_as(C.POINTER(C.c_int))), "rt_shard_assign")
    return out


def gather_sum(t, group=None):
    """Gather rank-disjoint partial results (zeros where another rank owns
    the entry) into the full result on every rank: an all-reduce sum."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def trace_image(ctx, grid, v, freqs, opts, rank: int, world_size: int, group=None, diag=False):
    """This rank's share of rt_trace_image over (v, freqs), gathered: every
    rank returns the full [nf, ny, nx] maps (and, with diag=True, this
    rank's own diagnostics, zero for the rays of other ranks).  Per-ray
    arithmetic is that of the single-GPU trace."""
    p = plan(ctx, grid, v, freqs, opts, rank, world_size, diag=diag)
    p.launch()
    out = p.outputs[0]
    p.destroy()
    tb, d = out if diag else (out, None)
    gather_sum(tb, group)
    return (tb, d) if diag else tb


def plan(ctx, grid, v, freqs, opts, rank: int, world_size: int, diag=False):
    """The batch plan of this rank's share of one image request, with
    zero-initialised outputs."""
    from . import BatchPlan, ImageRequest
    return BatchPlan(ctx, grid, [ImageRequest(v, np.atleast_1d(freqs))], opts, diag=diag, shard=(rank, world_size))


def backward(ctx, grid, v, freqs, dL_dTb, opts, rank: int, world_size: int, group=None):
    """Sharded rt_backward: this rank traces its share (to learn which rays
    it owns and their step counts), runs the adjoint on those rays only, and
    the gradients are summed over the ranks.  Returns (dL/dn_e, dL/dT_e) on
    every rank."""
    import torch
    p = plan(ctx, grid, v, freqs, opts, rank, world_size, diag=True)
    p.launch()
    _, d = p.outputs[0]
    mine = d[..., 6] != 0                     # status: nonzero exactly on this rank's rays
    w = torch.as_tensor(dL_dTb, dtype=torch.float32, device=d.device).reshape(mine.shape)
    w = torch.where(mine, w, torch.zeros_like(w)).contiguous()
    dne, dte = ctx.backward(grid, v, freqs, w, opts, fwd_diag=d)
    p.destroy()
    gather_sum(dne, group)
    gather_sum(dte, group)
    return dne, dte
