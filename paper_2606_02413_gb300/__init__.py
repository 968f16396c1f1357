"""GB300-native refractive radio ray tracing (arXiv 2606.02413 hot path).

Thin Python binding over the C ABI of ``librt.so`` (``include/rt.h``).  The
functions here only marshal arguments: device memory and streams come from
PyTorch, and every step of the ray tracing runs in librt's CUDA kernels.

    ctx = Context(0)
    grid = ctx.load_grid(r, theta, phi, ne, te)          # host numpy or CUDA tensors
    tb = ctx.trace_image(grid, view, freqs, options(...))  # torch [nf, ny, nx] on the GPU
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import (RT_MAG_OFF, RT_MIXED, RT_PLAIN_F32, RT_STEPWISE, RT_TUBE, RAY_STATUS, RtError,
                   check, lib)

__all__ = ["Context", "Grid", "BatchPlan", "Tape", "RayTraceFn", "options", "view", "RtError", "RT_STEPWISE", "RT_TUBE", "RT_MAG_OFF",
           "RT_PLAIN_F32", "RT_MIXED", "RAY_STATUS", "diag_to_numpy"]


def options(**kw) -> _abi.Options:
    """rt_options with the library defaults, overridden by keyword."""
    o = _abi.Options()
    lib().rt_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"rt_options has no field {k}")
        setattr(o, k, v)
    return o


def view(v) -> _abi.View:
    """rt_view from any object with lon_rad, lat_rad, nx, ny, x0, x1, y0, y1."""
    if isinstance(v, _abi.View):
        return v
    return _abi.View(float(v.lon_rad), float(v.lat_rad), int(v.nx), int(v.ny), float(v.x0), float(v.x1),
                     float(v.y0), float(v.y1))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Grid:
    """A library-owned device copy of a coronal grid (rt_grid)."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, shape):
        self.ctx = ctx
        self.handle = handle
        self.shape = shape

    def free(self):
        if self.handle and self.ctx.handle:
            check(lib().rt_free_grid(self.ctx.handle, self.handle), "rt_free_grid")
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Tape:
    """An adjoint tape (rt_tape): the forward of trace_image_tape with its
    checkpoints, reversed by backward() without tracing the rays again."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, grid: Grid, nf: int, ny: int, nx: int, diag):
        self.ctx = ctx
        self.handle = handle
        self.grid = grid      # the tape refers to the grid: keep it alive
        self.shape = (nf, ny, nx)
        self.diag = diag      # the caller-visible diagnostics the tape keeps

    def backward(self, dL_dTb, stream=None):
        """rt_backward_tape: (dL/dn_e, dL/dT_e) of sum(dL_dTb * T_b), float32
        CUDA tensors shaped like the grid."""
        import torch
        dev = torch.device("cuda", self.ctx.device)
        g = torch.as_tensor(dL_dTb, dtype=torch.float32, device=dev).contiguous()
        assert g.numel() == self.shape[0] * self.shape[1] * self.shape[2]
        dne = torch.empty(self.grid.shape, dtype=torch.float32, device=dev)
        dte = torch.empty(self.grid.shape, dtype=torch.float32, device=dev)
        check(lib().rt_backward_tape(self.handle, C.c_void_p(g.data_ptr()), C.c_void_p(dne.data_ptr()),
                                     C.c_void_p(dte.data_ptr()), _stream_ptr(stream)), "rt_backward_tape")
        return dne, dte

    def info(self, stream=None):
        """(pool slots taken, pool capacity); taken > capacity: it overflowed."""
        used, cap = C.c_ulonglong(0), C.c_ulonglong(0)
        check(lib().rt_tape_info(self.handle, _stream_ptr(stream), C.byref(used), C.byref(cap)), "rt_tape_info")
        return int(used.value), int(cap.value)

    def free(self):
        if self.handle:
            check(lib().rt_tape_free(self.handle), "rt_tape_free")
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class ImageRequest:
    """One image request of a batch: a view and its frequencies [Hz]."""

    def __init__(self, view, freqs_hz):
        self.view = view
        self.freqs_hz = freqs_hz


class BatchPlan:
    """rt_batch_plan: one graph-captured persistent launch over many requests.
    ``outputs`` holds each request's T_b tensor [nf, ny, nx] (and diag).
    shard=(rank, world_size): the plan of one rank of a multi-GPU partition
    (rt_batch_plan_create_shard); its outputs start at zero and hold only
    that rank's rays."""

    def __init__(self, ctx: "Context", grid: Grid, requests, opts=None, diag=False, shard=None):
        import torch
        self.ctx = ctx
        self._keep = []
        n = len(requests)
        arr = (_abi.Request * n)()
        self.outputs = []
        dev = torch.device("cuda", ctx.device)
        for i, req in enumerate(requests):
            v = view(req.view)
            f = np.ascontiguousarray(np.atleast_1d(req.freqs_hz), dtype=np.float64)
            alloc = torch.zeros if shard is not None else torch.empty
            tb = alloc((len(f), v.ny, v.nx), dtype=torch.float32, device=dev)
            d = alloc((len(f), v.ny, v.nx, 7), dtype=torch.int32, device=dev) if diag else None
            self._keep += [v, f]
            arr[i] = _abi.Request(C.pointer(v), f.ctypes.data_as(C.POINTER(C.c_double)), len(f), tb.data_ptr(),
                                  d.data_ptr() if d is not None else None)
            self.outputs.append((tb, d) if diag else tb)
        self._arr = arr
        o = opts if opts is not None else options()
        h = C.c_void_p()
        if shard is None:
            check(lib().rt_batch_plan_create(ctx.handle, grid.handle, arr, n, C.byref(o), C.byref(h)),
                  "rt_batch_plan_create")
        else:
            check(lib().rt_batch_plan_create_shard(ctx.handle, grid.handle, arr, n, C.byref(o), int(shard[0]),
                                                   int(shard[1]), C.byref(h)), "rt_batch_plan_create_shard")
        self.handle = h

    def launch(self, stream=None):
        check(lib().rt_batch_plan_launch(self.handle, _stream_ptr(stream)), "rt_batch_plan_launch")

    def stats(self, stream=None):
        s = _abi.Stats()
        check(lib().rt_batch_plan_stats(self.handle, _stream_ptr(stream), C.byref(s)), "rt_batch_plan_stats")
        return {"ray_steps": int(s.ray_steps), "rays": int(s.rays)}

    def destroy(self):
        if self.handle:
            lib().rt_batch_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Context:
    """An rt_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        torch.cuda.init()
        self.device = device
        h = C.c_void_p()
        check(lib().rt_create(C.byref(h), device), "rt_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().rt_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- grids
    def load_grid(self, r, theta, phi, ne, te, stream=None) -> Grid:
        """rt_load_grid.  ne, te: [n_r, n_theta, n_phi] float32/float64, as
        host numpy arrays or CUDA torch tensors (copied; caller keeps them)."""
        import torch
        r = np.ascontiguousarray(r, dtype=np.float64)
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        if isinstance(ne, torch.Tensor):
            assert ne.is_cuda and te.is_cuda and ne.dtype == te.dtype
            ne, te = ne.contiguous(), te.contiguous()
            dtype = _abi.RT_F64 if ne.dtype == torch.float64 else _abi.RT_F32
            pne, pte, on_dev = ne.data_ptr(), te.data_ptr(), 1
            shape = tuple(ne.shape)
        else:
            dt = np.float64 if np.asarray(ne).dtype == np.float64 else np.float32
            ne = np.ascontiguousarray(ne, dtype=dt)
            te = np.ascontiguousarray(te, dtype=dt)
            dtype = _abi.RT_F64 if dt == np.float64 else _abi.RT_F32
            pne, pte, on_dev = ne.ctypes.data, te.ctypes.data, 0
            shape = ne.shape
        desc = _abi.GridDesc(len(r), len(theta), len(phi), r.ctypes.data, theta.ctypes.data, phi.ctypes.data,
                             dtype, on_dev)
        h = C.c_void_p()
        check(lib().rt_load_grid(self.handle, C.byref(desc), C.c_void_p(pne), C.c_void_p(pte),
                                 _stream_ptr(stream), C.byref(h)), "rt_load_grid")
        return Grid(self, h, shape)

    def load(self, g, stream=None) -> Grid:
        """rt_load_grid from a corona_synth.Grid-like object."""
        return self.load_grid(g.r, g.theta, g.phi, g.ne, g.te, stream)

    # ----------------------------------------------------------- tracing
    def trace_image(self, grid: Grid, v, freqs, opts=None, out=None, diag=False, stream=None):
        """rt_trace_image.  Returns T_b [nf, ny, nx] float32 on the GPU (and,
        with diag=True, an int32 [nf, ny, nx, 7] tensor holding rt_ray_diag)."""
        import torch
        vs = view(v)
        f = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
        nf = len(f)
        dev = torch.device("cuda", self.device)
        if out is None:
            out = torch.empty((nf, vs.ny, vs.nx), dtype=torch.float32, device=dev)
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == nf * vs.ny * vs.nx
        d = torch.empty((nf, vs.ny, vs.nx, 7), dtype=torch.int32, device=dev) if diag else None
        o = opts if opts is not None else options()
        check(lib().rt_trace_image(self.handle, grid.handle, C.byref(vs),
                                   f.ctypes.data_as(C.POINTER(C.c_double)), nf, C.byref(o),
                                   C.c_void_p(out.data_ptr()), C.c_void_p(d.data_ptr() if d is not None else 0),
                                   _stream_ptr(stream)), "rt_trace_image")
        return (out, d) if diag else out

    def trace_image_tape(self, grid: Grid, v, freqs, opts=None, pool_bytes=0, stream=None):
        """rt_trace_image_tape: T_b [nf, ny, nx] (as trace_image), the
        diagnostics [nf, ny, nx, 7] and a Tape whose backward() gives the
        gradients without tracing again.  pool_bytes = 0: sized from an
        estimate of the path lengths."""
        import torch
        vs = view(v)
        f = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
        nf = len(f)
        dev = torch.device("cuda", self.device)
        out = torch.empty((nf, vs.ny, vs.nx), dtype=torch.float32, device=dev)
        d = torch.empty((nf, vs.ny, vs.nx, 7), dtype=torch.int32, device=dev)
        o = opts if opts is not None else options()
        h = C.c_void_p()
        check(lib().rt_trace_image_tape(self.handle, grid.handle, C.byref(vs),
                                        f.ctypes.data_as(C.POINTER(C.c_double)), nf, C.byref(o),
                                        C.c_size_t(int(pool_bytes)), C.c_void_p(out.data_ptr()),
                                        C.c_void_p(d.data_ptr()), C.byref(h), _stream_ptr(stream)),
              "rt_trace_image_tape")
        return out, d, Tape(self, h, grid, nf, vs.ny, vs.nx, d)

    def batch_plan(self, grid: Grid, requests, opts=None, diag=False) -> BatchPlan:
        """rt_batch_plan_create over requests (objects with .view and .freqs_hz)."""
        return BatchPlan(self, grid, requests, opts, diag)

    def backward(self, grid: Grid, v, freqs, dL_dTb, opts=None, want_tb=False, fwd_diag=None, stream=None):
        """rt_backward: gradients of sum(dL_dTb * T_b) w.r.t. the grid node
        values.  Returns (dL/dn_e, dL/dT_e) as float32 CUDA tensors shaped like
        the grid (and the forward T_b with want_tb=True).  fwd_diag: the diag
        tensor of trace_image(..., diag=True) for the same inputs, which spares
        the call its step-counting forward pass."""
        import torch
        vs = view(v)
        f = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
        dev = torch.device("cuda", self.device)
        g = torch.as_tensor(dL_dTb, dtype=torch.float32, device=dev).contiguous()
        assert g.numel() == len(f) * vs.ny * vs.nx
        dne = torch.empty(grid.shape, dtype=torch.float32, device=dev)
        dte = torch.empty(grid.shape, dtype=torch.float32, device=dev)
        tb = torch.empty((len(f), vs.ny, vs.nx), dtype=torch.float32, device=dev) if want_tb else None
        o = opts if opts is not None else options()
        if fwd_diag is not None:
            assert fwd_diag.is_cuda and fwd_diag.is_contiguous() and fwd_diag.numel() * 4 == 28 * g.numel()
        check(lib().rt_backward(self.handle, grid.handle, C.byref(vs), f.ctypes.data_as(C.POINTER(C.c_double)),
                                len(f), C.byref(o), C.c_void_p(g.data_ptr()), C.c_void_p(dne.data_ptr()),
                                C.c_void_p(dte.data_ptr()), C.c_void_p(tb.data_ptr() if tb is not None else 0),
                                C.c_void_p(fwd_diag.data_ptr() if fwd_diag is not None else 0),
                                _stream_ptr(stream)), "rt_backward")
        return (dne, dte, tb) if want_tb else (dne, dte)

    def disk_mean_tb(self, v, tb, radius=0.5, stream=None):
        """rt_disk_mean_tb: the mean T_b within `radius` R_sun of disk centre of
        each map in tb (a [nf, ny, nx] float32 CUDA tensor traced with view v).
        Returns a float64 CUDA tensor [nf]."""
        import torch
        vs = view(v)
        assert tb.is_cuda and tb.dtype == torch.float32 and tb.is_contiguous()
        nf = tb.numel() // (vs.nx * vs.ny)
        assert nf * vs.nx * vs.ny == tb.numel()
        out = torch.empty(nf, dtype=torch.float64, device=tb.device)
        check(lib().rt_disk_mean_tb(C.byref(vs), C.c_void_p(tb.data_ptr()), nf, float(radius),
                                    C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "rt_disk_mean_tb")
        return out

    def trace_paths(self, grid: Grid, v, freq_hz, pixels, opts=None, cap=100000, stream=None):
        """rt_trace_paths: the node-by-node paths of the rays of `pixels` (flat
        indices of view v) at one frequency.  Returns a list of dicts of numpy
        arrays (r [m, 3], ln_s, dlns_ds, tau, ne, te) and the rays' T_b and
        diagnostics."""
        import torch
        vs = view(v)
        pix = np.ascontiguousarray(np.atleast_1d(pixels), dtype=np.int32)
        n = len(pix)
        dev = torch.device("cuda", self.device)
        nodes = torch.empty((n, cap, 8), dtype=torch.float32, device=dev)
        counts = torch.empty(n, dtype=torch.int32, device=dev)
        tb = torch.empty(n, dtype=torch.float32, device=dev)
        d = torch.empty((n, 7), dtype=torch.int32, device=dev)
        o = opts if opts is not None else options()
        check(lib().rt_trace_paths(self.handle, grid.handle, C.byref(vs), float(freq_hz),
                                   pix.ctypes.data_as(C.POINTER(C.c_int)), n, C.byref(o), int(cap),
                                   C.c_void_p(nodes.data_ptr()), C.c_void_p(counts.data_ptr()),
                                   C.c_void_p(tb.data_ptr()), C.c_void_p(d.data_ptr()), _stream_ptr(stream)),
              "rt_trace_paths")
        torch.cuda.synchronize(dev)
        nd, cn = nodes.cpu().numpy(), counts.cpu().numpy()
        paths = []
        for i in range(n):
            m = min(int(cn[i]), cap)
            a = nd[i, :m]
            paths.append({"r": a[:, 0:3].astype(np.float64), "ln_s": a[:, 3].astype(np.float64),
                          "dlns_ds": a[:, 4].astype(np.float64), "tau": a[:, 5].astype(np.float64),
                          "ne": a[:, 6].astype(np.float64), "te": a[:, 7].astype(np.float64),
                          "n_nodes": int(cn[i])})
        return paths, tb, d

    def beam_convolve(self, v, tb, freqs, baseline_m, stream=None):
        """rt_beam_convolve: the maps tb ([nf, ny, nx] float32 CUDA tensor traced
        with view v at freqs) convolved with the Gaussian beam of an
        interferometer of maximum baseline baseline_m metres."""
        import torch
        vs = view(v)
        f = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
        assert tb.is_cuda and tb.dtype == torch.float32 and tb.is_contiguous()
        assert tb.numel() == len(f) * vs.nx * vs.ny
        scratch = torch.empty_like(tb)
        out = torch.empty_like(tb)
        check(lib().rt_beam_convolve(C.byref(vs), C.c_void_p(tb.data_ptr()), f.ctypes.data_as(C.POINTER(C.c_double)),
                                     len(f), float(baseline_m), C.c_void_p(scratch.data_ptr()),
                                     C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "rt_beam_convolve")
        return out

    def probe_field(self, grid: Grid, xyz, stream=None):
        """rt_probe_field: (n_e, T_e, grad n_e) at points xyz [n, 3] -> [n, 5]."""
        import torch
        pts = torch.as_tensor(xyz, dtype=torch.float32).reshape(-1, 3).contiguous().to(f"cuda:{self.device}")
        out = torch.empty((pts.shape[0], 5), dtype=torch.float32, device=pts.device)
        check(lib().rt_probe_field(self.handle, grid.handle, C.c_void_p(pts.data_ptr()), pts.shape[0],
                                   C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "rt_probe_field")
        return out

    def sync(self, stream=None):
        check(lib().rt_sync(self.handle, _stream_ptr(stream)), "rt_sync")

    def stats(self, stream=None):
        s = _abi.Stats()
        check(lib().rt_get_stats(self.handle, _stream_ptr(stream), C.byref(s)), "rt_get_stats")
        return {"ray_steps": int(s.ray_steps), "rays": int(s.rays)}


def diag_to_numpy(d):
    """Split an int32 [..., 7] rt_ray_diag tensor into numpy fields."""
    a = d.cpu().numpy()
    f = a.view(np.float32)
    return {"exit": f[..., 0:3].astype(np.float64), "tau": f[..., 3].astype(np.float64),
            "ln_s": f[..., 4].astype(np.float64), "steps": a[..., 5].astype(np.int64),
            "status": a[..., 6].astype(np.int32)}


class RayTraceFn:
    """torch.autograd.Function: T_b maps from grid tensors, differentiable
    with respect to n_e and T_e: the forward keeps an adjoint tape
    (rt_trace_image_tape), the backward reverses it (rt_backward_tape).

        tb = RayTraceFn.apply(ne, te, ctx, r, theta, phi, view, freqs, opts)

    ne, te: CUDA tensors [n_r, n_theta, n_phi] (float32 or float64)."""

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(fctx, ne, te, ctx, r, theta, phi, v, freqs, opts):
                grid = ctx.load_grid(r, theta, phi, ne.detach(), te.detach())
                o = opts if opts is not None else options()
                differentiable = (not o.straight) and (o.s_mode == RT_MAG_OFF or (o.s_mode == RT_STEPWISE
                                                                                  and o.n_nb == 4))
                if differentiable and any(fctx.needs_input_grad[:2]):
                    tb, _, tape = ctx.trace_image_tape(grid, v, freqs, o)
                else:  # no gradient wanted, or a form the adjoint does not cover
                    tb, tape = ctx.trace_image(grid, v, freqs, o), None
                fctx.state = (grid, tape, ne.dtype, te.dtype)
                return tb

            @staticmethod
            def backward(fctx, grad_tb):
                grid, tape, dne_t, dte_t = fctx.state
                if tape is None:
                    raise RuntimeError("RayTraceFn: the adjoint covers step-wise magnification with 4 "
                                       "neighbours or magnification off, not straight lines or tube mode")
                dne, dte = tape.backward(grad_tb.contiguous())
                tape.free()
                grid.free()
                return dne.to(dne_t), dte.to(dte_t), None, None, None, None, None, None, None

        return _F

    @classmethod
    def apply(cls, *args):
        if not hasattr(cls, "_impl"):
            cls._impl = cls._fn()
        return cls._impl.apply(*args)

