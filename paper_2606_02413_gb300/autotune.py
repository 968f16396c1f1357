"""Autotuner for the ray-tracing launch (step size and launch shape).

For a (grid, view, frequencies) workload it chooses

* the RK4 step: the largest dtau in {1, 2, 4, 8} x 1e-3 R_sun whose T_b maps
  on a 32x32 image of the same field of view stay within `gate` (relative
  to max(T_b, 1e-2 of the map maximum)) of the maps at dtau = 1e-3 R_sun,
  computed by this library.  The step is part of the method's result (the
  step-wise magnification is first order in it), so the gate, not speed,
  decides it;
* the launch shape: the pixel walk (64-pixel chunks longest first, or each
  frequency in tiles of 4, 8, 16) and
  the persistent blocks per SM, timed with CUDA events on a reduced image
  of the workload at the chosen step (results do not depend on them).

Results are cached in a JSON file keyed by the GPU name and a hash of the
workload and the fixed options.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import options as make_options
from . import view as make_view

STEPS = (1e-3, 2e-3, 4e-3, 8e-3)
TILES = (0, 4, 8, 16)


def _key(grid, v, freqs, opts, gate):
    import torch
    vs = make_view(v)
    h = hashlib.sha256()
    h.update(json.dumps([list(grid.shape), [vs.lon_rad, vs.lat_rad, vs.nx, vs.ny, vs.x0, vs.x1, vs.y0, vs.y1],
                         [float(f) for f in np.atleast_1d(freqs)],
                         [opts.s_mode, opts.n_nb, opts.eps_mode, opts.eta, opts.delta, opts.tau_stop,
                          opts.tbc_mode, opts.tbc_K, opts.emission, opts.straight, opts.precision], gate]).encode())
    return f"{torch.cuda.get_device_name()}|{h.hexdigest()[:16]}"


def _rel_err(a, b):
    """Per-pixel |a - b| / max(b, 1e-2 of the map maximum)."""
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    m = b.reshape(b.shape[0], -1).max(axis=1).clip(min=1e-30)
    return np.abs(a - b) / np.maximum(b, 1e-2 * m[:, None, None])


def _time(ctx, grid, v, freqs, opts, reps=2):
    import torch
    ctx.trace_image(grid, v, freqs, opts)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.trace_image(grid, v, freqs, opts)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def step_gate(ctx, grid, v, freqs, opts=None, gate=1e-3, side=32):
    """The step-size part of tune(): the largest step in STEPS whose side^2
    maps of the field of view of v stay within `gate` (every pixel) of the
    maps at the smallest step.  Returns (dtau, {step: worst error},
    {step: 99th-percentile error})."""
    from types import SimpleNamespace
    opts = opts if opts is not None else make_options()
    vs = make_view(v)
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    base = _fields(opts)
    small = SimpleNamespace(lon_rad=vs.lon_rad, lat_rad=vs.lat_rad, nx=side, ny=side, x0=vs.x0, x1=vs.x1,
                            y0=vs.y0, y1=vs.y1)
    ref = ctx.trace_image(grid, small, freqs, make_options(**{**base, "dtau": STEPS[0]}))
    dtau, worst, p99 = STEPS[0], {}, {}
    for h in STEPS:
        tb = ctx.trace_image(grid, small, freqs, make_options(**{**base, "dtau": h}))
        rel = _rel_err(tb, ref)
        worst[f"{h:g}"] = float(rel.max())                    # the gate: every pixel
        p99[f"{h:g}"] = float(np.percentile(rel, 99))         # reported only
        if worst[f"{h:g}"] <= gate:
            dtau = h
    return dtau, worst, p99


def tune(ctx, grid, v, freqs, opts=None, gate=1e-3, cache=None, time_side=128, tune_step=True):
    """Returns (rt_options with dtau, tile and blocks_per_sm set, report)."""
    from types import SimpleNamespace
    opts = opts if opts is not None else make_options()
    key = _key(grid, v, freqs, opts, gate)
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            table = json.load(fh)
        if key in table:
            r = table[key]
            return make_options(**{**_fields(opts), **r["choice"]}), r
    vs = make_view(v)
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    report = {"gate": gate, "steps": {}, "steps_p99": {}, "launch": {}}
    base = _fields(opts)
    # 1) step size on a 32x32 image of the same field of view
    dtau = base["dtau"]
    if tune_step:
        dtau, report["steps"], report["steps_p99"] = step_gate(ctx, grid, v, freqs, opts, gate)
    # 2) launch shape on a reduced image at the chosen step
    red = SimpleNamespace(lon_rad=vs.lon_rad, lat_rad=vs.lat_rad, nx=min(vs.nx, time_side),
                          ny=min(vs.ny, time_side), x0=vs.x0, x1=vs.x1, y0=vs.y0, y1=vs.y1)
    best = None
    for tile in TILES:
        for bps in (0, 6, 4):
            o = make_options(**{**base, "dtau": dtau, "tile": tile, "blocks_per_sm": bps})
            ms = _time(ctx, grid, red, freqs, o)
            report["launch"][f"tile={tile},blocks_per_sm={bps}"] = ms
            if best is None or ms < best[0]:
                best = (ms, tile, bps)
    choice = {"dtau": dtau, "tile": best[1], "blocks_per_sm": best[2]}
    report["choice"] = choice
    if cache:
        table = {}
        if os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        table[key] = report
        tmp = cache + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1)
        os.replace(tmp, cache)
    return make_options(**{**base, **choice}), report


def _fields(o):
    return {name: getattr(o, name) for name, _ in o._fields_}
