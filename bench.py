"""Benchmark: ray-steps/s and maps/s of the GB300 ray tracer.

Workload (N = 1): the 256(r, 1-30 R_sun stretched) x 180(theta) x 360(phi)
MAS-like synthetic corona, a 512x512 image over +-3 R_sun at 16 frequencies
log-spaced 40-800 MHz, one ray bundle (central ray + 4 step-wise neighbours)
per pixel and frequency, RK4 step 2e-3 R_sun, free-free transfer with the
magnification term, compensated (mixed) form.  One step = one rt_trace_image
call over the whole workload (16 maps, 4.19 M ray bundles).

With N > 1 ranks (torchrun) the ranks split the one job (strong scaling): each
traces its share of the (frequency, 64-pixel chunk) items of the longest-first
greedy partition (rt_batch_plan_create_shard) and the maps are gathered by an
all-reduce sum (NCCL); `value` is the job's ray-steps over the slowest rank's
time, the gather included.

--impl reference runs the FP64 CPU oracle (the only reference arm this
method has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray-steps/s & maps/s (512^2 x 16 freq, 1 GB300); adjoint/forward time ratio"
R_SUN_UNITS = "R_sun"

# Algorithmic FP32 operations (FMA = 2) of the kernel's operation list:
# one field evaluation (radius and cell lookup, two arctangents, trilinear
# value and three partials, Cartesian chain rule) = 111; the central ray's RK4
# step = 4 evaluations + 60 (stage points, force scaling, G and A sums); a
# step-wise neighbour = its seed and RK4 stages 1-3 (its end position needs
# no fourth stage) = 3 evaluations + 36; per central step the bookkeeping
# (tube area, basis, transfer, termination) = 120, the stage-1 T_e
# interpolation = 15, and the neighbour-pair differences 3 per pair.
FLOP_EVAL = 111
FLOP_CENTRAL_RK4 = 60
FLOP_NEIGHBOUR_RK4 = 36
FLOP_STEP_BOOK = 135


def flops_per_ray_step(n_nb: int) -> int:
    return (4 * FLOP_EVAL + FLOP_CENTRAL_RK4 + n_nb * (3 * FLOP_EVAL + FLOP_NEIGHBOUR_RK4) + FLOP_STEP_BOOK
            + 3 * (n_nb // 2))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


FORWARD_SOURCES = ("csrc/rt_device.cuh", "csrc/rt_bundle.cuh", "csrc/rt_rays.cuh", "build.py")


def kernel_source_hash() -> str:
    """Hash of what the headline kernel (trace_rays) is compiled from: its
    device sources and the build script with its compiler flags (file names
    and contents).  A committed counter capture is valid only for this hash."""
    import hashlib
    h = hashlib.sha256()
    for name in FORWARD_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2606_02413_gb300", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "trace_rays_global_512x512x16_launches.md")


def committed_traffic():
    """DRAM bytes per launch of the headline kernel from the committed ncu
    launch list (line 'traffic: source=<hash> bytes_per_launch=<n>'), or
    None when the kernel sources changed since that capture."""
    try:
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                if line.startswith("traffic:"):
                    kv = dict(item.split("=", 1) for item in line.split()[1:])
                    if kv.get("source") == kernel_source_hash():
                        return float(kv["bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def reduce_over_ranks(total_ms: float, ray_steps: float, world_size: int, device="cpu"):
    """The job's time is the slowest rank's, its work the sum over ranks
    (a reduction of two numbers after the timed region)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(ray_steps)], dtype=torch.float64, device=device)
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def cpu_baseline(g, v, f, target_s=12.0, max_pixels=4096, threads=None):
    """The FP64 oracle (as it stands) on a bounded pixel sample of the same
    workload, on this host's cores (all of them, or `threads`); ray-steps/s
    and the sample description."""
    import oracle
    F = oracle.grid_field(g)
    opts = oracle.default_options(tau_stop=30.0)
    rng = np.random.default_rng(12345)
    cores = threads or os.cpu_count() or 1
    n = 16
    total_steps, elapsed, used = 0, 0.0, 0
    while elapsed < target_s and used < max_pixels:
        pix = rng.choice(v.nx * v.ny, size=n, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        r = oracle.trace(F, v, f, opts, pixels=pix, nthreads=cores)
        dt = time.perf_counter() - t0
        total_steps += int(r["steps"].sum())
        elapsed += dt
        used += n
        n = min(max(int(n * max(target_s - elapsed, 0.5) / max(dt, 1e-3) / 2), 16), max_pixels - used)
        if n <= 0:
            break
    return {"value": total_steps / elapsed, "unit": "ray-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{used} random pixels x {len(f)} frequencies of the 512^2 workload "
                      f"({total_steps} ray-steps in {elapsed:.1f} s, FP64, OpenMP over rays)"}


def run_reference(args):
    import corona_synth as cs
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    g, v, f = cs.global_workload(device="cpu")
    # each step: a bounded sample of the workload through the oracle
    times, steps = [], []
    for i in range(args.warmup + args.steps):
        res = cpu_baseline(g, v, f, target_s=max(4.0, 40.0 / max(args.steps, 1)), max_pixels=64)
        if i >= args.warmup:
            times.append(res)
    val = float(np.mean([t["value"] for t in times]))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "ray-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "MAS-like 256x180x360 corona, 512x512 x 16 freq 40-800 MHz, 4 neighbours"},
            "cpu_baseline": {"value": val, "unit": "ray-steps/s", "cores": times[0]["cores"], "kind": "oracle",
                             "sample": times[0]["sample"]},
            "e2e": {"value": val, "unit": "ray-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(name):
    """One launch of a named case, small enough for an ncu capture.
    fwd-WxHxF: the headline corona, a WxH view over +-3 R_sun at 60 and 300
    MHz (F <= 2) or F frequencies log-spaced over 40-800 MHz, compensated
    form.  adj-WxHxF: rt_backward on the 128x90x180
    differentiation corona, a WxH view over +-2.5 R_sun at F of its 8
    frequencies (40-400 MHz, evenly picked; adj-256x256x8 is the full
    differentiation workload), dL/dT_b = 1."""
    import torch

    import corona_synth as cs
    from paper_2606_02413_gb300 import build as rt_build
    rt_build.build()
    import paper_2606_02413_gb300 as rt
    ctx = rt.Context(0)
    kind, dims = name.split("-")
    nx, ny, nf = (int(x) for x in dims.split("x"))
    if kind == "fwd":
        g, _, _ = cs.global_workload()
        grid = ctx.load(g)
        v = cs.View(0.0, 0.0, nx, ny, -3.0, 3.0, -3.0, 3.0)
        fr = [60e6, 300e6][:nf] if nf <= 2 else list(cs.log_freqs(nf, 40e6, 800e6))
        ctx.trace_image(grid, v, fr, rt.options(precision=rt.RT_MIXED))
    else:
        g, v, f = cs.adjoint_workload()
        grid = ctx.load(g)
        v = cs.View(v.lon_rad, v.lat_rad, nx, ny, v.x0, v.x1, v.y0, v.y1)
        f = [float(f[i]) for i in np.linspace(0, len(f) - 1, min(nf, len(f))).round().astype(int)]
        ctx.backward(grid, v, f, torch.ones((len(f), v.ny, v.nx), device="cuda"), rt.options(precision=rt.RT_MIXED))
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "stats": ctx.stats()}))


def run_autotune():
    """The autotuner on the headline workload (compensated form, 4
    step-wise neighbours): step-size gate against the dtau = 1e-3 maps on a
    32x32 image, launch shape timed on 128x128 x 16 maps."""
    import torch

    import corona_synth as cs
    from paper_2606_02413_gb300 import build as rt_build
    rt_build.build()
    import paper_2606_02413_gb300 as rt
    from paper_2606_02413_gb300 import autotune
    ctx = rt.Context(0)
    g, v, f = cs.global_workload()
    grid = ctx.load(g)
    t0 = time.perf_counter()
    opts, report = autotune.tune(ctx, grid, v, f, rt.options(precision=rt.RT_MIXED), gate=1e-3)
    torch.cuda.synchronize()
    report["tuning_s"] = time.perf_counter() - t0
    report["workload"] = "MAS-like 256x180x360, 512x512 x 16 freq 40-800 MHz, 4 step-wise neighbours, compensated"
    print(json.dumps({"autotune": report}))


def run_batch_workload():
    """The batching workload: 64 independent requests on the symmetric
    64x32x64 corona (image side in {128, 256, 512, 1024}, 1-8 frequencies in
    40-800 MHz, random longitude; ~1e8 rays of very uneven length), plain
    FP32 stepping, 4 step-wise neighbours; and, for contrast, 512 small
    requests (sides 16-64) that one launch each would leave the GPU mostly
    idle for.  Times one graph-captured persistent launch over each batch
    against one rt_trace_image per request on the same stream, and checks
    that the two give the same maps."""
    import torch

    import corona_synth as cs
    from paper_2606_02413_gb300 import build as rt_build
    rt_build.build()
    import paper_2606_02413_gb300 as rt
    ctx = rt.Context(0)
    g, _, _ = cs.tiny_workload()
    grid = ctx.load(g)
    opts = rt.options(precision=rt.RT_PLAIN_F32)
    stream = torch.cuda.current_stream()
    # warm both paths on a small batch (kernel load, graph machinery)
    small = cs.batch_requests(4, sides=(32,))
    wp = ctx.batch_plan(grid, small, opts)
    wp.launch()
    for r in small:
        ctx.trace_image(grid, r.view, r.freqs_hz, opts)
    torch.cuda.synchronize()
    wp.destroy()

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def measure(reqs, label):
        n_maps = sum(len(r.freqs_hz) for r in reqs)
        n_rays = sum(len(r.freqs_hz) * r.view.nx * r.view.ny for r in reqs)
        plan = ctx.batch_plan(grid, reqs, opts)
        ms_b = timed(plan.launch)
        steps = plan.stats()["ray_steps"]
        outs = [torch.empty((len(r.freqs_hz), r.view.ny, r.view.nx), dtype=torch.float32, device="cuda")
                for r in reqs]

        def sequential():
            for r, o in zip(reqs, outs):
                ctx.trace_image(grid, r.view, r.freqs_hz, opts, out=o)
        ms_s = timed(sequential)
        same = all(torch.equal(x, y) for x, y in zip(plan.outputs, outs))
        plan.destroy()
        return {"requests": len(reqs), "what": label, "maps": n_maps, "rays": n_rays, "ray_steps": steps,
                "batched_ms": ms_b, "batched_maps_per_s": n_maps / (ms_b / 1e3),
                "batched_ray_steps_per_s": steps / (ms_b / 1e3),
                "per_request_ms": ms_s, "per_request_maps_per_s": n_maps / (ms_s / 1e3),
                "per_request_ray_steps_per_s": steps / (ms_s / 1e3),  # the same rays, ray for ray
                "speedup": ms_s / ms_b, "identical_maps": bool(same)}

    out = {"form": "plain FP32, 4 step-wise neighbours, h = 2e-3 R_sun, 64x32x64 corona",
           "batch_64": measure(cs.batch_requests(64), "sides 128-1024, 1-8 frequencies"),
           "batch_512_small": measure(cs.batch_requests(512, sides=(16, 32, 64)), "sides 16-64, 1-8 frequencies")}
    print(json.dumps({"batch_workload": out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    choices=["fwd-128x128x2", "fwd-256x256x2", "fwd-256x256x8", "fwd-256x256x16", "fwd-512x512x2",
                             "adj-64x64x2",
                             "adj-128x128x8", "adj-256x256x8"],
                    help="run one launch of a small named case (for ncu captures) and exit")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--batch-workload", action="store_true",
                    help="time the 64-request batching workload batched and per request, print and exit")
    ap.add_argument("--autotune", action="store_true",
                    help="run the autotuner on the headline workload, print its report and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.autotune:
        run_autotune()
        return
    if args.batch_workload:
        run_batch_workload()
        return

    import torch
    import torch.distributed as dist

    import corona_synth as cs
    from paper_2606_02413_gb300 import build as rt_build
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    rt_build.build()
    import paper_2606_02413_gb300 as rt

    g, v, f = cs.global_workload()
    ctx = rt.Context(local)
    grid = ctx.load(g)
    prec = rt.RT_MIXED if args.precision == "mixed" else rt.RT_PLAIN_F32
    opts = rt.options(precision=prec)
    stream = torch.cuda.current_stream()
    dev = f"cuda:{local}"

    # one step = the whole job: 16 maps of 512^2 rays.  With N > 1 ranks the
    # job is split (rt_batch_plan_create_shard: longest-first greedy partition
    # of its (frequency, 64-pixel chunk) items) and the maps are gathered by a
    # sum over the ranks (each pixel is written by one rank).
    if ws > 1:
        from paper_2606_02413_gb300 import shard
        plan = shard.plan(ctx, grid, v, f, opts, rank, ws)
        part = plan.outputs[0]
        out = torch.empty_like(part)

        def trace():
            plan.launch(stream)

        def gather():
            out.copy_(part)
            shard.gather_sum(out)

        def steps_of_last():
            return plan.stats()
    else:
        out = torch.empty((len(f), v.ny, v.nx), dtype=torch.float32, device=dev)

        def trace():
            ctx.trace_image(grid, v, f, opts, out=out)

        def gather():
            pass

        def steps_of_last():
            return ctx.stats()

    for _ in range(args.warmup):
        trace()
        gather()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for e0, e1, e2 in ev:
        e0.record(stream)
        trace()
        e1.record(stream)
        gather()
        e2.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    stats = steps_of_last()  # counters of the last timed step (every step traces the same rays)
    ray_steps = stats["ray_steps"] * args.steps
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [e0.elapsed_time(e1) for e0, e1, _ in ev]
    gather_ms = [e1.elapsed_time(e2) for _, e1, e2 in ev]
    rays_rank = stats["rays"]
    total_ms, all_steps = reduce_over_ranks(total_ms, ray_steps, ws, device=dev)
    _, all_rays = reduce_over_ranks(0.0, rays_rank, ws, device=dev)
    value = all_steps / (total_ms / 1e3)
    maps_per_s = len(f) * args.steps / (total_ms / 1e3)

    # end to end through the public API: pinned host grid -> rt_load_grid ->
    # trace (this rank's share) -> gather -> T_b maps back to pinned host memory
    e2e = None
    if not args.no_e2e:
        ne_h = torch.from_numpy(g.ne).pin_memory()
        te_h = torch.from_numpy(g.te).pin_memory()
        tb_h = torch.empty(out.shape, dtype=torch.float32).pin_memory()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr = ctx.load_grid(g.r, g.theta, g.phi, ne_h.numpy(), te_h.numpy())
        if ws > 1:
            tb_full = shard.trace_image(ctx, gr, v, f, opts, rank, ws)
        else:
            tb_full = ctx.trace_image(gr, v, f, opts, out=out)
        tb_h.copy_(tb_full, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        gr.free()
        dt, _ = reduce_over_ranks(dt * 1e3, 0.0, ws, device=dev)
        dt /= 1e3
        e2e = {"value": all_steps / args.steps / dt, "unit": "ray-steps/s",
               "h2d_bytes_per_step": int(ne_h.numel() * 4 + te_h.numel() * 4) * ws,
               "d2h_bytes_per_step": int(tb_h.numel() * 4) * ws, "seconds_per_step": dt}

    forms = {"mixed" if prec == rt.RT_MIXED else "plain": {
        "ms": total_ms / args.steps, "ray_steps_per_s": value, "maps_per_s": maps_per_s}}
    adjoint = None
    next1 = None
    if ws == 1 and not args.no_forms:
        forms.update(run_forms(ctx, grid, v, f, prec, stream))
    if ws == 1 and not args.no_adjoint:
        adjoint = run_adjoint(ctx)
    step_gate = None
    if ws == 1 and not args.no_forms:
        next1 = run_next1(ctx, grid, f)
        from paper_2606_02413_gb300 import autotune
        h_gate, worst, p99 = autotune.step_gate(ctx, grid, v, f, opts, gate=1e-3)
        step_gate = {"configured_dtau": float(opts.dtau), "autotuner_dtau_at_gate_1e-3": h_gate,
                     "worst_pixel_error_vs_dtau_1e-3": worst, "p99_error_vs_dtau_1e-3": p99,
                     "note": "the bench runs the workload's configured step; the autotuner's every-pixel gate "
                             "picks the step shown"}

    peaks, peak_src = load_peaks()
    clk = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = 2.0 * 128 * n_sm * clk * 1e6 / 1e12  # TFLOP/s: 128 FP32 lanes x FMA per SM per clock
    flop_step = flops_per_ray_step(4)
    kmean = float(np.mean(kern_ms))
    achieved = flop_step * stats["ray_steps"] / (kmean / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": committed_traffic(),
            "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                              + os.path.relpath(TRAFFIC_FILE, ROOT) + " (null if the kernel changed)",
            "peak_source": f"FP32 FMA: 128 lanes x {n_sm} SMs x 2 x {clk:.0f} MHz median SM clock under load",
            "flop_per_ray_step": flop_step, "kernel": "trace_rays<4, mixed>", "kernel_ms": kmean,
            "issue_bound_note": "the kernel is bound by instruction issue; see profiles/ for its issue-slot use"}

    if rank == 0:
        cpu = None
        cpu_1t = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(g, v, f)
            cpu_1t = cpu_baseline(g, v, f, target_s=8.0, threads=1)
        line = {"metric": METRIC, "value": value, "unit": "ray-steps/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "MAS-like synthetic corona 256(r, 1-30 R_sun) x 180 x 360, FP32 fields; "
                                       "512x512 image +-3 R_sun x 16 freq log 40-800 MHz; step-wise tube, "
                                       "4 neighbours, RK4 h = 2e-3 R_sun",
                           "precision": args.precision, "maps_per_step": len(f), "rays_per_step": int(all_rays),
                           "l2": "inputs larger than L2 (1.06 GB corner-packed grid, 4.19 M rays/step)",
                           "parallelism": f"one job split over {ws} GPU(s): longest-first greedy partition of "
                                          f"(frequency, 64-pixel chunk) items, maps gathered by an all-reduce sum"
                                          if ws > 1 else "1 GPU"},
                "maps_per_s": maps_per_s, "ray_steps_per_step": all_steps / args.steps,
                "gather_ms": float(np.mean(gather_ms)),
                "adjoint_forward_ratio": adjoint["mixed"]["ratio"] if adjoint else None,
                "adjoint": adjoint, "forms": forms, "next1": next1, "step_gate": step_gate,
                "gpu_launches": args.steps,
                "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_1_thread": cpu_1t, "e2e": e2e,
                "clocks": clocks, "peaks_source": peak_src}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def timed_ms(fn, stream, warm=True):
    """One warm call (unless warm=False), then one call timed with CUDA
    events on `stream`."""
    import torch
    if warm:
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def run_forms(ctx, grid, v, f, prec, stream):
    """The other forms on the headline workload (plain FP32 or compensated,
    and the graph-captured persistent batch launch of the same 16 maps), and
    the batching workload: 64 independent requests on the 64x32x64 corona
    (sides 128-1024, 1-8 frequencies, random longitude) at the autotuned step,
    one batched launch against one rt_trace_image per request."""
    import torch

    import corona_synth as cs
    import paper_2606_02413_gb300 as rt
    from paper_2606_02413_gb300 import autotune
    forms = {}
    out = torch.empty((len(f), v.ny, v.nx), dtype=torch.float32, device=f"cuda:{ctx.device}")
    other = rt.RT_PLAIN_F32 if prec == rt.RT_MIXED else rt.RT_MIXED
    o2 = rt.options(precision=other)
    ms2 = timed_ms(lambda: ctx.trace_image(grid, v, f, o2, out=out), stream)
    st2 = ctx.stats()
    forms["plain" if other == rt.RT_PLAIN_F32 else "mixed"] = {
        "ms": ms2, "ray_steps_per_s": st2["ray_steps"] / (ms2 / 1e3), "maps_per_s": len(f) / (ms2 / 1e3)}
    plan = ctx.batch_plan(grid, [cs.Request(v, f)], rt.options(precision=prec))
    ms3 = timed_ms(plan.launch, stream)
    st3 = plan.stats()
    forms["batched"] = {"ms": ms3, "ray_steps_per_s": st3["ray_steps"] / (ms3 / 1e3),
                        "maps_per_s": len(f) / (ms3 / 1e3), "launch": "CUDA graph, longest-first chunks"}
    plan.destroy()

    # the batching workload at the autotuned step (plain FP32 stepping)
    gt, _, _ = cs.tiny_workload()
    grid_t = ctx.load(gt)
    tv = cs.View(0.0, 0.0, 64, 64, -2.5, 2.5, -2.5, 2.5)
    tuned, rep = autotune.tune(ctx, grid_t, tv, cs.log_freqs(8, 40e6, 800e6), rt.options(precision=rt.RT_PLAIN_F32),
                               gate=1e-3, time_side=64)
    ob = rt.options(precision=rt.RT_PLAIN_F32, dtau=tuned.dtau)
    reqs = cs.batch_requests(64)
    n_maps = sum(len(r.freqs_hz) for r in reqs)
    bplan = ctx.batch_plan(grid_t, reqs, ob)
    ms_b = timed_ms(bplan.launch, stream, warm=False)  # kernels and graph machinery are warm by now
    steps_b = bplan.stats()["ray_steps"]
    outs = [torch.empty((len(r.freqs_hz), r.view.ny, r.view.nx), dtype=torch.float32, device=out.device)
            for r in reqs]

    def per_request():
        for r, o in zip(reqs, outs):
            ctx.trace_image(grid_t, r.view, r.freqs_hz, ob, out=o)
    ms_s = timed_ms(per_request, stream, warm=False)
    same = all(torch.equal(x, y) for x, y in zip(bplan.outputs, outs))
    bplan.destroy()
    grid_t.free()
    forms["batch_64"] = {"workload": "64 requests, sides 128-1024, 1-8 frequencies 40-800 MHz, random longitude, "
                                     "64x32x64 corona, plain FP32",
                         "autotuned_dtau": tuned.dtau, "autotune_step_errors": rep["steps"],
                         "maps": n_maps, "ray_steps": steps_b,
                         "batched_ms": ms_b, "batched_maps_per_s": n_maps / (ms_b / 1e3),
                         "per_request_ms": ms_s, "per_request_maps_per_s": n_maps / (ms_s / 1e3),
                         "speedup": ms_s / ms_b, "identical_maps": bool(same)}
    return forms


def run_adjoint(ctx):
    """Adjoint/forward time ratio on the differentiation workload (128x90x180
    corona, 256^2 x 8 frequencies 40-400 MHz) for the misfit
    L = sum (T_b - T_target)^2 against the maps of its perturbed grid, in
    both arithmetic forms: the autograd path (the forward keeps a tape,
    rt_trace_image_tape; the backward reverses it, rt_backward_tape) over the
    plain forward (rt_trace_image); also rt_backward given the forward's
    diagnostics (it traces twice more) and standalone."""
    import torch

    import corona_synth as cs
    import paper_2606_02413_gb300 as rt
    ga, va, fa = cs.adjoint_workload()
    grid_a = ctx.load(ga)
    grid_t = ctx.load(cs.perturbed_target(ga))
    adjoint = {"workload": "Newkirk 128x90x180 grid, 256x256 x 8 freq 40-400 MHz, 4 neighbours",
               "loss": "sum (T_b - T_target)^2, T_target traced through the perturbed grid",
               "ratio_definition": "ratio: rt_backward_tape (the autograd backward) / rt_trace_image; "
                                   "tape_forward_s: rt_trace_image_tape (the autograd forward); "
                                   "ratio_retrace: rt_backward given the forward's diagnostics / rt_trace_image; "
                                   "ratio_standalone: rt_backward with its own counting pass"}
    for nm, pr in (("mixed", rt.RT_MIXED), ("plain", rt.RT_PLAIN_F32)):
        oa = rt.options(precision=pr)
        tgt = ctx.trace_image(grid_t, va, fa, oa)
        ctx.trace_image(grid_a, va, fa, oa)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.trace_image(grid_a, va, fa, oa)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        tbf, dg = ctx.trace_image(grid_a, va, fa, oa, diag=True)
        wgt = 2.0 * (tbf - tgt)
        ctx.backward(grid_a, va, fa, wgt, oa, fwd_diag=dg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.backward(grid_a, va, fa, wgt, oa, fwd_diag=dg)
        torch.cuda.synchronize()
        tbk = time.perf_counter() - t0
        t0 = time.perf_counter()
        ctx.backward(grid_a, va, fa, wgt, oa)
        torch.cuda.synchronize()
        tbs = time.perf_counter() - t0
        ctx.trace_image_tape(grid_a, va, fa, oa)[2].free()  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, tape = ctx.trace_image_tape(grid_a, va, fa, oa)
        torch.cuda.synchronize()
        tft = time.perf_counter() - t0
        used, cap = tape.info()
        tape.backward(wgt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tape.backward(wgt)
        torch.cuda.synchronize()
        tbt = time.perf_counter() - t0
        tape.free()
        adjoint[nm] = {"forward_s": tf, "tape_forward_s": tft, "backward_s": tbt, "ratio": tbt / tf,
                       "tape_slots_used": used, "tape_slots_cap": cap,
                       "backward_retrace_s": tbk, "ratio_retrace": tbk / tf,
                       "backward_standalone_s": tbs, "ratio_standalone": tbs / tf}
    grid_a.free()
    grid_t.free()
    return adjoint


def run_next1(ctx, grid, f, side=128):
    """The paper's comparisons on the headline corona (Sec. 3.3-3.4) at a
    reduced image (side^2 over +-3 R_sun, the 16 frequencies): the disk-mean
    (< 0.5 R_sun) T_b spectrum of refracted rays with the magnification term,
    without it, and of straight lines of sight; and the change the
    magnification term makes to each disk pixel's T_b."""
    import torch

    import corona_synth as cs
    import paper_2606_02413_gb300 as rt
    v = cs.View(0.0, 0.0, side, side, -3.0, 3.0, -3.0, 3.0)
    res = {"image": f"{side}x{side} over +-3 R_sun", "freqs_MHz": [round(float(x) / 1e6, 2) for x in f]}
    maps = {}
    for nm, o in (("traced", rt.options(precision=rt.RT_MIXED)),
                  ("traced_S_off", rt.options(precision=rt.RT_MIXED, s_mode=rt.RT_MAG_OFF)),
                  ("straight_los", rt.options(precision=rt.RT_MIXED, straight=1))):
        tb = ctx.trace_image(grid, v, f, o)
        maps[nm] = tb
        res[f"disk_mean_tb_{nm}"] = [float(x) for x in ctx.disk_mean_tb(v, tb, 0.5).cpu().numpy()]
    torch.cuda.synchronize()
    u = -3.0 + (np.arange(side) + 0.5) * (6.0 / side)
    disk = torch.from_numpy((u[None, :] ** 2 + u[:, None] ** 2) < 1.0).to(maps["traced"].device)
    on, off = maps["traced"], maps["traced_S_off"]
    rel = ((on - off).abs() / off.clamp(min=1.0))[:, disk]
    res["S_term_rel_change_disk_max"] = [float(x) for x in rel.max(dim=1).values.cpu().numpy()]
    res["S_term_rel_change_disk_median"] = [float(x) for x in rel.median(dim=1).values.cpu().numpy()]
    return res


if __name__ == "__main__":
    main()
