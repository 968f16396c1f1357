"""rt_backward (the adjoint kernel) against the oracle's tape reverse-mode
gradient (itself pinned to FP64 central differences in the oracle pins), on
the same seeded inputs: dL/dn_e and dL/dT_e at every grid node for
L = sum(w * T_b) with random weights w.

Bar: relative L2 error over all nodes <= 5e-3, and <= 2e-2 on each node
whose oracle gradient exceeds 1% of the largest.  The reverse sweep runs in
FP32 with atomics (summation order varies), and the trajectory sensitivity
it carries amplifies FP32 rounding the way the forward's conditioning does.
"""
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


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def smooth_grid(nr=24, nt=16, npp=24):
    g = cs.newkirk_grid(nr, nt, npp, 4.0)
    R, T, P = np.meshgrid(g.r, g.theta, g.phi, indexing="ij")
    return cs.Grid(g.r, g.theta, g.phi, g.ne * (1 + 0.3 * np.sin(2 * T) * np.cos(P - 0.5) * np.exp(-(R - 1))),
                   g.te * (1 + 0.2 * np.cos(T) * np.sin(2 * P)))


def grad_errors(gpu, ref):
    """Relative L2 error over all nodes, and the worst relative error on the
    nodes whose oracle gradient exceeds 1% of the largest."""
    g = gpu.cpu().numpy().astype(np.float64).ravel()
    o = ref.ravel()
    rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)
    big = np.abs(o) > 1e-2 * np.abs(o).max()
    per = np.abs(g[big] - o[big]) / np.abs(o[big])
    return float(rel), float(per.max()), int(big.sum())


def compare_grads(gpu, ref, label, l2=5e-3, node=2e-2):
    rel, worst, nbig = grad_errors(gpu, ref)
    assert rel <= l2, f"{label}: relative L2 error {rel:.3e}"
    assert worst <= node, f"{label}: worst node {worst:.3e} of {nbig}"
    return rel


@pytest.mark.parametrize("s_mode,freqs", [(2, [80e6, 300e6]), (0, [80e6, 300e6]), (0, [600e6])])
def test_adjoint_matches_oracle(rt, ctx, orc, s_mode, freqs):
    import torch
    g = smooth_grid()
    v = cs.View(0.4, 0.2, 5, 4, -1.6, 1.6, -1.4, 1.4)
    h = 1e-2
    rng = np.random.default_rng(9)
    w = rng.normal(size=(len(freqs), v.ny, v.nx))
    grid = ctx.load(g)
    opts = rt.options(precision=1, s_mode=s_mode, dtau=h)
    dne, dte, tb = ctx.backward(grid, v, freqs, w, opts, want_tb=True)
    torch.cuda.synchronize()
    gne, gte, tb_o = orc.backward(orc.grid_field(g), v, freqs, w.reshape(len(freqs), -1),
                                  orc.default_options(s_mode=s_mode, dtau=h, tau_stop=30.0))
    scale = np.maximum(tb_o, 1e-2 * tb_o.max())
    assert (np.abs(tb.cpu().numpy().reshape(tb_o.shape) - tb_o) <= 1e-3 * scale).all()
    compare_grads(dne, gne, f"dne mode{s_mode}")
    compare_grads(dte, gte, f"dte mode{s_mode}")


def test_adjoint_linear_in_weights_and_zero(rt, ctx):
    import torch
    g = smooth_grid()
    v = cs.View(0.0, 0.0, 4, 4, -1.5, 1.5, -1.5, 1.5)
    grid = ctx.load(g)
    opts = rt.options(precision=1, dtau=1e-2)
    w = np.random.default_rng(1).normal(size=(1, 4, 4))
    a = ctx.backward(grid, v, [150e6], w, opts)
    b = ctx.backward(grid, v, [150e6], 2 * w, opts)
    z = ctx.backward(grid, v, [150e6], 0 * w, opts)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.allclose(2 * x, y, rtol=1e-4, atol=1e-30 + 1e-6 * x.abs().max().item())
    assert all(float(t.abs().max()) == 0.0 for t in z)


def test_autograd_function(rt, ctx):
    import torch
    g = smooth_grid()
    v = cs.View(0.0, 0.0, 3, 3, -1.2, 1.2, -1.2, 1.2)
    ne = torch.tensor(g.ne, dtype=torch.float32, device="cuda", requires_grad=True)
    te = torch.tensor(g.te, dtype=torch.float32, device="cuda", requires_grad=True)
    opts = rt.options(precision=1, dtau=1e-2)
    tb = rt.RayTraceFn.apply(ne, te, ctx, g.r, g.theta, g.phi, v, [200e6], opts)
    loss = (tb ** 2).sum() * 1e-12
    loss.backward()
    grid = ctx.load(g)
    dne, dte = ctx.backward(grid, v, [200e6], 2e-12 * tb.detach(), opts)
    torch.cuda.synchronize()
    assert torch.allclose(ne.grad, dne, rtol=1e-5, atol=1e-30 + 1e-6 * dne.abs().max().item())
    assert torch.allclose(te.grad, dte, rtol=1e-5, atol=1e-30 + 1e-6 * dte.abs().max().item())


def test_backward_reuses_forward_diag(rt, ctx):
    """fwd_diag (the forward's step counts) spares the counting pass and gives
    the same gradients; a diag of another forward is refused."""
    import torch
    g = smooth_grid()
    v = cs.View(0.3, 0.1, 6, 5, -1.8, 1.8, -1.6, 1.6)
    grid = ctx.load(g)
    opts = rt.options(precision=1, dtau=1e-2)
    w = torch.as_tensor(np.random.default_rng(4).normal(size=(1, v.ny, v.nx)), dtype=torch.float32, device="cuda")
    _, d = ctx.trace_image(grid, v, [60e6], opts, diag=True)
    a = ctx.backward(grid, v, [60e6], w, opts, fwd_diag=d)
    b = ctx.backward(grid, v, [60e6], w, opts)
    torch.cuda.synchronize()
    for x, y in zip(a, b):  # equal up to the order of the float atomics
        assert torch.allclose(x, y, rtol=1e-4, atol=1e-30 + 1e-5 * y.abs().max().item())
    _, d_other = ctx.trace_image(grid, v, [400e6], opts, diag=True)  # other frequency: other step counts
    assert not torch.equal(d_other[..., 5], d[..., 5])
    with pytest.raises(RuntimeError, match="fwd_diag"):
        ctx.backward(grid, v, [60e6], w, opts, fwd_diag=d_other)


def test_tape_forward_and_reverse(rt, ctx):
    """rt_trace_image_tape: the forward of rt_trace_image (identical T_b and
    diagnostics) with one pool slot per started 32-step segment of every ray;
    rt_backward_tape gives rt_backward's gradients, is linear in the weights
    and can be reversed again; a pool that overflows falls back to tracing
    again, with the same gradients."""
    import torch
    g = smooth_grid()
    v = cs.View(0.3, 0.1, 6, 5, -1.8, 1.8, -1.6, 1.6)
    f = [60e6, 250e6]
    grid = ctx.load(g)
    opts = rt.options(precision=1, dtau=1e-2)
    tb_t, d_t, tape = ctx.trace_image_tape(grid, v, f, opts)
    tb, d = ctx.trace_image(grid, v, f, opts, diag=True)
    torch.cuda.synchronize()
    assert torch.equal(tb_t, tb) and torch.equal(d_t, d)
    steps = d[..., 5].cpu().numpy().astype(np.int64)
    used, cap = tape.info()
    assert used == int(((steps - 1) // 32 + 1)[steps > 0].sum()) and used <= cap
    w = torch.as_tensor(np.random.default_rng(5).normal(size=(len(f), v.ny, v.nx)), dtype=torch.float32,
                        device="cuda")
    a = tape.backward(w)
    a2 = tape.backward(2 * w)
    b = ctx.backward(grid, v, f, w, opts)
    small = ctx.trace_image_tape(grid, v, f, opts, pool_bytes=72 * 3)[2]
    su, sc = small.info()
    assert sc == 3 and su > sc
    c = small.backward(w)
    torch.cuda.synchronize()
    for x, x2, y, z in zip(a, a2, b, c):  # equal up to the order of the float atomics
        tol = 1e-30 + 1e-5 * y.abs().max().item()
        assert torch.allclose(x, y, rtol=1e-4, atol=tol)
        assert torch.allclose(2 * x, x2, rtol=1e-4, atol=2 * tol)
        assert torch.allclose(z, y, rtol=1e-4, atol=tol)
    tape.free()
    small.free()


@pytest.fixture(scope="module")
def misfit_case(orc):
    """The differentiation workload (128x90x180 corona, 256x256 x 8 frequencies
    40-400 MHz, step 2e-3 R_sun, 4 step-wise neighbours): the misfit
    L = sum (T_b - T_target)^2 over 32 seeded pixels of the image at all 8
    frequencies (the oracle's cost bounds the sample), T_target traced by the
    oracle through the perturbed copy of the grid (n_e x (1 + 0.1 N(0,1)),
    smoothed over one cell).  Holds the oracle's side: its T_b, its tape
    gradient for dL/dT_b = 2 (T_b - T_target), and central differences of L
    on 64 n_e and 32 T_e nodes drawn among those with a gradient above 1e-3
    of the largest.

    Step of the differences: a relative 1e-6 of the node value.  The
    trilinear interpolant's gradient jumps at cell faces, so L is smooth only
    between the values at which some RK4 stage point crosses a face; the
    step must be small enough that rarely happens (at 1e-4, 7 of 12 nodes
    straddled one) and large enough to stay above the FP64 rounding of
    ~3000-step paths (at 1e-8 the differences scatter by 1e-2)."""
    g, v, f = cs.adjoint_workload()
    gt = cs.perturbed_target(g)
    rng = np.random.default_rng(41)
    pix = np.sort(rng.choice(v.nx * v.ny, size=32, replace=False)).astype(np.int32)
    opts = orc.default_options(tau_stop=30.0)
    tgt = orc.trace(orc.grid_field(gt), v, f, opts, pixels=pix)["tb"]
    ne64, te64 = g.ne.astype(np.float64), g.te.astype(np.float64)

    def loss(ne, te):
        r = orc.trace(orc.grid_field(cs.Grid(g.r, g.theta, g.phi, ne, te)), v, f, opts, pixels=pix)
        return float(((r["tb"] - tgt) ** 2).sum()), r

    L0, r0 = loss(ne64, te64)
    w = 2.0 * (r0["tb"] - tgt)
    gne, gte, _ = orc.backward(orc.grid_field(g), v, f, w, opts, pixels=pix)
    fd = {}
    for which, n, tape, base in (("ne", 64, gne, ne64), ("te", 32, gte, te64)):
        cells = cs.fd_cells(tape.shape, n=n, mask=np.abs(tape) > 1e-3 * np.abs(tape).max())
        vals = []
        for c in cells:
            d = 1e-6 * base.flat[c]
            side = []
            for sgn in (1.0, -1.0):
                a = base.copy()
                a.flat[c] += sgn * d
                L, r = loss(a, te64) if which == "ne" else loss(ne64, a)
                event = bool((r["steps"] != r0["steps"]).any() or (r["status"] != r0["status"]).any())
                side.append((L, event))
            vals.append(((side[0][0] - side[1][0]) / (2 * d), side[0][1] or side[1][1]))
        fd[which] = (cells, vals)
    return dict(g=g, v=v, f=f, pix=pix, tgt=tgt, w=w, gne=gne, gte=gte, fd=fd)


# Bars of the differentiation workload, by arithmetic form.  The
# compensated form: worst node (of those above 1% of the largest gradient)
# against the tape 5e-2 (measured 3.2e-2), every finite-difference node 1e-2
# with the oracle's weights and with the GPU's own (measured 1.3e-3, 2.0e-3).
# The plain FP32 form accumulates the position and wave vector without
# compensation, so its path drifts from the FP64 one (exit points by up to
# 1e-3 R_sun on the tiny corona) and gradients of single nodes follow
# (measured: worst node 0.15, own-weight T_e node 1.4e-2): it is held to
# 0.2 and 2e-2 there, to the same L2 and oracle-weight bars otherwise.
DIFF_NODE_BAR = {1: 5e-2, 0: 0.2}
DIFF_OWN_FD_BAR = {1: 1e-2, 0: 2e-2}


@pytest.mark.parametrize("precision", [1, 0])
def test_differentiation_workload_against_tape_and_fd(rt, ctx, misfit_case, precision):
    """rt_backward on the differentiation workload's misfit (Sec. 2.1 Eqs. 4-12
    differentiated; the workload's step 2e-3 R_sun) against
      (a) the oracle's FP64 tape adjoint with the same dL/dT_b, at every node
          (relative L2 <= 5e-3; DIFF_NODE_BAR on nodes above 1% of the
          largest), and
      (b) the FP64 central differences of the oracle's misfit (misfit_case),
          <= 1e-2 per node.  A node whose +-step changes a ray's step count or
          status, or where the tape adjoint (which holds the discrete events
          fixed) and the differences disagree by more than 2e-3, straddles a
          discrete event and is excluded with a count; at least 3/4 of the
          nodes must remain.
    The GPU side's own dL/dT_b = 2 (T_b - T_target), from its own maps, is
    checked against the differences (b) too."""
    import torch
    M = misfit_case
    g, v, f, pix, tgt = M["g"], M["v"], M["f"], M["pix"], M["tgt"]
    grid = ctx.load(g)
    o = rt.options(precision=precision)
    tb_gpu = ctx.trace_image(grid, v, f, o).cpu().numpy().reshape(len(f), -1)[:, pix].astype(np.float64)
    wmap = np.zeros((len(f), v.ny * v.nx))
    wmap[:, pix] = M["w"]
    dne, dte = ctx.backward(grid, v, f, wmap.reshape(len(f), v.ny, v.nx), o)
    wmap[:, pix] = 2.0 * (tb_gpu - tgt)
    dne_own, dte_own = ctx.backward(grid, v, f, wmap.reshape(len(f), v.ny, v.nx), o)
    torch.cuda.synchronize()
    report = {"precision": precision, "tape_ne": grad_errors(dne, M["gne"]), "tape_te": grad_errors(dte, M["gte"])}
    for which, tape, gpu, own in (("ne", M["gne"], dne, dne_own), ("te", M["gte"], dte, dte_own)):
        cells, vals = M["fd"][which]
        gg = gpu.cpu().numpy().astype(np.float64).ravel()
        go = own.cpu().numpy().astype(np.float64).ravel()
        errs, errs_own, excluded = [], [], 0
        for c, (d_fd, event) in zip(cells, vals):
            if event or abs(tape.flat[c] - d_fd) > 2e-3 * abs(d_fd):
                excluded += 1
                continue
            errs.append(abs(gg[c] - d_fd) / abs(d_fd))
            errs_own.append(abs(go[c] - d_fd) / abs(d_fd))
        report[which] = {"cells": len(cells), "excluded": excluded, "max_rel_err": max(errs),
                         "max_rel_err_own_weights": max(errs_own)}
    print("differentiation workload", report)
    for which in ("ne", "te"):
        rel, worst, _ = report["tape_" + which]
        assert rel <= 5e-3, (which, report)
        assert worst <= DIFF_NODE_BAR[precision], (which, report)
        r = report[which]
        assert r["cells"] - r["excluded"] >= 0.75 * r["cells"], (which, r)
        assert r["max_rel_err"] <= 1e-2, (which, r)
        assert r["max_rel_err_own_weights"] <= DIFF_OWN_FD_BAR[precision], (which, r)
