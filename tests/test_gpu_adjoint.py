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


def compare_grads(gpu, ref, label):
    g = gpu.cpu().numpy().astype(np.float64).ravel()
    o = ref.ravel()
    rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)
    big = np.abs(o) > 1e-2 * np.abs(o).max()
    per = np.abs(g[big] - o[big]) / np.abs(o[big])
    assert rel <= 5e-3, f"{label}: relative L2 error {rel:.3e}"
    assert per.max() <= 2e-2, f"{label}: worst node {per.max():.3e} of {big.sum()}"
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
