"""The paper's comparison outputs (Sec. 3.3-3.4) on the GPU: the disk-mean
T_b spectrum reduction (rt_disk_mean_tb) against the oracle's plain mean, on
the oracle's own maps and on maps traced by both sides; straight lines of
sight and magnification off are the existing trace modes."""
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


def test_disk_mean_reduction_on_oracle_maps(rt, ctx, orc):
    """The reduction alone: the oracle's FP64 maps (rounded to FP32 as a trace
    would store them) of the symmetric corona at three frequencies, on a
    ragged view; the GPU mean equals the plain FP64 mean of the same FP32
    values up to summation order."""
    import torch
    g, _, _ = cs.tiny_workload()
    v = cs.View(0.0, 0.0, 37, 29, -1.3, 1.1, -0.9, 1.4)
    f = [60e6, 150e6, 600e6]
    ref = orc.trace(orc.grid_field(g), v, f, orc.default_options(tau_stop=30.0))["tb"]
    maps = ref.reshape(len(f), v.ny, v.nx).astype(np.float32)
    for radius in (0.5, 0.3, 2.0, 1e-3):
        want = orc.disk_mean_tb(v, maps.astype(np.float64), radius)
        got = ctx.disk_mean_tb(v, torch.from_numpy(maps).cuda(), radius).cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0.0), (radius, got, want)
    assert orc.disk_mean_tb(v, maps.astype(np.float64), 1e-3).max() == 0.0  # no pixel centre inside


def test_disk_mean_spectrum_traced(rt, ctx, orc):
    """End to end: the disk-mean spectrum of GPU-traced maps (step-wise
    magnification, straight lines of sight, magnification off) against that
    of the oracle's maps, 40-800 MHz, within the T_b bar (1e-3)."""
    import torch
    g, _, _ = cs.tiny_workload()
    v = cs.View(0.0, 0.0, 24, 24, -0.6, 0.6, -0.6, 0.6)
    f = cs.log_freqs(5, 40e6, 800e6)
    grid = ctx.load(g)
    for opt in (dict(), dict(straight=1, s_mode=2), dict(s_mode=2)):
        tb = ctx.trace_image(grid, v, f, rt.options(precision=1, **opt))
        got = ctx.disk_mean_tb(v, tb, 0.5).cpu().numpy()
        torch.cuda.synchronize()
        ref = orc.trace(orc.grid_field(g), v, f, orc.default_options(tau_stop=30.0, **opt))["tb"]
        want = orc.disk_mean_tb(v, ref, 0.5)
        assert np.all(np.abs(got - want) <= 1e-3 * want), (opt, got, want)


@pytest.mark.parametrize("baseline", [15e3, 5e3])
def test_beam_convolution(rt, ctx, orc, baseline):
    """rt_beam_convolve against the oracle's plain separable convolution: on
    random maps of a ragged view at three frequencies (beam sigmas from 0.5 to
    27 pixels, edges included), and on traced maps of the tiny corona."""
    import torch
    v = cs.View(0.0, 0.0, 121, 81, -0.3025, 0.3025, -0.2025, 0.2025)   # square pixels of 0.005 R_sun
    f = np.array([40e6, 150e6, 800e6])
    rng = np.random.default_rng(8)
    maps = rng.uniform(0.0, 1e6, size=(3, v.ny, v.nx)).astype(np.float32)
    got = ctx.beam_convolve(v, torch.from_numpy(maps).cuda(), f, baseline).cpu().numpy()
    want = orc.beam_convolve(v, maps.astype(np.float64), f, baseline)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    g, _, _ = cs.tiny_workload()
    grid = ctx.load(g)
    tb = ctx.trace_image(grid, v, f, rt.options(precision=1))
    got = ctx.beam_convolve(v, tb, f, baseline).cpu().numpy()
    want = orc.beam_convolve(v, tb.cpu().numpy().astype(np.float64), f, baseline)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
