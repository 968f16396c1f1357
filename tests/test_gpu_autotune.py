"""The autotuner (step size gated against the library's own fine-step maps,
launch shape timed) and the launch knobs it sets: the tile walk and the
persistent block count change the schedule, never the per-ray result."""
import json

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


def test_launch_knobs_do_not_change_results(rt):
    import torch
    ctx = rt.Context(0)
    g, _, _ = cs.tiny_workload()
    grid = ctx.load(g)
    v = cs.View(0.3, 0.0, 37, 29, -2.5, 2.5, -2.0, 2.4)  # ragged against every tile size
    f = [70e6, 400e6]
    ref, dref = ctx.trace_image(grid, v, f, rt.options(precision=1), diag=True)
    for tile, bps in ((4, 0), (8, 3), (16, 8), (32, 1)):
        tb, d = ctx.trace_image(grid, v, f, rt.options(precision=1, tile=tile, blocks_per_sm=bps), diag=True)
        torch.cuda.synchronize()
        assert torch.equal(tb, ref) and torch.equal(d, dref), (tile, bps)
    assert ctx.stats()["rays"] == 2 * 37 * 29
    with pytest.raises(rt.RtError, match="RT_ERR_ARG"):
        ctx.trace_image(grid, v, f, rt.options(tile=1))


def test_autotune_gate_and_cache(rt, orc, tmp_path):
    from paper_2606_02413_gb300 import autotune
    ctx = rt.Context(0)
    g, _, _ = cs.tiny_workload()
    grid = ctx.load(g)
    v = cs.View(0.0, 0.0, 96, 96, -2.5, 2.5, -2.5, 2.5)
    f = [80e6, 300e6]
    cache = str(tmp_path / "tune.json")
    opts, rep = autotune.tune(ctx, grid, v, f, rt.options(precision=1), gate=1e-3, cache=cache, time_side=64)
    assert opts.dtau in autotune.STEPS and rep["steps"][f"{opts.dtau:g}"] <= 1e-3
    # every larger step in the ladder failed the gate or was taken
    assert all(rep["steps"][f"{h:g}"] > 1e-3 for h in autotune.STEPS if h > opts.dtau) or opts.dtau == max(autotune.STEPS)
    table = json.load(open(cache))
    assert len(table) == 1
    again, rep2 = autotune.tune(ctx, grid, v, f, rt.options(precision=1), gate=1e-3, cache=cache)
    assert (again.dtau, again.tile, again.blocks_per_sm) == (opts.dtau, opts.tile, opts.blocks_per_sm)
    # parity at the tuned step: GPU against the oracle run with the same step
    pix = np.arange(0, 96 * 96, 613).astype(np.int32)
    tb = ctx.trace_image(grid, v, f, opts).cpu().numpy().reshape(2, -1)[:, pix]
    ref = orc.trace(orc.grid_field(g), v, f, orc.default_options(dtau=opts.dtau, tau_stop=30.0), pixels=pix)
    scale = np.maximum(ref["tb"], 1e-2 * ref["tb"].max(axis=1, keepdims=True))
    assert (np.abs(tb - ref["tb"]) <= 1e-3 * scale).all()
