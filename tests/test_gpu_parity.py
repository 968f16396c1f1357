"""GPU parity: librt's CUDA path against the FP64 oracle, element by element
on the same seeded inputs, through the C ABI.

Bars (the strict bars are the tolerances of the method's FP32 form):
  T_b:   |dT_b| <= 1e-3 * max(T_b, 1e-2 * max over the map of T_b);
  exit:  the exit position of a ray ending on a sphere within 1e-4 R_sun;
  status equal; ln(S_N / S_0) within lns_abs where a test states it.

Conditioning.  A ray's path on the trilinear interpolant is chaotic where
stage points fall within rounding distance of a cell face (the
interpolant's gradient jumps there), so on a corona that is rough at the
cell scale no FP32 implementation reproduces every FP64 ray.  The oracle
measures each ray's own sensitivity by re-tracing it with every lookup's r
perturbed by a relative JITTER and theta, phi by 3 JITTER rad.  JITTER =
1e-6 is ten times the GPU's FP32 geometry rounding: a face flip is a rare
event per stage point, and a probe at the rounding amplitude itself (1e-7,
eight seeds) missed rays that the GPU's own rounding did flip (the GPU then
missed the strict bars by 600 times the probe's spread), so the
classification uses the stronger probe.  A ray is well-conditioned when no
seed flips its status and its largest change stays below a tenth of the
bar, for each output separately: T_b; the exit point of a ray ending on a
sphere; ln S where a test checks it.  A ray is held to the strict bar of
every output it is well-conditioned for.  In T_b an ill-conditioned ray is
held to TB_CAP = 1e-2 of the scale; its exit point and ln S are reported,
not bounded (on chaotic rays they differ by up to whole R_sun between two
correct FP32 runs).  Status must match unless it flipped under the probe.
Each test states the fraction of its rays that must be T_b-well-conditioned
(so that the strict bar is not vacuous), measured with the oracle alone:
the step-wise tests on smooth coronae ~100% (floor 90%), the white-noise
corona 87% (floor 80%), tube mode 50-63% (floor 40%: persistent neighbours
carry every face kink to the end of the path), the headline corona's
sampled rays 74% (4% at 40 MHz rising to 100% from 241 MHz; floor 65%).
Each comparison prints, per frequency, the well-conditioned fractions of
each output and the largest errors among well- and ill-conditioned rays.
"""
import numpy as np
import pytest

import corona_synth as cs

pytestmark = pytest.mark.gpu

TB_REL = 1e-3
EXIT_ABS = 1e-4
TB_CAP = 1e-2
JITTER = 1e-6
SEEDS = 6


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


@pytest.fixture(scope="module")
def tiny():
    return cs.tiny_workload()


def smooth_grid():
    """The tiny grid with a smooth, non-symmetric modulation of n_e and T_e."""
    g, _, _ = cs.tiny_workload()
    R, T, P = np.meshgrid(g.r, g.theta, g.phi, indexing="ij")
    return cs.Grid(g.r, g.theta, g.phi, g.ne * (1 + 0.3 * np.sin(2 * T) * np.cos(P - 0.5) * np.exp(-(R - 1))),
                   g.te * (1 + 0.2 * np.cos(T) * np.sin(2 * P)))


def run_gpu(rt, ctx, grid_obj, v, freqs, **opt):
    import torch
    tb, d = ctx.trace_image(grid_obj, v, freqs, rt.options(**opt), diag=True)
    torch.cuda.synchronize()
    nf = len(np.atleast_1d(freqs))
    dd = rt.diag_to_numpy(d)
    out = {"tb": tb.cpu().numpy().reshape(nf, -1).astype(np.float64)}
    for k, a in dd.items():
        out[k] = a.reshape((nf, -1) + a.shape[3:])
    return out


def run_oracle(orc, g, v, freqs, pixels=None, **opt):
    opt.setdefault("tau_stop", 30.0)
    opt.pop("precision", None)
    return orc.trace(orc.grid_field(g), v, freqs, orc.default_options(**opt), pixels=pixels)


def spreads(orc, g, v, freqs, ref, pixels=None, **opt):
    """Per-ray single-precision conditioning of the oracle (T_b, exit, ln S, status flips)."""
    stb = np.zeros_like(ref["tb"])
    sex = np.zeros(ref["tb"].shape)
    sls = np.zeros(ref["tb"].shape)
    flip = np.zeros(ref["tb"].shape, bool)
    for seed in range(1, SEEDS + 1):
        j = run_oracle(orc, g, v, freqs, pixels=pixels, jitter=JITTER, jitter_seed=seed, **dict(opt))
        stb = np.maximum(stb, np.abs(j["tb"] - ref["tb"]))
        sex = np.maximum(sex, np.linalg.norm(j["exit"] - ref["exit"], axis=-1))
        sls = np.maximum(sls, np.abs(j["ln_s"] - ref["ln_s"]))
        flip |= j["status"] != ref["status"]
    return stb, sex, sls, flip


def _scale(ref_tb):
    return np.maximum(ref_tb, np.maximum(1e-2 * ref_tb.max(axis=1, keepdims=True), 1e-30))


def classify(ref, cond, tb_rel=TB_REL, exit_abs=EXIT_ABS, lns_abs=None):
    """Per-output conditioning of each ray (see the module docstring):
    (well_tb, well_exit, well_lns, flip).  A ray is well-conditioned for an
    output when no probe seed flips its status and the probe moves that
    output by less than a tenth of its bar."""
    scale = _scale(ref["tb"])
    ends = (ref["status"] == 1) | (ref["status"] == 2)
    if cond is None:
        ok = np.ones(ref["tb"].shape, bool)
        return ok, ok & ends, ok, ~ok
    stb, sex, sls, flip = cond
    well_tb = ~flip & (stb <= 0.1 * tb_rel * scale)
    well_ex = ~flip & ends & (sex <= 0.1 * exit_abs)
    well_ls = ~flip & (sls <= 0.1 * max(lns_abs if lns_abs is not None else 0.0, 1e-30))
    return well_tb, well_ex, well_ls, flip


def compare(gpu, ref, pixels=None, tb_rel=TB_REL, exit_abs=EXIT_ABS, lns_abs=None, cond=None, label="",
            min_well=0.6, freqs=None):
    """Element-by-element comparison (see the module docstring for the bars):
    T_b of T_b-well-conditioned rays within tb_rel of the scale, of the others
    within TB_CAP; exit points of exit-well-conditioned rays within exit_abs;
    ln S of ln S-well-conditioned rays within lns_abs.  At least min_well of
    the rays must be T_b-well-conditioned.  Returns a report with the
    per-frequency fractions and largest errors."""
    sel = (lambda a: a) if pixels is None else (lambda a: a[:, pixels])
    g_tb, g_st, g_ex, g_ls = sel(gpu["tb"]), sel(gpu["status"]), sel(gpu["exit"]), sel(gpu["ln_s"])
    scale = _scale(ref["tb"])
    dtb = np.abs(g_tb - ref["tb"])
    dex = np.linalg.norm(g_ex - ref["exit"], axis=-1)
    dls = np.abs(g_ls - ref["ln_s"])
    ends = (ref["status"] == 1) | (ref["status"] == 2)
    well, well_ex, well_ls, flip = classify(ref, cond, tb_rel, exit_abs, lns_abs)
    tb_bound = np.where(well, tb_rel * scale, TB_CAP * scale)
    bad_st = ~flip & (g_st != ref["status"])
    assert not bad_st.any(), f"{label}: status differs at {np.argwhere(bad_st)[:5]}"
    bad_tb = dtb > tb_bound
    if bad_tb.any():
        idx = [tuple(i) for i in np.argwhere(bad_tb)[:4]]
        det = [(i, g_tb[i], ref["tb"][i], tb_bound[i], bool(well[i]), cond[0][i] if cond else None) for i in idx]
        raise AssertionError(f"{label}: T_b out of bounds (idx, gpu, oracle, bound, well, spread) {det}; "
                             f"max rel {(dtb / scale).max():.3e}")
    bad_ex = well_ex & (dex > exit_abs)
    if bad_ex.any():
        idx = [tuple(i) for i in np.argwhere(bad_ex)[:4]]
        det = [(i, dex[i], cond[1][i] if cond else None, ref["status"][i]) for i in idx]
        raise AssertionError(f"{label}: exit error of exit-well-conditioned rays (idx, err, spread, status) {det}")
    if lns_abs is not None:
        bad_ls = well_ls & (dls > lns_abs)
        if bad_ls.any():
            idx = [tuple(i) for i in np.argwhere(bad_ls)[:4]]
            det = [(i, g_ls[i], ref["ln_s"][i], cond[2][i] if cond else None) for i in idx]
            raise AssertionError(f"{label}: ln S of ln S-well-conditioned rays out of bounds (idx, gpu, oracle, "
                                 f"spread) {det}")
    rel = dtb / scale

    def mx(a, m):
        return float(a[m].max()) if m.any() else 0.0
    per_f = []
    for fi in range(ref["tb"].shape[0]):
        per_f.append({"f_MHz": None if freqs is None else round(float(freqs[fi]) / 1e6, 2),
                      "well_tb": round(float(well[fi].mean()), 4),
                      "well_exit": round(float(well_ex[fi].sum() / max(ends[fi].sum(), 1)), 4),
                      "well_lns": round(float(well_ls[fi].mean()), 4) if lns_abs is not None else None,
                      "max_tb_rel_well": mx(rel[fi], well[fi]), "max_tb_rel_ill": mx(rel[fi], ~well[fi]),
                      "max_exit_well": mx(dex[fi], well_ex[fi]), "max_exit_ill": mx(dex[fi], ends[fi] & ~well_ex[fi])})
    report = {"label": label, "rays": int(well.size), "well_tb": round(float(well.mean()), 4),
              "well_exit": round(float(well_ex.sum() / max(ends.sum(), 1)), 4),
              "well_lns": round(float(well_ls.mean()), 4) if lns_abs is not None else None,
              "max_tb_rel": float(rel.max()), "max_tb_rel_well": mx(rel, well),
              "max_exit_well": mx(dex, well_ex), "max_lns_well": mx(dls, well_ls) if lns_abs is not None else None,
              "per_frequency": per_f}
    print("parity", report)
    frac = float(well.mean())
    assert frac >= min_well, f"{label}: only {frac:.1%} of rays T_b-well-conditioned (need {min_well:.0%})"
    return report


# ------------------------------------------------------------ field row

def test_field_probe_matches_oracle(rt, ctx, orc):
    """Field evaluation (trilinear n_e, T_e and the exact gradient) at random
    points, including the polar caps, the phi wrap, below r_min and in the
    outer vacuum band, against the oracle's interpolant of the same FP32 node
    values.  The gradient bar scales with the node values: near the poles the
    phi term is a small difference of node values amplified by 1/rho."""
    import torch
    g = smooth_grid()
    g32 = cs.Grid(g.r, g.theta, g.phi, g.ne.astype(np.float32).astype(np.float64),
                  g.te.astype(np.float32).astype(np.float64))
    grid = ctx.load(g)
    F = orc.grid_field(g32)
    rng = np.random.default_rng(4)
    pts = rng.normal(size=(4000, 3))
    pts[:200, :2] *= 1e-3                          # near the poles
    pts[200:400, 1] = np.abs(pts[200:400, 1]) * 1e-4  # just across phi = 0
    pts *= (rng.uniform(0.95, 4.0, size=(4000, 1)) / np.linalg.norm(pts, axis=1, keepdims=True))
    pts = pts.astype(np.float32).astype(np.float64)
    out = ctx.probe_field(grid, pts).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    dr = np.diff(g.r).min()
    dth = g.theta[1] - g.theta[0]
    dph = g.phi[1] - g.phi[0]
    bad = []
    for p, o in zip(pts, out):
        ne, gr, te = orc.field_eval(F, p)
        assert abs(o[0] - ne) <= 1e-5 * abs(ne) + 1e-3, (p, o[0], ne)
        assert abs(o[1] - te) <= 1e-5 * abs(te) + 1e-3, (p, o[1], te)
        r, rho = np.linalg.norm(p), np.hypot(p[0], p[1])
        node_scale = abs(ne) * (1 / dr + 1 / (r * dth) + 1 / (max(rho, 1e-12) * dph))
        if np.linalg.norm(o[2:] - gr) > 1e-4 * np.linalg.norm(gr) + 2e-6 * node_scale:
            # a point within rounding of a cell face takes the neighbour cell's gradient
            bad.append((p.tolist(), o[2:].tolist(), gr.tolist()))
    assert len(bad) <= 4, (len(bad), bad[:3])


def test_field_probe_vacuum_boundary(rt, ctx, orc):
    """Vacuum beyond r_vac = r_max (1 + 1e-6) (reading R4): inside the band the
    last cell extends linearly, as in the oracle; beyond it n_e, T_e and the
    gradient are exactly zero, out to radii far past the grid.  Radii stay
    several FP32 ulps away from r_vac so both sides agree on the side."""
    import torch
    g = smooth_grid()
    g32 = cs.Grid(g.r, g.theta, g.phi, g.ne.astype(np.float32).astype(np.float64),
                  g.te.astype(np.float32).astype(np.float64))
    grid = ctx.load(g)
    F = orc.grid_field(g32)
    rng = np.random.default_rng(11)
    r_max = float(g.r[-1])
    scales = np.array([1 - 1e-3, 1 - 1e-7, 1 + 2e-7, 1 + 3e-6, 1 + 1e-3, 1.5, 10.0, 1e3])
    d = rng.normal(size=(400, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = (d * (r_max * scales[np.arange(400) % len(scales)])[:, None]).astype(np.float32).astype(np.float64)
    out = ctx.probe_field(grid, pts).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    r_vac = r_max * (1 + 1e-6)
    for p, o in zip(pts, out):
        r = np.linalg.norm(p)
        ne, gr, te = orc.field_eval(F, p)
        if r > r_vac:
            assert ne == 0.0 and te == 0.0 and not gr.any(), (r, ne, te)
            assert (o == 0.0).all(), (p, r, o)
        else:
            assert ne > 0 and te > 0
            assert abs(o[0] - ne) <= 1e-5 * abs(ne), (p, o[0], ne)
            assert abs(o[1] - te) <= 1e-5 * abs(te), (p, o[1], te)
            assert np.linalg.norm(o[2:] - gr) <= 1e-3 * np.linalg.norm(gr) + 1e-6 * abs(ne), (p, o[2:], gr)


# ------------------------------------------------------------ strict parity

def test_tiny_full_map_mixed(rt, ctx, orc, tiny):
    """64x64 map of the spherically symmetric corona at 100 MHz, 4 neighbours,
    compensated form: the strict bar on every ray."""
    g, v, f = tiny
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, f, precision=1)
    ref = run_oracle(orc, g, v, f)
    compare(gpu, ref, lns_abs=1e-3, label="tiny mixed")
    assert (np.abs(gpu["steps"] - ref["steps"]) <= 1).all()
    st = ctx.stats()
    assert st["rays"] == 64 * 64 and st["ray_steps"] == int(gpu["steps"].sum())


def test_tiny_full_map_plain(rt, ctx, orc, tiny):
    """Plain FP32 (uncompensated sums): meets the T_b bar; its exit points and
    ln S drift by the accumulated rounding of ~3000 steps (bounded here at
    1e-3 R_sun and 1e-2), which the compensated form removes."""
    g, v, f = tiny
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, f, precision=0)
    ref = run_oracle(orc, g, v, f)
    compare(gpu, ref, exit_abs=1e-3, lns_abs=1e-2, label="tiny plain")


@pytest.mark.parametrize("freq", [40e6, 250e6, 800e6])
def test_tiny_other_frequencies(rt, ctx, orc, tiny, freq):
    g, _, _ = tiny
    v = cs.View(0.0, 0.0, 31, 29, -2.5, 2.5, -2.4, 2.6)  # ragged sizes
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, [freq], precision=1)
    ref = run_oracle(orc, g, v, [freq])
    compare(gpu, ref, lns_abs=1e-3, label=f"tiny {freq / 1e6:.0f} MHz")


@pytest.mark.parametrize("n_nb,s_mode", [(2, 0), (4, 0), (8, 0), (4, 2), (2, 1), (4, 1), (8, 1)])
def test_neighbour_counts_and_modes(rt, ctx, orc, n_nb, s_mode):
    """Step-wise with 2 (paper), 4 and 8 neighbours, magnification off, and
    tube mode with 2, 4, 8 persistent neighbours, on a smooth non-symmetric
    corona seen from an off-axis observer."""
    g = smooth_grid()
    v = cs.View(0.7, 0.3, 13, 7, -2.2, 2.6, -1.9, 2.1)
    freqs = [45e6, 150e6, 700e6]
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, freqs, n_nb=n_nb, s_mode=s_mode, precision=1)
    ref = run_oracle(orc, g, v, freqs, n_nb=n_nb, s_mode=s_mode)
    cond = spreads(orc, g, v, freqs, ref, n_nb=n_nb, s_mode=s_mode)
    compare(gpu, ref, cond=cond, lns_abs=0.0 if s_mode == 2 else 1e-3, label=f"nb{n_nb} mode{s_mode}",
            min_well=TUBE_MIN_WELL if s_mode == 1 else 0.9)


# Tube mode (persistent neighbours) on the trilinear interpolant is far less
# well-conditioned than the step-wise retrace: a neighbour's RK4 stage point
# that crosses a cell face one step earlier or later than in the reference
# changes its acceleration by the face's kink, a jump as large as the whole
# offset difference, and the tube carries it to the end of the path.
# Measured with the oracle's own 1e-6 probe, 50-63% of the tube rays of
# these views are T_b-well-conditioned (and only 23-39% in ln S) against
# ~100% of the step-wise rays; the floor for tube mode is 40%.
TUBE_MIN_WELL = 0.4


@pytest.mark.parametrize("n_nb", [2, 4, 8])
def test_tube_mode_symmetric(rt, ctx, orc, tiny, n_nb):
    """Tube mode on the spherically symmetric corona, per-ray conditioned bars."""
    g, _, _ = tiny
    v = cs.View(0.0, 0.0, 17, 15, -2.4, 2.4, -2.2, 2.5)
    freqs = [70e6, 250e6]
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, freqs, s_mode=1, n_nb=n_nb, precision=1)
    ref = run_oracle(orc, g, v, freqs, s_mode=1, n_nb=n_nb)
    cond = spreads(orc, g, v, freqs, ref, s_mode=1, n_nb=n_nb)
    compare(gpu, ref, cond=cond, lns_abs=1e-3, label=f"tube nb{n_nb}", min_well=TUBE_MIN_WELL)
    assert np.abs(ref["ln_s"]).max() > 1e-3  # the tube does change


def test_rough_corona_conditioned(rt, ctx, orc, tiny):
    """White-noise modulation at the cell scale (the worst case for the
    interpolant's face kinks): matched within each ray's conditioning."""
    g, _, _ = tiny
    rng = np.random.default_rng(3)
    gm = cs.Grid(g.r, g.theta, g.phi, g.ne * (1 + 0.3 * rng.random(g.ne.shape)),
                 g.te * (1 + 0.2 * rng.random(g.ne.shape)))
    v = cs.View(0.7, 0.3, 13, 7, -2.2, 2.6, -1.9, 2.1)
    freqs = [45e6, 150e6]
    grid = ctx.load(gm)
    gpu = run_gpu(rt, ctx, grid, v, freqs, precision=1)
    ref = run_oracle(orc, gm, v, freqs)
    compare(gpu, ref, cond=spreads(orc, gm, v, freqs, ref), label="rough", min_well=0.8)


def test_straight_line_of_sight(rt, ctx, orc, tiny):
    g = smooth_grid()
    v = cs.View(0.3, -0.2, 9, 9, -2.0, 2.0, -2.0, 2.0)
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, [80e6, 400e6], straight=1, precision=1)
    ref = run_oracle(orc, g, v, [80e6, 400e6], straight=1, s_mode=2)
    compare(gpu, ref, label="LOS")


def test_options_edge_cases(rt, ctx, orc, tiny):
    g, _, _ = tiny
    v = cs.View(0.0, 0.0, 6, 5, -4.5, 4.5, -4.5, 4.5)  # corners miss the r_max sphere
    grid = ctx.load(g)
    for opt in (dict(emission=0, tbc_mode=1, tbc_K=1e4), dict(tau_stop=3.0), dict(max_steps=25),
                dict(eps_mode=1, delta=5e-4), dict(dtau=4e-3), dict(tbc_mode=1, tbc_K=2e5)):
        gpu = run_gpu(rt, ctx, grid, v, [120e6, 400e6], precision=1, **opt)
        ref = run_oracle(orc, g, v, [120e6, 400e6], **dict(opt))
        compare(gpu, ref, label=str(opt))
    assert np.any(ref["status"] == 5)


def test_single_pixel_and_max_frequencies(rt, ctx, orc, tiny):
    g, _, _ = tiny
    grid = ctx.load(g)
    v1 = cs.View(0.2, 0.0, 1, 1, 0.3, 0.5, -0.2, 0.0)
    freqs = cs.log_freqs(64, 40e6, 800e6)
    gpu = run_gpu(rt, ctx, grid, v1, freqs, precision=1)
    ref = run_oracle(orc, g, v1, freqs)
    compare(gpu, ref, label="1 pixel x 64 f")


def test_deterministic_and_both_forms_agree(rt, ctx, tiny):
    import torch
    g, v, f = tiny
    grid = ctx.load(g)
    a = ctx.trace_image(grid, v, [60e6, 200e6], rt.options(precision=0))
    b = ctx.trace_image(grid, v, [60e6, 200e6], rt.options(precision=0))
    c = ctx.trace_image(grid, v, [60e6, 200e6], rt.options(precision=1))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert (a - c).abs().max().item() <= 1e-3 * c.abs().max().item()


def test_invalid_arguments(rt, ctx, tiny):
    g, v, f = tiny
    grid = ctx.load(g)
    with pytest.raises(rt.RtError, match="RT_ERR_ARG"):
        ctx.trace_image(grid, v, [], rt.options())
    with pytest.raises(rt.RtError, match="RT_ERR_ARG"):
        ctx.trace_image(grid, v, np.full(65, 1e8), rt.options())
    with pytest.raises(rt.RtError, match="RT_ERR_ARG"):
        ctx.trace_image(grid, v, [-1.0], rt.options())
    for bad in (dict(dtau=0.0), dict(n_nb=3), dict(precision=7), dict(s_mode=9)):
        with pytest.raises(rt.RtError, match="RT_ERR_ARG"):
            ctx.trace_image(grid, v, [1e8], rt.options(**bad))
    ne = g.ne.copy()
    ne[3, 4, 5] = np.nan
    with pytest.raises(rt.RtError, match="RT_ERR_GRID"):
        ctx.load_grid(g.r, g.theta, g.phi, ne, g.te)
    ne = g.ne.copy()
    ne[1, 1, 1] = -1.0
    with pytest.raises(rt.RtError, match="RT_ERR_GRID"):
        ctx.load_grid(g.r, g.theta, g.phi, ne, g.te)
    te = g.te.copy()
    te[0, 0, 0] = 0.0
    with pytest.raises(rt.RtError, match="RT_ERR_GRID"):
        ctx.load_grid(g.r, g.theta, g.phi, g.ne, te)
    r = g.r.copy()
    r[5] = r[4]
    with pytest.raises(rt.RtError, match="RT_ERR_GRID"):
        ctx.load_grid(r, g.theta, g.phi, g.ne, g.te)
    th = g.theta.copy()
    th[3] += 1e-3
    with pytest.raises(rt.RtError, match="RT_ERR_GRID"):
        ctx.load_grid(g.r, th, g.phi, g.ne, g.te)
    # the context still works afterwards
    tb = ctx.trace_image(grid, cs.View(0, 0, 2, 2), [1e8], rt.options())
    ctx.sync()
    assert np.isfinite(tb.cpu().numpy()).all()


def test_device_resident_grid_input(rt, ctx, orc, tiny):
    import torch
    g, _, _ = tiny
    v = cs.View(0.0, 0.0, 8, 8, -2.5, 2.5, -2.5, 2.5)
    grid = ctx.load_grid(g.r, g.theta, g.phi, torch.from_numpy(g.ne).cuda(), torch.from_numpy(g.te).cuda())
    gpu = run_gpu(rt, ctx, grid, v, [100e6], precision=1)
    ref = run_oracle(orc, g, v, [100e6])
    compare(gpu, ref, label="device grid")


def sample_pixels(nx, ny, n, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nx * ny, size=n, replace=False)).astype(np.int32)


def test_global_corona_sampled(rt, ctx, orc):
    """The 256x180x360 MAS-like corona, 512x512 x 16 frequencies, in the
    launch configuration the benchmark times; 48 sampled pixels at every
    frequency against the oracle.  Well-conditioned rays (GLOBAL_MIN_WELL of
    them at least) meet the strict T_b, exit and ln S bars; the others the
    capped conditioned T_b bound."""
    g, v, f = cs.global_workload()
    grid = ctx.load(g)
    gpu = run_gpu(rt, ctx, grid, v, f, precision=1)
    pix = sample_pixels(v.nx, v.ny, 48, seed=1)
    ref = run_oracle(orc, g, v, f, pixels=pix)
    cond = spreads(orc, g, v, f, ref, pixels=pix)
    compare(gpu, ref, pixels=pix, cond=cond, lns_abs=GLOBAL_LNS_ABS, label="global mixed", freqs=f,
            min_well=GLOBAL_MIN_WELL)
    # invariants at full size: every ray finished with a terminal status
    assert np.isin(gpu["status"], [1, 2, 3, 5]).all()
    assert np.isfinite(gpu["tb"]).all() and (gpu["tb"] >= 0).all()


GLOBAL_LNS_ABS = 1e-3
GLOBAL_MIN_WELL = 0.65
