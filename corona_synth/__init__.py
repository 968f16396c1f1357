"""Seeded synthetic coronae, observer views, frequency lists and batch requests.

This module only makes inputs.  It holds none of the ray-tracing or transfer
arithmetic: both the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2606_02413_gb300``) receive the arrays it returns, so the two never
regenerate an input differently.

The stand-in workloads follow the paper's global-MHD input (Sec. 3.1: a
spherical r/theta/phi grid of electron density and temperature, 40-800 MHz
maps).  The real model is not available, so every corona here is synthetic:

* ``newkirk_grid``   - spherically symmetric Newkirk-type corona
                        n_e = 4.2e4 * 10**(4.32 / r) cm^-3, T_e = 1 MK.
* ``mas_like_grid``  - the same background on a stretched radial grid out to
                        30 R_sun, times a seeded lognormal modulation, six
                        Gaussian active-region blobs and coronal-hole
                        sectors.
* ``batch_requests`` - independent image requests of uneven size, frequency
                        count and observer longitude.

Arrays are C-ordered [i_r][i_theta][i_phi] (phi fastest).  theta nodes are
cell-centred, theta_j = (j + 1/2) pi / N_theta; phi nodes are periodic,
phi_k = 2 pi k / N_phi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

R_SUN_CM = 6.957e10  # IAU nominal solar radius [cm]

GRID_SEED = 20260601
BATCH_SEED = 3
TARGET_SEED = 4
FD_CELL_SEED = 44


@dataclass
class Grid:
    """Node coordinates and node values of a spherical coronal grid."""
    r: np.ndarray          # [n_r]   radii in R_sun, strictly increasing
    theta: np.ndarray      # [n_t]   colatitudes in rad, strictly increasing in (0, pi)
    phi: np.ndarray        # [n_p]   longitudes in rad, strictly increasing, periodic with 2 pi
    ne: np.ndarray         # [n_r, n_t, n_p] electron density [cm^-3]
    te: np.ndarray         # [n_r, n_t, n_p] electron temperature [K]

    @property
    def shape(self):
        return self.ne.shape


@dataclass
class View:
    """Observer direction and image-plane extent (lengths in R_sun)."""
    lon_rad: float = 0.0
    lat_rad: float = 0.0
    nx: int = 64
    ny: int = 64
    x0: float = -2.5
    x1: float = 2.5
    y0: float = -2.5
    y1: float = 2.5


@dataclass
class Request:
    """One image request of a batch: a view and its frequencies [Hz]."""
    view: View
    freqs_hz: np.ndarray = field(default_factory=lambda: np.zeros(0))


def theta_cell_centred(n_t: int) -> np.ndarray:
    return (np.arange(n_t) + 0.5) * math.pi / n_t


def phi_periodic(n_p: int) -> np.ndarray:
    return np.arange(n_p) * (2.0 * math.pi / n_p)


def r_log(n_r: int, r_min: float = 1.0, r_max: float = 4.0) -> np.ndarray:
    i = np.arange(n_r, dtype=np.float64)
    return r_min * (r_max / r_min) ** (i / (n_r - 1))


def r_stretched(n_r: int = 256, r_min: float = 1.0, r_max: float = 30.0,
                beta: float = 5.0) -> np.ndarray:
    """Exponentially stretched radii: fine near the surface, coarse far out."""
    i = np.arange(n_r, dtype=np.float64)
    return r_min + (r_max - r_min) * np.expm1(beta * i / (n_r - 1)) / math.expm1(beta)


def newkirk_ne(r):
    """Newkirk-type hydrostatic density profile [cm^-3], r in R_sun."""
    return 4.2e4 * 10.0 ** (4.32 / np.asarray(r, dtype=np.float64))


def newkirk_grid(n_r: int, n_t: int, n_p: int, r_max: float = 4.0,
                 te_k: float = 1.0e6, dtype=np.float64) -> Grid:
    """Spherically symmetric corona: n_e(r) Newkirk, uniform T_e."""
    r = r_log(n_r, 1.0, r_max)
    th = theta_cell_centred(n_t)
    ph = phi_periodic(n_p)
    ne = np.broadcast_to(newkirk_ne(r)[:, None, None], (n_r, n_t, n_p)).astype(dtype)
    te = np.full((n_r, n_t, n_p), te_k, dtype=dtype)
    return Grid(r, th, ph, np.ascontiguousarray(ne), te)


def _node_xyz(r, th, ph):
    st, ct = np.sin(th), np.cos(th)
    sp, cp = np.sin(ph), np.cos(ph)
    x = r[:, None, None] * (st[None, :, None] * cp[None, None, :])
    y = r[:, None, None] * (st[None, :, None] * sp[None, None, :])
    z = r[:, None, None] * np.broadcast_to(ct[None, :, None], (1, len(th), len(ph)))
    return x, y, z


def _smooth_step(x):
    return 0.5 * (1.0 + np.tanh(x))


def mas_like_grid(n_r: int = 256, n_t: int = 180, n_p: int = 360,
                  seed: int = GRID_SEED, n_modes: int = 256, sigma: float = 0.3,
                  corr_len: float = 0.1, device: str | None = None) -> Grid:
    """Global-MHD-like corona on a stretched 1-30 R_sun grid (FP32 fields).

    background Newkirk n_e(r), T_e = 1 MK
      x lognormal modulation exp(sigma g - sigma^2/2); g is a unit-variance
        Gaussian random field with covariance exp(-d^2 / 2 l^2), l = corr_len,
        synthesised from ``n_modes`` random Fourier features at the node
        Cartesian positions
      x 6 Gaussian active-region blobs on the r = 1.05 sphere
        (n_e x U(5, 20), T_e -> U(2, 3) MK, radius U(0.05, 0.15))
      x 0.3 in coronal holes: polar caps theta < 30 deg / > 150 deg and one
        40-deg-wide longitude sector at 30 < theta < 90 deg, tanh edges 3 deg.

    The random-feature sum is evaluated with torch in float32 (on ``device``,
    default CUDA when available): the result is reproducible per device kind.
    """
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    r = r_stretched(n_r)
    th = theta_cell_centred(n_t)
    ph = phi_periodic(n_p)
    x, y, z = _node_xyz(r, th, ph)

    kvec = rng.normal(0.0, 1.0 / corr_len, size=(3, n_modes))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    pts = torch.from_numpy(np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32))
    kt = torch.from_numpy(kvec.astype(np.float32)).to(device)
    pt = torch.from_numpy(phase.astype(np.float32)).to(device)
    g = torch.empty(pts.shape[0], dtype=torch.float32)
    chunk = 1 << 18
    for s in range(0, pts.shape[0], chunk):
        p = pts[s:s + chunk].to(device)
        g[s:s + chunk] = torch.cos(p @ kt + pt).sum(1).cpu()
    g = g.numpy().astype(np.float64).reshape(x.shape) * math.sqrt(2.0 / n_modes)

    ne = newkirk_ne(r)[:, None, None] * np.exp(sigma * g - 0.5 * sigma * sigma)
    te = np.full(ne.shape, 1.0e6)

    # active-region blobs
    for _ in range(6):
        u = rng.uniform(-1.0, 1.0)
        lon = rng.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(1.0 - u * u)
        c = 1.05 * np.array([s * math.cos(lon), s * math.sin(lon), u])
        amp = rng.uniform(5.0, 20.0)
        tblob = rng.uniform(2.0e6, 3.0e6)
        rad = rng.uniform(0.05, 0.15)
        gb = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2.0 * rad * rad))
        ne *= 1.0 + (amp - 1.0) * gb
        te += (tblob - te) * gb

    # coronal holes
    deg = math.pi / 180.0
    edge = 3.0 * deg
    thg = th[None, :, None]
    phg = ph[None, None, :]
    polar = _smooth_step((30 * deg - thg) / edge) + _smooth_step((thg - 150 * deg) / edge)
    lon_c = rng.uniform(0.0, 2.0 * math.pi)
    dphi = np.abs((phg - lon_c + math.pi) % (2.0 * math.pi) - math.pi)
    sector = (_smooth_step((thg - 30 * deg) / edge) * _smooth_step((90 * deg - thg) / edge)
              * _smooth_step((20 * deg - dphi) / edge))
    hole = np.maximum(np.minimum(polar, 1.0), sector)
    ne *= 1.0 - 0.7 * hole

    return Grid(r, th, ph, np.ascontiguousarray(ne, dtype=np.float32),
                np.ascontiguousarray(te, dtype=np.float32))


def log_freqs(n: int, f_lo: float, f_hi: float) -> np.ndarray:
    """n frequencies log-spaced from f_lo to f_hi inclusive [Hz]."""
    if n == 1:
        return np.array([f_lo])
    return f_lo * (f_hi / f_lo) ** (np.arange(n) / (n - 1.0))


# ---------------------------------------------------------------- workloads

def tiny_workload():
    """64x32x64 log-r 1-4 R_sun Newkirk grid (FP64), 64x64 image +-2.5 R_sun,
    one frequency 100 MHz."""
    return newkirk_grid(64, 32, 64, 4.0, dtype=np.float64), View(0.0, 0.0, 64, 64), np.array([100e6])


def global_workload(device=None, nx: int = 512):
    """Stretched 256x180x360 MAS-like grid (FP32), 512x512 image +-3 R_sun,
    16 frequencies log-spaced 40-800 MHz."""
    g = mas_like_grid(device=device)
    v = View(0.0, 0.0, nx, nx, -3.0, 3.0, -3.0, 3.0)
    return g, v, log_freqs(16, 40e6, 800e6)


def batch_requests(n_req: int = 64, seed: int = BATCH_SEED, sides=(128, 256, 512, 1024),
                   max_nf: int = 8, f_lo: float = 40e6, f_hi: float = 800e6,
                   extent: float = 2.5):
    """Independent requests: image side uniform over ``sides``, 1..max_nf
    frequencies log-uniform in [f_lo, f_hi], observer longitude uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_req):
        side = int(rng.choice(np.asarray(sides)))
        nf = int(rng.integers(1, max_nf + 1))
        f = np.exp(rng.uniform(math.log(f_lo), math.log(f_hi), size=nf))
        lon = float(rng.uniform(0.0, 2.0 * math.pi))
        out.append(Request(View(lon, 0.0, side, side, -extent, extent, -extent, extent), f))
    return out


def adjoint_workload():
    """128x90x180 log-r 1-4 R_sun Newkirk grid (FP32), 256x256 image
    +-2.5 R_sun, 8 frequencies log-spaced 40-400 MHz."""
    g = newkirk_grid(128, 90, 180, 4.0, dtype=np.float32)
    return g, View(0.0, 0.0, 256, 256), log_freqs(8, 40e6, 400e6)


def perturbed_target(g: Grid, seed: int = TARGET_SEED, amp: float = 0.1,
                     smooth_cells: float = 1.0) -> Grid:
    """Copy of ``g`` whose n_e is multiplied by 1 + amp * N(0,1) per node,
    the noise field smoothed by a Gaussian of ``smooth_cells`` cells
    (phi periodic, r and theta clamped)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.normal(0.0, 1.0, size=g.ne.shape)
    noise = gaussian_filter(noise, sigma=smooth_cells, mode=("nearest", "nearest", "wrap"))
    ne = (g.ne.astype(np.float64) * (1.0 + amp * noise)).astype(g.ne.dtype)
    return Grid(g.r, g.theta, g.phi, np.ascontiguousarray(ne), g.te.copy())


def fd_cells(shape, n: int = 64, seed: int = FD_CELL_SEED, mask=None):
    """n distinct random node indices (flat, C order) for finite-difference
    checks, drawn from ``mask`` (boolean, same shape) when given."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = np.flatnonzero(mask.ravel()) if mask is not None else np.arange(int(np.prod(shape)))
    return np.sort(rng.choice(pool, size=min(n, pool.size), replace=False))


def precision_workload():
    """512x360x720 log-r 1-4 R_sun Newkirk grid (FP32), 1024x1024 image
    +-2.5 R_sun, 32 frequencies log-spaced 40-800 MHz."""
    g = newkirk_grid(512, 360, 720, 4.0, dtype=np.float32)
    return g, View(0.0, 0.0, 1024, 1024), log_freqs(32, 40e6, 800e6)
