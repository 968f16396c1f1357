"""Oracle test infrastructure: ctypes access to the FP64 CPU oracle.

The oracle (``rt_oracle.cpp``) is a plain, slow FP64 restatement of the
paper's method (Sec. 2-3, Eqs. 1-12).  Only ``tests/``, the package smoke
check and the benchmark's CPU-baseline leg may import this module.  It shares
no code with the CUDA library; the two meet only in the seeded inputs of
``corona_synth``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "rt_oracle.cpp")]
_DEPS = _SRC + [os.path.join(_HERE, "rt_oracle.h"), os.path.join(_HERE, "ad_tape.h")]
# RT_ORACLE_LIB points the tests at another build of the same source (the
# mutation test compiles deliberately broken copies of the oracle).
LIB_PATH = os.environ.get("RT_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")

GRID, UNIFORM, VACUUM, SLAB, NEWKIRK = 0, 1, 2, 3, 4
STEPWISE, TUBE, MAG_OFF = 0, 1, 2
STATUS = {0: "RUNNING", 1: "EXIT_OUTER", 2: "HIT_INNER", 3: "TAU_STOP", 4: "STEP_LIMIT",
          5: "MISS", 6: "NAN"}


class Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("r_min", C.c_double), ("r_max", C.c_double),
                ("n_r", C.c_int), ("n_t", C.c_int), ("n_p", C.c_int),
                ("r", C.c_void_p), ("theta", C.c_void_p), ("phi", C.c_void_p),
                ("ne", C.c_void_p), ("te", C.c_void_p),
                ("ne0", C.c_double), ("te0", C.c_double),
                ("q", C.c_double * 3), ("c", C.c_double)]


class ViewS(C.Structure):
    _fields_ = [("lon", C.c_double), ("lat", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double)]


class Options(C.Structure):
    _fields_ = [("dtau", C.c_double), ("s_mode", C.c_int), ("n_nb", C.c_int),
                ("eps_mode", C.c_int), ("eta", C.c_double), ("delta", C.c_double),
                ("tau_stop", C.c_double), ("max_steps", C.c_int), ("tbc_mode", C.c_int),
                ("tbc_K", C.c_double), ("emission", C.c_int), ("straight", C.c_int),
                ("jitter", C.c_double), ("jitter_seed", C.c_ulonglong)]


class Ray(C.Structure):
    _fields_ = [("tb", C.c_double), ("tau", C.c_double), ("ln_s", C.c_double),
                ("exit", C.c_double * 3), ("alpha", C.c_double),
                ("status", C.c_int), ("steps", C.c_int)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (FP64, OpenMP, no fast-math)."""
    if os.environ.get("RT_ORACLE_LIB"):
        return LIB_PATH
    newest = max(os.path.getmtime(p) for p in _DEPS)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-o", tmp] + _SRC
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            L.orc_c_pe.restype = C.c_double
            L.orc_r_sun_cm.restype = C.c_double
            L.orc_kappa_vac.restype = C.c_double
            L.orc_kappa_vac.argtypes = [C.c_double, C.c_double, C.c_double]
            _lib = L
        return _lib


def default_options(**kw) -> Options:
    o = Options(dtau=2e-3, s_mode=STEPWISE, n_nb=4, eps_mode=0, eta=0.5, delta=1e-3,
                tau_stop=0.0, max_steps=0, tbc_mode=0, tbc_K=0.0, emission=1, straight=0,
                jitter=0.0, jitter_seed=1)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class FieldHandle:
    """An orc_field plus the numpy arrays it points into (kept alive)."""

    def __init__(self, s: Field, keep):
        self.s = s
        self._keep = keep

    @property
    def ptr(self):
        return C.byref(self.s)


def grid_field(g) -> FieldHandle:
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (g.r, g.theta, g.phi, g.ne, g.te)]
    s = Field(kind=GRID, r_min=float(arrs[0][0]), r_max=float(arrs[0][-1]),
              n_r=len(arrs[0]), n_t=len(arrs[1]), n_p=len(arrs[2]),
              r=arrs[0].ctypes.data, theta=arrs[1].ctypes.data, phi=arrs[2].ctypes.data,
              ne=arrs[3].ctypes.data, te=arrs[4].ctypes.data)
    return FieldHandle(s, arrs)


def analytic_field(kind, r_min=1.0, r_max=4.0, ne0=0.0, te0=1e6, q=(0.0, 0.0, 1.0), c=0.0):
    s = Field(kind=kind, r_min=r_min, r_max=r_max, ne0=ne0, te0=te0, c=c)
    s.q[0], s.q[1], s.q[2] = q
    return FieldHandle(s, [])


def view_struct(v) -> ViewS:
    return ViewS(v.lon_rad, v.lat_rad, v.nx, v.ny, v.x0, v.x1, v.y0, v.y1)


def rays_to_dict(out, nf, npix):
    n = nf * npix
    res = {
        "tb": np.array([out[i].tb for i in range(n)]).reshape(nf, npix),
        "tau": np.array([out[i].tau for i in range(n)]).reshape(nf, npix),
        "ln_s": np.array([out[i].ln_s for i in range(n)]).reshape(nf, npix),
        "exit": np.array([list(out[i].exit) for i in range(n)]).reshape(nf, npix, 3),
        "alpha": np.array([out[i].alpha for i in range(n)]).reshape(nf, npix),
        "status": np.array([out[i].status for i in range(n)], dtype=np.int32).reshape(nf, npix),
        "steps": np.array([out[i].steps for i in range(n)], dtype=np.int64).reshape(nf, npix),
    }
    return res


def trace(field: FieldHandle, view, freqs, opts: Options | None = None, pixels=None,
          nthreads: int = 0):
    """Trace pixels (flat iy*nx+ix indices; None = all) at every frequency.
    Returns a dict of [nf, npix] arrays."""
    L = lib()
    opts = opts or default_options()
    freqs = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
    vs = view_struct(view)
    if pixels is None:
        npix = view.nx * view.ny
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32)
        npix = len(pix)
        pix_ptr = pix.ctypes.data_as(C.POINTER(C.c_int))
    out = (Ray * (len(freqs) * npix))()
    rc = L.orc_trace(field.ptr, C.byref(vs), freqs.ctypes.data_as(C.POINTER(C.c_double)),
                     len(freqs), C.byref(opts), pix_ptr, npix, out, nthreads)
    if rc != 0:
        raise ValueError("orc_trace rejected its arguments")
    return rays_to_dict(out, len(freqs), npix)


def trace_path(field: FieldHandle, view, f_hz, pixel, opts: Options | None = None, cap=200000):
    L = lib()
    opts = opts or default_options()
    vs = view_struct(view)
    r = np.zeros((cap, 3))
    k = np.zeros((cap, 3))
    ne = np.zeros(cap)
    te = np.zeros(cap)
    ls = np.zeros(cap)
    n = C.c_int(0)
    ray = Ray()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    rc = L.orc_trace_path(field.ptr, C.byref(vs), C.c_double(f_hz), C.byref(opts), pixel, cap,
                          dp(r), dp(k), dp(ne), dp(te), dp(ls), C.byref(n), C.byref(ray))
    if rc != 0:
        raise ValueError("orc_trace_path rejected its arguments")
    m = min(n.value, cap)
    d = rays_to_dict([ray], 1, 1)
    d = {key: val[0, 0] for key, val in d.items()}
    d.update(r=r[:m], k=k[:m], ne=ne[:m], te=te[:m], ln_s_path=ls[:m], n_nodes=n.value)
    return d


def field_eval(field: FieldHandle, p):
    L = lib()
    p = np.ascontiguousarray(p, dtype=np.float64)
    g = np.zeros(3)
    ne = C.c_double(0)
    te = C.c_double(0)
    rc = L.orc_field_eval(field.ptr, p.ctypes.data_as(C.POINTER(C.c_double)), C.byref(ne),
                          g.ctypes.data_as(C.POINTER(C.c_double)), C.byref(te))
    if rc != 0:
        raise ValueError("bad field")
    return ne.value, g, te.value


def rk4_step(field: FieldHandle, f_hz, h, r, k, straight=0):
    L = lib()
    r = np.array(r, dtype=np.float64)
    k = np.array(k, dtype=np.float64)
    rc = L.orc_rk4_step(field.ptr, C.c_double(f_hz), C.c_double(h), straight,
                        r.ctypes.data_as(C.POINTER(C.c_double)), k.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise ValueError("bad field")
    return r, k


def stepwise_m(field: FieldHandle, f_hz, opts: Options, r, k):
    L = lib()
    r = np.ascontiguousarray(r, dtype=np.float64)
    k = np.ascontiguousarray(k, dtype=np.float64)
    m = C.c_double(0)
    rc = L.orc_stepwise_m(field.ptr, C.c_double(f_hz), C.byref(opts),
                          r.ctypes.data_as(C.POINTER(C.c_double)),
                          k.ctypes.data_as(C.POINTER(C.c_double)), C.byref(m))
    if rc != 0:
        raise ValueError("bad args")
    return m.value


def kappa_vac(ne, te, f_hz):
    return lib().orc_kappa_vac(float(ne), float(te), float(f_hz))


def c_pe():
    return lib().orc_c_pe()


def r_sun_cm():
    return lib().orc_r_sun_cm()


def backward(field: FieldHandle, view, freqs, dL_dTb, opts: Options | None = None, pixels=None,
             nthreads: int = 0):
    """Tape-AD gradient of sum(dL_dTb * T_b) w.r.t. grid n_e and T_e nodes.
    dL_dTb: [nf, npix].  Returns (dL_dne, dL_dte, tb) with grid-shaped grads."""
    L = lib()
    opts = opts or default_options()
    freqs = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
    vs = view_struct(view)
    if pixels is None:
        npix = view.nx * view.ny
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32)
        npix = len(pix)
        pix_ptr = pix.ctypes.data_as(C.POINTER(C.c_int))
    s = field.s
    nn = s.n_r * s.n_t * s.n_p
    g = np.ascontiguousarray(dL_dTb, dtype=np.float64).reshape(-1)
    assert g.size == len(freqs) * npix
    gne = np.zeros(nn)
    gte = np.zeros(nn)
    tb = np.zeros(len(freqs) * npix)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    rc = L.orc_backward(field.ptr, C.byref(vs), dp(freqs), len(freqs), C.byref(opts), pix_ptr, npix,
                        dp(g), dp(gne), dp(gte), dp(tb), nthreads)
    if rc != 0:
        raise ValueError("orc_backward rejected its arguments")
    shp = (s.n_r, s.n_t, s.n_p)
    return gne.reshape(shp), gte.reshape(shp), tb.reshape(len(freqs), npix)


def disk_mean_tb(view, tb, radius=0.5):
    """Mean brightness temperature within ``radius`` R_sun of disk centre, per
    frequency (Sec. 3.4: the near-centre quiet-Sun spectrum of Fig. 10): for
    tb [nf, ny, nx] traced with ``view``, the plain mean over the pixels whose
    centre (u, v) satisfies u^2 + v^2 < radius^2 (0 if none does)."""
    tb = np.asarray(tb, dtype=np.float64).reshape(-1, view.ny, view.nx)
    u = view.x0 + (np.arange(view.nx) + 0.5) * ((view.x1 - view.x0) / view.nx)
    v = view.y0 + (np.arange(view.ny) + 0.5) * ((view.y1 - view.y0) / view.ny)
    inside = (u[None, :] ** 2 + v[:, None] ** 2) < radius * radius
    if not inside.any():
        return np.zeros(tb.shape[0])
    return np.array([m[inside].mean() for m in tb])


C_CM_S = 2.99792458e10               # speed of light [cm/s]
AU_RSUN = 1.495978707e13 / 6.957e10  # 1 AU in R_sun (IAU)


def beam_sigma_pixels(view, f_hz, baseline_m):
    """Standard deviation, in pixels of ``view``, of the circular Gaussian beam
    of an interferometer of maximum baseline B (Sec. 3.3): FWHM = lambda / B
    radians, placed on the image plane at 1 AU."""
    fwhm_rsun = C_CM_S / f_hz / (baseline_m * 100.0) * AU_RSUN
    dx = abs(view.x1 - view.x0) / view.nx
    return fwhm_rsun / math.sqrt(8.0 * math.log(2.0)) / dx


def beam_convolve(view, tb, freqs, baseline_m):
    """The maps tb [nf, ny, nx] convolved with the beam of beam_sigma_pixels:
    separable, rows then columns, zero outside the image, with the samples
    exp(-d^2 / 2 sigma^2) at |d| <= ceil(4 sigma) normalised to sum 1."""
    from scipy.ndimage import convolve1d
    tb = np.asarray(tb, dtype=np.float64).reshape(-1, view.ny, view.nx)
    out = np.empty_like(tb)
    for i, f in enumerate(np.atleast_1d(freqs)):
        sigma = beam_sigma_pixels(view, float(f), baseline_m)
        hw = int(math.ceil(4.0 * sigma))
        d = np.arange(-hw, hw + 1, dtype=np.float64)
        w = np.exp(-0.5 * d * d / (sigma * sigma))
        w /= w.sum()
        rows = convolve1d(tb[i], w, axis=1, mode="constant", cval=0.0)
        out[i] = convolve1d(rows, w, axis=0, mode="constant", cval=0.0)
    return out

