// Device code of librt: field evaluation, RK4, and the warp-cooperative
// ray-bundle kernel (Sec. 2.1 Eqs. 4-12, Sec. 3.2 of arXiv 2606.02413).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rt {

constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxFreq = 64;
constexpr int kThreads = 128;
#ifndef RT_MIN_BLOCKS
#define RT_MIN_BLOCKS 8
#endif
constexpr int kMinBlocks = RT_MIN_BLOCKS;  // __launch_bounds__ occupancy target: 8 x 128 threads per SM
constexpr int kMinBlocksTube = 6;          // tube bundles: the offset evaluation needs more registers

// ------------------------------------------------------------------ grid
// Cells are corner-packed: cell (i, j, k) stores the 8 node values of its
// corners as two float4, corner index a*4 + b*2 + c for the (r, theta, phi)
// offsets (a, b, c), so one evaluation is one 32-byte load of one sector.
// Cell k = n_phi - 1 wraps to node 0 (phi is periodic).
//
// The radial axis (any monotone spacing) is resolved by bins no wider than
// the narrowest cell, so at most one node lies inside a bin; a bin holds
// everything one lookup needs in one 32-byte sector: the cell at its lower
// edge, the node inside it (or +inf), and the base radius and inverse width
// of the two cells it can select.  Cells i = n_r - 1 form an all-zero shell:
// the last cell's bins (and every radius beyond them) select it above r_vac,
// so a lookup there yields n_e = T_e = 0 and a zero gradient (vacuum).
struct __align__(32) RadBin {
  int base;     // cell at the bin's lower edge
  float split;  // R_{base+1} when that node lies inside the bin, else +inf
  float r0;     // R_base
  float inv0;   // 1 / (R_{base+1} - R_base)
  float inv1;   // 1 / (R_{base+2} - R_{base+1}) (used only when split is finite)
  float pad[3];
};

struct GridDev {
  const float4* ne;      // [cells][2]
  const float4* te;      // [cells][2]
  const RadBin* r_bins;  // [r_lut_n]
  const float2* r_cell;  // [n_r - 1]: (R_i, 1 / (R_{i+1} - R_i))
  int n_r, n_t, n_p;
  int r_lut_n;
  float r_lut_inv;             // radial bins from r = 0, each 1 / r_lut_inv wide
  float r_min, r_max, r_vac;  // r_vac = r_max (1 + 1e-6): beyond it, vacuum
  float t0, t_inv, t_last;    // theta_0, 1 / dtheta, n_t - 1
  float p0, p_inv;            // phi_0, n_p / (2 pi)
};

// One 32-byte load through the read-only path (a 256-bit vector load, sm_100
// and later); p must be 32-byte aligned.
__device__ __forceinline__ void ldg8(const void* p, float& v0, float& v1, float& v2, float& v3, float& v4,
                                     float& v5, float& v6, float& v7) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3), "=f"(v4), "=f"(v5), "=f"(v6), "=f"(v7)
      : "l"(p));
}

struct Sample {
  float ne, te, gx, gy, gz;  // n_e, T_e, grad n_e
};

// atan2 for the grid lookup: the argument is reduced to a = min/max in [0, 1],
// atan(a) = a P(a^2) with the degree-7 polynomial fitted by csrc/fit_atan.py
// (max error 3.7e-8 in exact arithmetic, ~2e-7 rad after FP32 rounding), and
// the quadrant of (x, y) restored.  At x = y = 0 the floor on the divisor
// gives a = 0 without a branch.  kYNonNeg: the caller guarantees y >= 0
// (theta from rho >= 0), so the sign of y needs no restoring.
template <bool kYNonNeg = false>
__device__ __forceinline__ float atan2_grid(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float a = __fdividef(mn, fmaxf(mx, 1e-30f));
  const float t = a * a;
  float p = -4.054565173e-03f;
  p = fmaf(p, t, 2.186295542e-02f);
  p = fmaf(p, t, -5.591233286e-02f);
  p = fmaf(p, t, 9.642198762e-02f);
  p = fmaf(p, t, -1.390863067e-01f);
  p = fmaf(p, t, 1.994656605e-01f);
  p = fmaf(p, t, -3.332986085e-01f);
  p = fmaf(p, t, 9.999993356e-01f);
  float r = a * p;
  if (ay > ax) r = 1.57079632679489662f - r;
  if (x < 0.f) r = 3.14159265358979324f - r;
  return kYNonNeg ? r : copysignf(r, y);
}

// Trilinear interpolant in (r, theta, phi) (linear in physical r) and its
// exact gradient chain-ruled to Cartesian:
//   grad f = f_r r_hat + f_theta theta_hat / r + f_phi phi_hat / (r sin theta).
// T_e is interpolated with the same weights when want_te (a per-lane flag:
// only the T_e loads diverge, the evaluation itself stays warp-uniform).
// sample_cell does the corner loads, the interpolation and the chain rule
// for cell (i, j, k) at fractions (u, v, w) of the point (x, y, z).
template <bool kTe>
__device__ __forceinline__ Sample sample_cell_t(const GridDev& G, int i, int j, int k, float u, float v, float w,
                                                float tsel, float inv_dr, float x, float y, float z, float inv_r,
                                                float rho, float inv_rho, bool want_te) {
  Sample s;
  const int cell = (i * (G.n_t - 1) + j) * G.n_p + k;
  float n000, n001, n010, n011, n100, n101, n110, n111;
  ldg8(G.ne + 2 * cell, n000, n001, n010, n011, n100, n101, n110, n111);
  const float d00 = n001 - n000, d01 = n011 - n010, d10 = n101 - n100, d11 = n111 - n110;
  const float a00 = fmaf(w, d00, n000), a01 = fmaf(w, d01, n010);
  const float a10 = fmaf(w, d10, n100), a11 = fmaf(w, d11, n110);
  const float e0 = a01 - a00, e1 = a11 - a10;
  const float b0 = fmaf(v, e0, a00), b1 = fmaf(v, e1, a10);
  const float fu = b1 - b0;
  s.ne = fmaf(u, fu, b0);
  const float fv = fmaf(u, e1 - e0, e0);
  const float g0 = fmaf(v, d01 - d00, d00), g1 = fmaf(v, d11 - d10, d10);
  const float fw = fmaf(u, g1 - g0, g0);

  const float f_r = fu * inv_dr;
  const float f_t = fv * G.t_inv * tsel;
  const float f_p = fw * G.p_inv;
  const float A = f_r * inv_r;
  const float ir2 = inv_r * inv_r;
  const float B = f_t * z * ir2 * inv_rho;   // theta term, x and y components (per x, y)
  const float C = f_p * inv_rho * inv_rho;   // phi term
  const float D = f_t * rho * ir2;           // theta term, z component
  s.gx = fmaf(A + B, x, -C * y);
  s.gy = fmaf(A + B, y, C * x);
  s.gz = fmaf(A, z, -D);
  s.te = 0.f;
  if (kTe && want_te) {
    float t000, t001, t010, t011, t100, t101, t110, t111;
    ldg8(G.te + 2 * cell, t000, t001, t010, t011, t100, t101, t110, t111);
    const float p00 = fmaf(w, t001 - t000, t000), p01 = fmaf(w, t011 - t010, t010);
    const float p10 = fmaf(w, t101 - t100, t100), p11 = fmaf(w, t111 - t110, t110);
    const float q0 = fmaf(v, p01 - p00, p00), q1 = fmaf(v, p11 - p10, p10);
    s.te = fmaf(u, q1 - q0, q0);
  }
  return s;
}

__device__ __forceinline__ Sample sample_cell(const GridDev& G, int i, int j, int k, float u, float v, float w,
                                              float tsel, float inv_dr, float x, float y, float z,
                                              float inv_r, float rho, float inv_rho, bool want_te) {
  return sample_cell_t<true>(G, i, j, k, u, v, w, tsel, inv_dr, x, y, z, inv_r, rho, inv_rho, want_te);
}

__device__ __forceinline__ Sample vacuum_sample() {
  Sample s;
  s.ne = 0.f; s.te = 0.f; s.gx = 0.f; s.gy = 0.f; s.gz = 0.f;
  return s;
}

// Radial cell of r and its base radius and inverse width, from one bin.
__device__ __forceinline__ int radial_lookup(const GridDev& G, float r, float& R, float& inv) {
  // r >= 0 (and a NaN r converts to 0): only the top needs a clamp
  const int bin = min(__float2int_rd(r * G.r_lut_inv), G.r_lut_n - 1);
  float base, split, r0, inv0, inv1, q0, q1, q2;
  ldg8(G.r_bins + bin, base, split, r0, inv0, inv1, q0, q1, q2);
  const bool up = r >= split;
  R = up ? split : r0;
  inv = up ? inv1 : inv0;
  return __float_as_int(base) + (up ? 1 : 0);
}

__device__ __forceinline__ int radial_cell(const GridDev& G, float r) {
  float R, inv;
  return radial_lookup(G, r, R, inv);
}

// The field at (x, y, z): trilinear n_e (and T_e when kTe and want_te) and
// the exact gradient of the n_e interpolant.
template <bool kTe>
__device__ __forceinline__ Sample eval_field_t(const GridDev& G, float x, float y, float z, bool want_te) {
  const float rho2 = fmaf(x, x, y * y);
  const float r2 = fmaf(z, z, rho2);
  const float inv_r = rsqrtf(r2);
  const float r = r2 * inv_r;
  // beyond r_vac the radial lookup selects the all-zero shell: vacuum, exactly
  float R, inv_dr;
  const int i = radial_lookup(G, r, R, inv_dr);
  const float u = (r - R) * inv_dr;

  // on the polar axis (rho = 0) the floor keeps inv_rho finite: rho = 0 and
  // the theta and phi terms of the gradient vanish with x = y = 0
  const float inv_rho = rsqrtf(fmaxf(rho2, 1e-20f));
  const float rho = rho2 * inv_rho;
  // theta cell: clamped to the outermost cells, where the fraction sticks
  // at 0 or 1 and the theta derivative is off (tsel = 0)
  const float tt = (atan2_grid<true>(rho, z) - G.t0) * G.t_inv;
  const int j = min(max(__float2int_rd(tt), 0), G.n_t - 2);
  const float v = fminf(fmaxf(tt - (float)j, 0.f), 1.f);
  const float tsel = (tt > 0.f && tt < G.t_last) ? 1.f : 0.f;
  float ph = atan2_grid(y, x) - G.p0;
  if (ph < 0.f) ph += kTwoPiF;
  if (ph >= kTwoPiF) ph -= kTwoPiF;
  const float pp = ph * G.p_inv;
  const int k = min(max(__float2int_rd(pp), 0), G.n_p - 1);
  const float w = pp - (float)k;
  return sample_cell_t<kTe>(G, i, j, k, u, v, w, tsel, inv_dr, x, y, z, inv_r, rho, inv_rho, want_te);
}

__device__ __forceinline__ Sample eval_field(const GridDev& G, float x, float y, float z, bool want_te) {
  return eval_field_t<true>(G, x, y, z, want_te);
}

// atan(num / den) with relative accuracy for small angles: the Taylor series
// through q^13 for den > 0 and |q| = |num / den| <= 1/4 (truncation below
// 3e-10 relative), else atan2_grid.
__device__ __forceinline__ float atan_ratio(float num, float den) {
  if (den > 0.f && fabsf(num) <= 0.25f * den) {
    const float q = num / den;
    const float t = q * q;
    float p = 1.f / 13.f;
    p = fmaf(p, t, -1.f / 11.f);
    p = fmaf(p, t, 1.f / 9.f);
    p = fmaf(p, t, -1.f / 7.f);
    p = fmaf(p, t, 1.f / 5.f);
    p = fmaf(p, t, -1.f / 3.f);
    return fmaf(q * t, p, q);
  }
  return atan2_grid(num, den);
}

// Evaluation about a base point.  A tube's neighbour ray sits ~1e-3 R_sun
// from its central ray and the stage points of one RK4 step lie within
// h |k| of its node; the tube needs the field's differences over such
// offsets.  Evaluated at the rounded FP32 sum of base and offset, a point
// moves by up to an ulp of |x| (~2e-7 R_sun), 1e-4 of a 1e-3 offset at
// every evaluation, and one that lands within that distance of a cell face
// takes the wrong cell's gradient (a kink jump as large as the whole
// offset difference).  So the base point's (r, theta, phi) are formed once
// per step, exactly as eval_field forms them, and each evaluation forms
// the offsets of r, theta, phi from o without cancellation
// (dr = (2 c.o + o.o) / (r + r_c), dtheta and dphi as the angles between
// c and c + o) and adds them only inside the cell fractions, which then
// keep FP32 precision relative to the cell; the cell is re-chosen from
// those fractions.
struct BasePoint {
  float x, y, z;
  float r, rho;    // |c|, its distance from the z axis
  float tt, pp;    // theta and phi in cell units
};

__device__ __forceinline__ BasePoint base_point(const GridDev& G, float x, float y, float z) {
  BasePoint c;
  c.x = x; c.y = y; c.z = z;
  const float rho2 = fmaf(x, x, y * y);
  const float r2 = fmaf(z, z, rho2);
  c.r = r2 * rsqrtf(r2);
  c.rho = rho2 * ((rho2 > 0.f) ? rsqrtf(rho2) : 0.f);
  c.tt = (atan2_grid<true>(c.rho, z) - G.t0) * G.t_inv;
  float ph = atan2_grid(y, x) - G.p0;
  if (ph < 0.f) ph += kTwoPiF;
  if (ph >= kTwoPiF) ph -= kTwoPiF;
  c.pp = ph * G.p_inv;
  return c;
}

__device__ __forceinline__ Sample eval_field_off(const GridDev& G, const BasePoint& c, float ox, float oy,
                                                 float oz, bool want_te) {
  const float x = c.x + ox, y = c.y + oy, z = c.z + oz;
  const float rho2 = fmaf(x, x, y * y);
  const float r2 = fmaf(z, z, rho2);
  const float inv_r = rsqrtf(r2);
  const float r = r2 * inv_r;
  if (!(r <= G.r_vac)) return vacuum_sample();
  const float inv_rho = (rho2 > 0.f) ? rsqrtf(rho2) : 0.f;
  const float rho = rho2 * inv_rho;
  // coordinate offsets
  const float cxy = fmaf(c.x, ox, c.y * oy);
  const float oxy = fmaf(ox, ox, oy * oy);
  const float sr = r + c.r, srho = rho + c.rho;
  const float dr = (sr > 0.f) ? fmaf(2.f, fmaf(c.z, oz, cxy), fmaf(oz, oz, oxy)) / sr : 0.f;
  const float drho = (srho > 0.f) ? fmaf(2.f, cxy, oxy) / srho : 0.f;
  const float dtt = atan_ratio(fmaf(c.z, drho, -c.rho * oz), fmaf(z, c.z, rho * c.rho)) * G.t_inv;
  const float dpp = atan_ratio(fmaf(c.x, oy, -c.y * ox), fmaf(c.x, x, c.y * y)) * G.p_inv;

  float2 rcell;
  int i = radial_lookup(G, r, rcell.x, rcell.y);
  float u = ((c.r - rcell.x) + dr) * rcell.y;
  if (u < 0.f && i > 0) {
    --i;
    rcell = __ldg(G.r_cell + i);
    u = ((c.r - rcell.x) + dr) * rcell.y;
  } else if (u >= 1.f && i < G.n_r - 2) {
    ++i;
    rcell = __ldg(G.r_cell + i);
    u = ((c.r - rcell.x) + dr) * rcell.y;
  }

  const float tt = c.tt + dtt;
  int j;
  float v, tsel;
  if (tt > 0.f && tt < G.t_last) {
    j = min(__float2int_rd(tt), G.n_t - 2);
    v = (c.tt - (float)j) + dtt;
    if (v < 0.f && j > 0) {
      --j;
      v = (c.tt - (float)j) + dtt;
    } else if (v >= 1.f && j < G.n_t - 2) {
      ++j;
      v = (c.tt - (float)j) + dtt;
    }
    tsel = 1.f;
  } else if (tt <= 0.f) {
    j = 0; v = 0.f; tsel = 0.f;
  } else {
    j = G.n_t - 2; v = 1.f; tsel = 0.f;
  }
  int k = __float2int_rd(c.pp + dpp);
  float w = (c.pp - (float)k) + dpp;
  if (w < 0.f) {
    --k;
    w = (c.pp - (float)k) + dpp;
  } else if (w >= 1.f) {
    ++k;
    w = (c.pp - (float)k) + dpp;
  }
  if (k < 0) k += G.n_p;  // periodic in phi
  else if (k >= G.n_p) k -= G.n_p;
  k = min(max(k, 0), G.n_p - 1);
  return sample_cell(G, i, j, k, u, v, w, tsel, rcell.y, x, y, z, inv_r, rho, inv_rho, want_te);
}

// ------------------------------------------------------------------- RK4
// One RK4 step of dr/dtau = k, dk/dtau = kf grad n_e (kf = -C_pe / (2 f^2),
// i.e. grad(n^2)/2) from (p, k).  Returns G = a1 + a2 + a3 and
// A = a1 + 2 a2 + 2 a3 + a4 so that
//   r' = r + h k + h^2/6 G,   k' = k + h/6 A
// (the textbook RK4 combination written in increment form), and the stage-1
// sample at p.
struct Rk4Out {
  float Gx, Gy, Gz, Ax, Ay, Az;
  float ne1, te1;
};

__device__ __forceinline__ Rk4Out rk4_step(const GridDev& G, float kf, float h, float px, float py,
                                           float pz, float kx, float ky, float kz, bool want_te) {
  Rk4Out o;
  const float hh = 0.5f * h;
  Sample s = eval_field(G, px, py, pz, want_te);
  o.ne1 = s.ne;
  o.te1 = s.te;
  float ax = kf * s.gx, ay = kf * s.gy, az = kf * s.gz;
  o.Gx = ax; o.Gy = ay; o.Gz = az;
  o.Ax = ax; o.Ay = ay; o.Az = az;
  // stage 2
  float qx = fmaf(hh, ax, kx), qy = fmaf(hh, ay, ky), qz = fmaf(hh, az, kz);
  s = eval_field(G, fmaf(hh, kx, px), fmaf(hh, ky, py), fmaf(hh, kz, pz), false);
  ax = kf * s.gx; ay = kf * s.gy; az = kf * s.gz;
  o.Gx += ax; o.Gy += ay; o.Gz += az;
  o.Ax = fmaf(2.f, ax, o.Ax); o.Ay = fmaf(2.f, ay, o.Ay); o.Az = fmaf(2.f, az, o.Az);
  // stage 3
  const float q3x = fmaf(hh, ax, kx), q3y = fmaf(hh, ay, ky), q3z = fmaf(hh, az, kz);
  s = eval_field(G, fmaf(hh, qx, px), fmaf(hh, qy, py), fmaf(hh, qz, pz), false);
  ax = kf * s.gx; ay = kf * s.gy; az = kf * s.gz;
  o.Gx += ax; o.Gy += ay; o.Gz += az;
  o.Ax = fmaf(2.f, ax, o.Ax); o.Ay = fmaf(2.f, ay, o.Ay); o.Az = fmaf(2.f, az, o.Az);
  // stage 4
  s = eval_field(G, fmaf(h, q3x, px), fmaf(h, q3y, py), fmaf(h, q3z, pz), false);
  o.Ax = fmaf(kf, s.gx, o.Ax); o.Ay = fmaf(kf, s.gy, o.Ay); o.Az = fmaf(kf, s.gz, o.Az);
  return o;
}

// One RK4 step of a ray of a tube bundle about the base point b, the
// FP32 node position of the bundle's central ray: the central ray is at
// b + l (l: the low part of its compensated position, 0 in plain FP32)
// with wave vector k, and this lane's ray at offsets (dp, dk) from it (0 on
// the central lane).  Every stage point is b plus an offset that holds
// l, the stage's displacement along k and the lane's own offsets, so each
// evaluation (eval_field_off) resolves it to FP32 precision of the offset.
// Outputs as rk4_step.
__device__ __forceinline__ Rk4Out rk4_step_base(const GridDev& G, float kf, float h, const BasePoint& b,
                                                float lx, float ly, float lz, float kx, float ky, float kz,
                                                float dpx, float dpy, float dpz, float dkx, float dky,
                                                float dkz, bool want_te) {
  Rk4Out o;
  const float hh = 0.5f * h;
  // stage 1 at b + l + dp
  Sample s = eval_field_off(G, b, lx + dpx, ly + dpy, lz + dpz, want_te);
  o.ne1 = s.ne;
  o.te1 = s.te;
  float ax = kf * s.gx, ay = kf * s.gy, az = kf * s.gz;
  o.Gx = ax; o.Gy = ay; o.Gz = az;
  o.Ax = ax; o.Ay = ay; o.Az = az;
  // stages 2 and 3 at b + (l + hh k) + dp + hh (dk [+ hh a1])
  const float mx = fmaf(hh, kx, lx), my = fmaf(hh, ky, ly), mz = fmaf(hh, kz, lz);
  const float s3x = fmaf(hh, fmaf(hh, ax, dkx), dpx), s3y = fmaf(hh, fmaf(hh, ay, dky), dpy),
              s3z = fmaf(hh, fmaf(hh, az, dkz), dpz);
  s = eval_field_off(G, b, mx + fmaf(hh, dkx, dpx), my + fmaf(hh, dky, dpy), mz + fmaf(hh, dkz, dpz), false);
  ax = kf * s.gx; ay = kf * s.gy; az = kf * s.gz;
  o.Gx += ax; o.Gy += ay; o.Gz += az;
  o.Ax = fmaf(2.f, ax, o.Ax); o.Ay = fmaf(2.f, ay, o.Ay); o.Az = fmaf(2.f, az, o.Az);
  // stage 4 at b + (l + h k) + dp + h (dk + hh a2)
  const float s4x = fmaf(h, fmaf(hh, ax, dkx), dpx), s4y = fmaf(h, fmaf(hh, ay, dky), dpy),
              s4z = fmaf(h, fmaf(hh, az, dkz), dpz);
  s = eval_field_off(G, b, mx + s3x, my + s3y, mz + s3z, false);
  ax = kf * s.gx; ay = kf * s.gy; az = kf * s.gz;
  o.Gx += ax; o.Gy += ay; o.Gz += az;
  o.Ax = fmaf(2.f, ax, o.Ax); o.Ay = fmaf(2.f, ay, o.Ay); o.Az = fmaf(2.f, az, o.Az);
  s = eval_field_off(G, b, fmaf(h, kx, lx) + s4x, fmaf(h, ky, ly) + s4y, fmaf(h, kz, lz) + s4z, false);
  o.Ax = fmaf(kf, s.gx, o.Ax); o.Ay = fmaf(kf, s.gy, o.Ay); o.Az = fmaf(kf, s.gz, o.Az);
  return o;
}

// --------------------------------------------------------- transfer bits
struct FreqDev {
  float kf;      // -C_pe / (2 f^2): dk/dtau = kf grad n_e
  float kn2;     // -C_pe / f^2:     n^2 = 1 + kn2 n_e
  float kap_c;   // 9.78e-3 / f^2
  float ln_f;    // ln f
  int out_slab;  // output slab of this frequency
};

// Free-free absorption coefficient in vacuum units [cm^-1] (Dulk 1985,
// pure hydrogen): 9.78e-3 n_e^2 G / (f^2 T^1.5), G = 24.5 + ln T - ln f
// (T > 2e5 K) or 18.2 + 1.5 ln T - ln f.
__device__ __forceinline__ float kappa_vac(float ne, float te, float kap_c, float ln_f) {
  if (!(ne > 0.f) || !(te > 0.f)) return 0.f;
  const float lnT = __logf(te);
  const float g = (te > 2e5f) ? (24.5f + lnT - ln_f) : fmaf(1.5f, lnT, 18.2f - ln_f);
  const float rs = rsqrtf(te);
  return (kap_c * ne) * ne * g * (rs * rs * rs);
}

// 1 - e^-x for x >= 0: Taylor series below 0.05 (truncation < 1e-9
// relative), else through the exponential (no cancellation there).
__device__ __forceinline__ float one_minus_exp_neg(float x) {
  if (x < 0.05f) {
    const float t = fmaf(-x, 0.2f, 1.f);
    const float u = fmaf(-x * 0.25f, t, 1.f);
    const float v = fmaf(-x * (1.f / 3.f), u, 1.f);
    return x * fmaf(-x * 0.5f, v, 1.f);
  }
  return 1.f - __expf(-x);
}

// ln(1 + m): series below |m| = 1e-2 (truncation < 2e-11), else the log.
__device__ __forceinline__ float log1p_small(float m) {
  if (fabsf(m) < 1e-2f) {
    const float a = fmaf(-0.75f, m, 1.f);        // 1 - 3m/4
    const float b = fmaf(-m * (2.f / 3.f), a, 1.f);
    return m * fmaf(-0.5f * m, b, 1.f);          // m - m^2/2 + m^3/3 - m^4/4
  }
  return __logf(fabsf(1.f + m));
}

// Error-free sum a + b = s + e (Knuth TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// a + b = s + e with three operations (Fast2Sum, Dekker 1971): exact when
// the exponent of a is at least that of b.  Used for a ray's position and
// wave vector, whose components outweigh their per-step increments except
// where a component passes within about one increment of zero; there e is
// off by at most an ulp of the increment (~1e-10), once, not accumulating.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Running sum.  kComp = true keeps the rounding error of every addition
// (TwoSum) and carries it, so 10^4-term sums stay near double precision;
// kComp = false is the plain FP32 sum.
template <bool kComp>
struct Acc {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    if (kComp) {
      float s, e;
      two_sum(hi, x, s, e);
      hi = s;
      lo += e;
    } else {
      hi += x;
    }
  }
  __device__ __forceinline__ float val() const { return kComp ? hi + lo : hi; }
};

// -------------------------------------------------------- kernel params
struct RayDiag {
  float exit_pos[3];
  float tau;
  float ln_s;
  int steps;
  int status;
};

enum RayStatus { kExitOuter = 1, kHitInner = 2, kTauStop = 3, kStepLimit = 4, kMiss = 5, kNan = 6 };

// Launch geometry of one image (Sec. 3.2): observer direction o, image axes
// e_u, e_v, and the pixel-centre mapping u = x0 + (ix + 1/2) dx.
struct ViewDev {
  float ox, oy, oz, eux, euy, euz, evx, evy, evz;
  float x0, dx, y0, dy;
  int nx, ny, npix;
  int tile, tiles_x;   // image mode: tickets walk tile x tile pixel blocks (0: rows)
  int tickets;         // tickets per frequency (npix, or padded to whole tiles)
};

// Batched work: one map = (request, frequency) with its output slab; one
// chunk = up to kChunk consecutive pixels of one map.  Chunks are listed
// longest-first; ticket t covers pixel (t mod kChunk) of chunk t / kChunk.
constexpr int kChunkShift = 6;
constexpr int kChunk = 1 << kChunkShift;
struct MapDev {
  FreqDev f;
  int view;           // index into the view table
  float* out;         // [ny][nx] T_b slab of this map
  RayDiag* diag;      // [ny][nx] or null
};
struct ChunkDev {
  int map;
  int pix0;           // first pixel of the chunk
  int count;          // pixels in the chunk (<= kChunk)
  int pad;
};

// Forward state at the start of every kCkptEvery-th central step, written
// (optionally) by the forward kernel for the adjoint's recomputation.
#ifndef RT_CKPT_EVERY
#define RT_CKPT_EVERY 32
#endif
constexpr int kCkptEvery = RT_CKPT_EVERY;
// The state of a ray at node `step` (a multiple of kCkptEvery): what the
// adjoint's recomputation of the following segment starts from.
struct Ckpt {
  float r[3], k[3], rl[3], kl[3];
  float tau_hi, tau_lo, lns_hi, lns_lo;
  int step;
};

struct TraceParams {
  GridDev G;
  float h, h2_6, h_6, h2_12, hrsun;  // step and derived constants, hrsun = h R_sun [cm]
  float eta, eps_fixed;              // eps = eta |dr|, or eps_fixed when > 0
  float tau_stop;                    // <= 0: never
  int max_steps;
  int tbc_mode;
  float tbc_K;
  int emission;
  int straight;
  int blocks_per_sm;                 // persistent blocks per SM (0: as many as fit)
  float tube_delta, inv_delta2;      // tube mode: image-plane offset and 1 / delta^2
  // image mode: one view, nf frequencies, ticket t -> (frequency t / npix, pixel t mod npix)
  ViewDev view;
  int nf;
  FreqDev freq[kMaxFreq];
  float* tb_out;
  RayDiag* diag;
  // batch mode (chunks != null): tickets go through the chunk table
  const ChunkDev* chunks;
  const MapDev* maps;
  const ViewDev* views;
  unsigned int* counter;            // work queue ticket (zeroed before launch)
  unsigned long long* stats;        // [0] ray steps, [1] rays
  unsigned int total;               // tickets
  // optional checkpoints (image mode): ray t owns ckpt[ck_off[t] .. ck_off[t+1]);
  // or, when ck_prev is set (a tape), each checkpoint takes the next pool slot
  // (pool_counter, at most pool_cap), ck_prev links it to the ray's previous
  // one (-1: none) and ck_last[t] names ray t's last one (-1: none)
  Ckpt* ckpt;
  const unsigned long long* ck_off;
  int* ck_prev;
  int* ck_last;
  unsigned long long* pool_counter;
  unsigned long long pool_cap;
  // optional (image mode): rays whose weight here is exactly 0 are not traced
  // (T_b 0, diagnostics zero); the adjoint's passes skip rays that cannot
  // contribute to the gradient
  const float* skip_zero;
};

}  // namespace rt
