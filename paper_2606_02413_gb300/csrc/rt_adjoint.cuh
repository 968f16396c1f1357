// Reverse-mode (adjoint) building blocks and the adjoint ray-bundle kernel.
//
// The adjoint differentiates the discrete forward computation (Sec. 2.1
// Eqs. 4-12, Sec. 3.2) with respect to the grid node values of n_e and T_e,
// holding the discrete events fixed (cell indices, the basis axis branch,
// the step count and the termination step), the convention of the FP64
// oracle's tape adjoint.
//
// Interpolant derivatives used here, for a cell with corner values N_c and
// trilinear weights w_c(u, v, w):
//   value       f = sum_c w_c N_c,     d f / d N_c = w_c,     grad f as forward
//   gradient    g = sum_c grad w_c N_c, lambda . d g / d N_c = lambda . grad w_c
//               = sum_a (lambda . grad a) d w_c / d a   (a = u, v, w)
//   position    d (lambda . g) / d x = H lambda, the Hessian of the interpolant
//               applied to lambda, obtained as the tangent of g evaluated on
//               dual numbers x + lambda (cell held fixed).
#pragma once
#include "rt_rays.cuh"

namespace rt {

// ------------------------------------------------------------- dual numbers
struct Dl {
  float v, d;
};
__device__ __forceinline__ Dl dl(float v) { return {v, 0.f}; }
__device__ __forceinline__ Dl operator+(Dl a, Dl b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dl operator-(Dl a, Dl b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dl operator*(Dl a, Dl b) { return {a.v * b.v, fmaf(a.d, b.v, a.v * b.d)}; }
__device__ __forceinline__ Dl operator*(float s, Dl a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dl operator-(Dl a) { return {-a.v, -a.d}; }

// --------------------------------------------------------- cell geometry
struct CellGeom {
  int i, j, k, k1;           // cell and wrapped phi neighbour
  float u, v, w, tsel;       // fractions; tsel = 0 in the clamped theta caps
  Vec du, dv, dw;            // Cartesian gradients of u, v, w
  float inv_r, rho, inv_rho; // 1 / |x|, distance from the z axis and its inverse (0 on the axis)
  bool vac;                  // beyond the outer band
};

__device__ __forceinline__ CellGeom cell_geom(const GridDev& G, float x, float y, float z) {
  CellGeom c;
  const float rho2 = fmaf(x, x, y * y);
  const float r2 = fmaf(z, z, rho2);
  const float inv_r = rsqrtf(r2);
  const float r = r2 * inv_r;
  c.vac = !(r <= G.r_vac);
  if (c.vac) {
    c.i = c.j = c.k = c.k1 = 0;
    c.u = c.v = c.w = c.tsel = 0.f;
    c.du = c.dv = c.dw = {0.f, 0.f, 0.f};
    c.inv_r = c.rho = c.inv_rho = 0.f;
    return c;
  }
  float2 rc;
  c.i = radial_lookup(G, r, rc.x, rc.y);
  c.u = (r - rc.x) * rc.y;
  const float inv_rho = (rho2 > 0.f) ? rsqrtf(rho2) : 0.f;
  const float rho = rho2 * inv_rho;
  c.inv_r = inv_r;
  c.rho = rho;
  c.inv_rho = inv_rho;
  // theta cell as in the field evaluation: clamped to the outermost cells,
  // where the fraction sticks at 0 or 1 and the theta derivative is off
  const float tt = (atan2_grid<true>(rho, z) - G.t0) * G.t_inv;
  c.j = min(max(__float2int_rd(tt), 0), G.n_t - 2);
  c.v = fminf(fmaxf(tt - (float)c.j, 0.f), 1.f);
  c.tsel = (tt > 0.f && tt < G.t_last) ? 1.f : 0.f;
  float ph = atan2_grid(y, x) - G.p0;
  if (ph < 0.f) ph += kTwoPiF;
  if (ph >= kTwoPiF) ph -= kTwoPiF;
  const float pp = ph * G.p_inv;
  c.k = min(max(__float2int_rd(pp), 0), G.n_p - 1);
  c.w = pp - (float)c.k;
  c.k1 = (c.k + 1 == G.n_p) ? 0 : c.k + 1;
  // grad u = r_hat / dr; grad v = theta_hat / (r dtheta); grad w = phi_hat / (rho dphi)
  const float a = rc.y * inv_r;
  c.du = {a * x, a * y, a * z};
  const float ir2 = inv_r * inv_r;
  const float bt = c.tsel * G.t_inv * ir2;
  c.dv = {bt * z * x * inv_rho, bt * z * y * inv_rho, -bt * rho};
  const float bp = G.p_inv * inv_rho * inv_rho;
  c.dw = {-bp * y, bp * x, 0.f};
  return c;
}

__device__ __forceinline__ long node_index(const GridDev& G, const CellGeom& c, int a, int b, int cc) {
  return ((long)(c.i + a) * G.n_t + (c.j + b)) * G.n_p + (cc ? c.k1 : c.k);
}

// Value scatter: d/dN_c of (lam_ne n_e + lam_te T_e) = w_c (lam_ne, lam_te);
// returns lam_ne grad n_e + lam_te grad T_e (the position adjoint).
__device__ __forceinline__ Vec value_adjoint(const GridDev& G, float x, float y, float z, float lam_ne, float lam_te,
                                             float* dne, float* dte) {
  const CellGeom c = cell_geom(G, x, y, z);
  if (c.vac) return {0.f, 0.f, 0.f};
  const int cell = (c.i * (G.n_t - 1) + c.j) * G.n_p + c.k;
  const float4 n0 = __ldg(G.ne + 2 * cell), n1 = __ldg(G.ne + 2 * cell + 1);
  const float4 t0 = __ldg(G.te + 2 * cell), t1 = __ldg(G.te + 2 * cell + 1);
  const float nv[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
  const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
  const float wu[2] = {1.f - c.u, c.u}, wv[2] = {1.f - c.v, c.v}, ww[2] = {1.f - c.w, c.w};
  const float sg[2] = {-1.f, 1.f};
  float fu = 0.f, fv = 0.f, fw = 0.f, tu = 0.f, tvv = 0.f, tw = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int q = a * 4 + b * 2 + cc;
        const float wgt = wu[a] * wv[b] * ww[cc];
        const long id = node_index(G, c, a, b, cc);
        if (lam_ne != 0.f) atomicAdd(dne + id, lam_ne * wgt);
        if (lam_te != 0.f) atomicAdd(dte + id, lam_te * wgt);
        const float gu = sg[a] * wv[b] * ww[cc], gv = wu[a] * sg[b] * ww[cc], gw = wu[a] * wv[b] * sg[cc];
        fu = fmaf(gu, nv[q], fu); fv = fmaf(gv, nv[q], fv); fw = fmaf(gw, nv[q], fw);
        tu = fmaf(gu, tv[q], tu); tvv = fmaf(gv, tv[q], tvv); tw = fmaf(gw, tv[q], tw);
      }
  const float an = lam_ne * fu + lam_te * tu, bn = lam_ne * fv + lam_te * tvv, cn = lam_ne * fw + lam_te * tw;
  return {an * c.du.x + bn * c.dv.x + cn * c.dw.x, an * c.du.y + bn * c.dv.y + cn * c.dw.y,
          an * c.du.z + bn * c.dv.z + cn * c.dw.z};
}

// Per-thread accumulator of the n_e node adjoints of one cell, in shared
// memory laid out [corner][thread] (a warp's accesses hit distinct banks).
// The force adjoints of a step lie within a few 1e-3 R_sun of its node, and
// mostly in the node's cell: they add here, and the sums reach the grid with
// 8 atomics when the node moves to another cell or the ray ends, instead of
// 8 atomics per force adjoint.  Stage points in another cell scatter directly.
struct NodeAcc {
  float* v;    // v[q * kThreads], corner q = 4 a + 2 b + c
  int* key;    // the cell held (-1: none)
  long* base;  // node index of its corner (0, 0, 0)
  int* dk1;    // k1 - k: 1, or 1 - n_phi across the phi seam
};

__device__ __forceinline__ void acc_flush(const GridDev& G, const NodeAcc& A, float* dne) {
  if (*A.key < 0) return;
  const long b0 = *A.base, sr = (long)G.n_t * G.n_p;
  const int dk = *A.dk1;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float x = A.v[q * kThreads];
    if (x != 0.f) atomicAdd(dne + b0 + (q >> 2) * sr + ((q >> 1) & 1) * G.n_p + (q & 1) * dk, x);
    A.v[q * kThreads] = 0.f;
  }
  *A.key = -1;
}

// Force adjoint at one RK4 stage: the force is a = kf grad n_e(p).  Given
// lam = dL/da, scatters kf lam . grad w_c to the n_e nodes (through the
// accumulator A when p lies in its cell; adopt: p is a node, whose cell the
// accumulator takes over) and returns kf H(p) lam (the position adjoint), H
// from dual numbers with the cell fixed.
__device__ __forceinline__ Vec force_adjoint(const GridDev& G, float kf, float x, float y, float z, const Vec& lam,
                                             float* dne, const NodeAcc& acc, bool adopt) {
  if (lam.x == 0.f && lam.y == 0.f && lam.z == 0.f) return {0.f, 0.f, 0.f};
  const CellGeom c = cell_geom(G, x, y, z);
  if (c.vac) return {0.f, 0.f, 0.f};
  const int cell = (c.i * (G.n_t - 1) + c.j) * G.n_p + c.k;
  if (adopt && cell != *acc.key) {
    acc_flush(G, acc, dne);
    *acc.key = cell;
    *acc.base = node_index(G, c, 0, 0, 0);
    *acc.dk1 = c.k1 - c.k;
  }
  const bool hit = cell == *acc.key;
  // node scatter
  const float gu = lam.x * c.du.x + lam.y * c.du.y + lam.z * c.du.z;
  const float gv = lam.x * c.dv.x + lam.y * c.dv.y + lam.z * c.dv.z;
  const float gw = lam.x * c.dw.x + lam.y * c.dw.y + lam.z * c.dw.z;
  const float wu[2] = {1.f - c.u, c.u}, wv[2] = {1.f - c.v, c.v}, ww[2] = {1.f - c.w, c.w};
  const float sg[2] = {-1.f, 1.f};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const float coef = sg[a] * wv[b] * ww[cc] * gu + wu[a] * sg[b] * ww[cc] * gv + wu[a] * wv[b] * sg[cc] * gw;
        // both branches as straight-line code: the shared add takes 0 on a
        // miss, the atomic is predicated (no divergence in the corner loop)
        const float val = kf * coef;
        acc.v[(a * 4 + b * 2 + cc) * kThreads] += hit ? val : 0.f;
        if (!hit) atomicAdd(dne + node_index(G, c, a, b, cc), val);
      }
  // Hessian-vector product: tangent of grad n_e along lam.  The tangents of
  // the fractions are lam . grad (u, v, w) = (gu, gv, gw); those of r, rho
  // follow from x . lam.
  const Dl X{x, lam.x}, Y{y, lam.y}, Z{z, lam.z};
  const float rho_d = (x * lam.x + y * lam.y) * c.inv_rho;
  const float r_d = fmaf(z, lam.z, x * lam.x + y * lam.y) * c.inv_r;
  const Dl inv_r{c.inv_r, -r_d * c.inv_r * c.inv_r};
  const Dl rho{c.rho, rho_d};
  const Dl inv_rho{c.inv_rho, -rho_d * c.inv_rho * c.inv_rho};
  const float2 rc = __ldg(G.r_cell + c.i);
  const float4 c0 = __ldg(G.ne + 2 * cell), c1 = __ldg(G.ne + 2 * cell + 1);
  const float d00 = c0.y - c0.x, d01 = c0.w - c0.z, d10 = c1.y - c1.x, d11 = c1.w - c1.z;
  const Dl W{c.w, gw};
  const Dl a00 = dl(c0.x) + d00 * W, a01 = dl(c0.z) + d01 * W;
  const Dl a10 = dl(c1.x) + d10 * W, a11 = dl(c1.z) + d11 * W;
  const Dl e0 = a01 - a00, e1 = a11 - a10;
  const Dl V{c.v, gv};
  const Dl b0 = a00 + V * e0, b1 = a10 + V * e1;
  const Dl U{c.u, gu};
  const Dl fu = b1 - b0;
  const Dl fv = e0 + U * (e1 - e0);
  const Dl g0 = dl(d00) + (d01 - d00) * V, g1 = dl(d10) + (d11 - d10) * V;
  const Dl fw = g0 + U * (g1 - g0);
  const Dl f_r = rc.y * fu;
  const Dl f_t = (G.t_inv * c.tsel) * fv;
  const Dl f_p = G.p_inv * fw;
  const Dl A = f_r * inv_r;
  const Dl ir2 = inv_r * inv_r;
  const Dl B = f_t * Z * ir2 * inv_rho;
  const Dl C = f_p * inv_rho * inv_rho;
  const Dl D = f_t * rho * ir2;
  const Dl gx = (A + B) * X - C * Y;
  const Dl gy = (A + B) * Y + C * X;
  const Dl gz = A * Z - D;
  return {kf * gx.d, kf * gy.d, kf * gz.d};
}

// Reverse of one RK4 step from (p, k) (rk4_central, or rk4_g3 for a
// neighbour's retrace), given the adjoints of its outputs: lr = dL/dr',
// lk = dL/dk' and lg on G = a1 + a2 + a3.  With r' = r + h k + h^2/6 G and
// k' = k + h/6 (a1 + 2 a2 + 2 a3 + a4), the stage points are
// P1 = p, P2 = p + h/2 k, P3 = p + h/2 k2, P4 = p + h k3 with
// k2 = k + h/2 a1, k3 = k + h/2 a2, and a_s = kf grad n_e(P_s).
// nst = 4 (central ray) or 3 (a neighbour: lr = lk = 0 and the fourth stage
// has no adjoint).  Adds dL/dp to lp and dL/dk to lko and scatters the n_e
// nodes.  The stages are reversed in one loop around a single force adjoint
// (the kernel's instruction footprint, not its arithmetic, bounds it).
__device__ __forceinline__ void rk4_reverse_any(const GridDev& G, float kf, float h, const Vec& p, const Vec& k,
                                                const Vec& lr, const Vec& lk, const Vec& lg, int nst, Vec& lp,
                                                Vec& lko, float* dne, const NodeAcc& A) {
  const float hh = 0.5f * h, h6 = h / 6.f, h3 = h / 3.f;
  // forward stage points (kept in registers: the stage loop selects among them)
  const Vec P2{fmaf(hh, k.x, p.x), fmaf(hh, k.y, p.y), fmaf(hh, k.z, p.z)};
  Vec P3, P4{0.f, 0.f, 0.f};
  {
    const Sample s1 = eval_field_t<false>(G, p.x, p.y, p.z, false);
    const Vec q{fmaf(hh, kf * s1.gx, k.x), fmaf(hh, kf * s1.gy, k.y), fmaf(hh, kf * s1.gz, k.z)};
    P3 = {fmaf(hh, q.x, p.x), fmaf(hh, q.y, p.y), fmaf(hh, q.z, p.z)};
  }
  if (nst == 4) {
    const Sample s2 = eval_field_t<false>(G, P2.x, P2.y, P2.z, false);
    const Vec q{fmaf(hh, kf * s2.gx, k.x), fmaf(hh, kf * s2.gy, k.y), fmaf(hh, kf * s2.gz, k.z)};
    P4 = {fmaf(h, q.x, p.x), fmaf(h, q.y, p.y), fmaf(h, q.z, p.z)};
  }
  // adjoints of the accelerations and velocities from the outputs
  // (k4 = k + h a3 enters r' only: its adjoint h/6 lr is applied at once)
  Vec La1{fmaf(h6, lk.x, lg.x), fmaf(h6, lk.y, lg.y), fmaf(h6, lk.z, lg.z)};
  Vec La2{fmaf(h3, lk.x, lg.x), fmaf(h3, lk.y, lg.y), fmaf(h3, lk.z, lg.z)};
  Vec La3{fmaf(h * h6, lr.x, La2.x), fmaf(h * h6, lr.y, La2.y), fmaf(h * h6, lr.z, La2.z)};
  const Vec La4{h6 * lk.x, h6 * lk.y, h6 * lk.z};
  Vec Lk2{h3 * lr.x, h3 * lr.y, h3 * lr.z}, Lk3 = Lk2;  // adjoints of k2, k3
  Vec Lp{lr.x, lr.y, lr.z};
  Vec Lk{lk.x + 2.f * h6 * lr.x, lk.y + 2.f * h6 * lr.y, lk.z + 2.f * h6 * lr.z};  // k itself and k4 = k + h a3
#pragma unroll 1
  for (int s = nst - 1; s >= 0; --s) {
    const Vec pt = (s == 3) ? P4 : (s == 2) ? P3 : (s == 1) ? P2 : p;
    const Vec la = (s == 3) ? La4 : (s == 2) ? La3 : (s == 1) ? La2 : La1;
    // the central ray's stage 1 is the node: the accumulator follows it
    const Vec LP = force_adjoint(G, kf, pt.x, pt.y, pt.z, la, dne, A, nst == 4 && s == 0);
    Lp = {Lp.x + LP.x, Lp.y + LP.y, Lp.z + LP.z};
    if (s == 3) {         // P4 = p + h k3, k3 = k + h/2 a2
      Lk3 = {fmaf(h, LP.x, Lk3.x), fmaf(h, LP.y, Lk3.y), fmaf(h, LP.z, Lk3.z)};
      Lk = {Lk.x + Lk3.x, Lk.y + Lk3.y, Lk.z + Lk3.z};
      La2 = {fmaf(hh, Lk3.x, La2.x), fmaf(hh, Lk3.y, La2.y), fmaf(hh, Lk3.z, La2.z)};
    } else if (s == 2) {  // P3 = p + h/2 k2, k2 = k + h/2 a1
      Lk2 = {fmaf(hh, LP.x, Lk2.x), fmaf(hh, LP.y, Lk2.y), fmaf(hh, LP.z, Lk2.z)};
      Lk = {Lk.x + Lk2.x, Lk.y + Lk2.y, Lk.z + Lk2.z};
      La1 = {fmaf(hh, Lk2.x, La1.x), fmaf(hh, Lk2.y, La1.y), fmaf(hh, Lk2.z, La1.z)};
    } else if (s == 1) {  // P2 = p + h/2 k
      Lk = {fmaf(hh, LP.x, Lk.x), fmaf(hh, LP.y, Lk.y), fmaf(hh, LP.z, Lk.z)};
    }
  }
  lp = {lp.x + Lp.x, lp.y + Lp.y, lp.z + Lp.z};
  lko = {lko.x + Lk.x, lko.y + Lk.y, lko.z + Lk.z};
}

// d kappa_vac / d n_e and d kappa_vac / d T_e (see kappa_vac).
__device__ __forceinline__ void kappa_partials(float ne, float te, float kap_c, float ln_f, float& dk_dne,
                                               float& dk_dte) {
  dk_dne = dk_dte = 0.f;
  if (!(ne > 0.f) || !(te > 0.f)) return;
  const float lnT = __logf(te);
  const bool hot = te > 2e5f;
  const float g = hot ? (24.5f + lnT - ln_f) : fmaf(1.5f, lnT, 18.2f - ln_f);
  const float rs = rsqrtf(te);
  const float base = (kap_c * ne) * (rs * rs * rs);  // kap_c n_e T^-1.5
  dk_dne = 2.f * base * g;
  dk_dte = base * ne * ((hot ? 1.f : 1.5f) - 1.5f * g) / te;
}

// ------------------------------------------------------------ the kernel
struct AdjParams {
  GridDev G;
  float h, h2_6, h_6, h2_12, hrsun, eta, eps_fixed, tbc_K;
  int tbc_mode, emission;
  ViewDev view;
  int nf;
  FreqDev freq[kMaxFreq];
  const RayDiag* diag;         // forward diagnostics (steps, status), output order
  const float* dL_dTb;         // [nf][npix], output order
  const Ckpt* ckpt;
  const unsigned long long* ck_off;  // ray t owns ckpt[ck_off[t] .. ck_off[t+1]); or, a tape:
  const int* ck_prev;                // the pool's links to each ray's previous checkpoint
  const int* ck_last;                // and each ray's last checkpoint
  float* dne;
  float* dte;
  unsigned int* counter;
  unsigned int total;
  unsigned long long* mismatch;  // rays whose step count does not match their checkpoint allocation
};

#ifndef RT_ADJ_MIN_BLOCKS
#define RT_ADJ_MIN_BLOCKS 3
#endif
// occupancy target (128-thread blocks): at 3 the kernel keeps its registers
// without spills and its resident step records take a quarter less of
// L1 and L2 than at 4
constexpr int kAdjMinBlocks = RT_ADJ_MIN_BLOCKS;

// One recomputed step of a segment (node m = m0 + j), in the thread's local
// memory (the reverse reads it back last to first).
struct StepRec {
  float r[3], k[3], dr[3];     // node state and the chord increment of step m
  float kap, te, ne, tau;      // node transfer values; optical depth at the node
  float lns_next, lnm;         // ln S at node m+1 and ln M^{m+1}
  float c1[3], c2[3];          // scaled separations of the +-e1, +-e2 pairs
};

// The adjoint of the forward (trace_rays), one thread per ray bundle.  Per
// ray, segment by segment from the last: recompute the segment's K central
// steps from its checkpoint with the forward's own step code (complete_step,
// retrace_step), then reverse it step by step: (A) the transfer of the
// segment and the tube area of the step (Eqs. 2, 9-12), (B) each
// neighbour's retrace (RK4 stages 1-3), (C) the central RK4 step with its
// chord, basis and eps (Eqs. 4-8).  Supported forms: step-wise with 4
// neighbours, or magnification off (NB = 0).
template <int NB, bool kMixed>
__global__ void __launch_bounds__(kThreads, kAdjMinBlocks) adjoint_rays(const __grid_constant__ AdjParams P) {
  static_assert(NB == 0 || NB == 4, "adjoint: 4 step-wise neighbours or none");
  constexpr int K = kCkptEvery;
  const int lane = threadIdx.x & 31;
  const float h = P.h;
  StepRec R[K + 1];
  __shared__ float acc_v[8 * kThreads];
  __shared__ int acc_key[kThreads], acc_dk1[kThreads];
  __shared__ long acc_base[kThreads];
  const NodeAcc A{acc_v + threadIdx.x, acc_key + threadIdx.x, acc_base + threadIdx.x, acc_dk1 + threadIdx.x};
#pragma unroll
  for (int q = 0; q < 8; ++q) A.v[q * kThreads] = 0.f;
  *A.key = -1;

  // per-ray state of the reverse sweep
  unsigned int item = 0;
  bool active = false, exhausted = false;
  int N = 0, status = 0, seg = 0;
  int slot = -1;  // tape: the pool slot of segment seg's checkpoint
  bool clipped = false;
  float kf = 0.f, kn2 = 0.f, kap_c = 0.f, ln_f = 0.f, lamT = 0.f, alpha = 1.f;
  float Wsuf = 0.f;                   // weight of everything beyond the node (sum of later terms)
  Vec Lr{0.f, 0.f, 0.f}, Lk{0.f, 0.f, 0.f};  // adjoints of the node state (r, k)
  float lkap = 0.f, lte = 0.f;        // partial adjoints of kappa and T_e at the node

  while (true) {
    // ---------------------------------------------------------- refill
    bool need = !active && !exhausted;
    unsigned needmask = __ballot_sync(kFull, need);
    while (needmask) {
      const int leader = __ffs(needmask) - 1;
      unsigned int first = 0;
      if (lane == leader) first = atomicAdd(P.counter, (unsigned)__popc(needmask));
      first = __shfl_sync(kFull, first, leader);
      if (need) {
        item = first + __popc(needmask & ((1u << lane) - 1u));
        if (item >= P.total) {
          exhausted = true;
          need = false;
        } else {
          const int fi = item / P.view.tickets;
          const int pix = item - fi * P.view.tickets;
          const FreqDev& F = P.freq[fi];
          const size_t o = (size_t)F.out_slab * P.view.npix + pix;
          const RayDiag d = P.diag[o];
          const float lw = P.dL_dTb[o];
          // the checkpoints were sized from a step count: it must be this ray's
          const unsigned long long n_ck =
              (d.steps > 0 && lw != 0.f) ? (unsigned long long)((d.steps - 1) / K + 1) : 0ull;
          // a tape's chain is checked segment by segment (the checkpoint's step)
          const bool fits = P.ck_prev ? true : P.ck_off[item + 1] - P.ck_off[item] == n_ck;
          if (!fits) atomicAdd(P.mismatch, 1ull);
          if (P.ck_prev) slot = P.ck_last[item];
          if (fits && d.steps > 0 && d.status >= kExitOuter && d.status <= kStepLimit && lw != 0.f) {
            N = d.steps;
            status = d.status;
            clipped = (d.status == kExitOuter || d.status == kHitInner);
            seg = (d.steps - 1) / K;
            kf = F.kf; kn2 = F.kn2; kap_c = F.kap_c; ln_f = F.ln_f;
            lamT = lw;
            alpha = 1.f;
            Wsuf = 0.f;
            Lr = {0.f, 0.f, 0.f};
            Lk = {0.f, 0.f, 0.f};
            lkap = lte = 0.f;
            active = true;
            need = false;
          }
        }
      }
      needmask = __ballot_sync(kFull, need);
    }
    if (!__any_sync(kFull, active)) break;
    if (!active) continue;

    // ---------------------------------------------- recompute the segment
    const int m0 = seg * K;
    const int n_s = min(K, N - m0);
    const bool last_seg = (m0 + n_s == N);
    float px, py, pz, kx, ky, kz, rlx, rly, rlz, klx, kly, klz, tau, lns;
    if (P.ck_prev && (slot < 0 || P.ckpt[slot].step != m0)) {
      // the tape does not hold this segment: the diagnostics belong to another forward
      atomicAdd(P.mismatch, 1ull);
      acc_flush(P.G, A, P.dne);
      active = false;
      continue;
    }
    {
      const Ckpt& c = P.ckpt[P.ck_prev ? (unsigned long long)slot : P.ck_off[item] + seg];
      px = c.r[0]; py = c.r[1]; pz = c.r[2];
      kx = c.k[0]; ky = c.k[1]; kz = c.k[2];
      rlx = c.rl[0]; rly = c.rl[1]; rlz = c.rl[2];
      klx = c.kl[0]; kly = c.kl[1]; klz = c.kl[2];
      tau = c.tau_hi + c.tau_lo;
      lns = c.lns_hi + c.lns_lo;
    }
    for (int j = 0; j < n_s; ++j) {
      const Rk4Out o = rk4_central(P.G, kf, h, px, py, pz, kx, ky, kz);
      const float kap = P.emission ? kappa_vac(o.ne1, o.te1, kap_c, ln_f) : 0.f;
      if (j > 0) tau += 0.5f * (R[j - 1].kap + kap) * P.hrsun;
      StepRec& rc = R[j];
      rc.r[0] = px; rc.r[1] = py; rc.r[2] = pz;
      rc.k[0] = kx; rc.k[1] = ky; rc.k[2] = kz;
      rc.kap = kap; rc.te = o.te1; rc.ne = o.ne1; rc.tau = tau;
      Vec dr, rn, kn;
      complete_step<kMixed>(h, P.h2_6, P.h_6, o, px, py, pz, kx, ky, kz, rlx, rly, rlz, klx, kly, klz, dr, rn, kn);
      rc.dr[0] = dr.x; rc.dr[1] = dr.y; rc.dr[2] = dr.z;
      if (NB > 0) {
        const Retrace T = retrace_step<(NB > 0 ? NB : 4)>(P.G, kf, h, P.h2_6, P.h2_12, P.eta, P.eps_fixed, px, py,
                                                          pz, kx, ky, kz, dr, Vec{o.Gx, o.Gy, o.Gz});
        rc.c1[0] = T.c1.x; rc.c1[1] = T.c1.y; rc.c1[2] = T.c1.z;
        rc.c2[0] = T.c2.x; rc.c2[1] = T.c2.y; rc.c2[2] = T.c2.z;
        rc.lnm = T.lm;
        lns += T.lm;
      } else {
        rc.lnm = 0.f;
      }
      rc.lns_next = lns;
      px = rn.x; py = rn.y; pz = rn.z;
      kx = kn.x; ky = kn.y; kz = kn.z;
    }
    // the closing node of the segment: node m0 + n_s (the crossing point on a clipped last step)
    {
      StepRec& rl = R[n_s];
      float qx = px, qy = py, qz = pz;
      if (last_seg && clipped) {
        const StepRec& rp = R[n_s - 1];
        const Vec rr{rp.r[0], rp.r[1], rp.r[2]}, dr{rp.dr[0], rp.dr[1], rp.dr[2]};
        const float a = (status == kHitInner) ? chord_crossing(rr, dr, P.G.r_min, false)
                                              : chord_crossing(rr, dr, P.G.r_max, true);
        alpha = a;
        qx = fmaf(a, dr.x, rr.x); qy = fmaf(a, dr.y, rr.y); qz = fmaf(a, dr.z, rr.z);
      }
      const Sample s = eval_field_t<true>(P.G, qx, qy, qz, true);
      const float kap = P.emission ? kappa_vac(s.ne, s.te, kap_c, ln_f) : 0.f;
      rl.r[0] = qx; rl.r[1] = qy; rl.r[2] = qz;
      rl.kap = kap; rl.te = s.te; rl.ne = s.ne;
      if (last_seg) {
        const float al = clipped ? alpha : 1.f;
        const float tauN = tau + 0.5f * (R[n_s - 1].kap + kap) * P.hrsun * al;
        rl.tau = tauN;
        const float sN = __expf(lns - tauN);
        float tbc = 0.f;
        if (status == kHitInner) tbc = (P.tbc_mode == 1) ? P.tbc_K : s.te;
        Wsuf = tbc * sN;  // the boundary term
        if (status == kHitInner && P.tbc_mode == 0) lte = lamT * sN;
      }
    }

    // ------------------------------------------------ reverse the segment
    // Step t (node m = m0 + t): (A) the transfer of segment m and the value
    // adjoints of node m + 1, (B) the neighbours' retraces of step m, (C) the
    // central step m.  After the first segment of the ray the loop takes one
    // more trip (t = -1) for node 0 alone.  Each heavy routine (the value
    // adjoint, the reverse RK4) has one call site.
    for (int t = n_s - 1; t >= (seg == 0 ? -1 : 0); --t) {
      const int tn = (t >= 0) ? t + 1 : 0;  // the node whose value adjoints are scattered
      // this step's two records, read once at the top of the trip
      const StepRec rn = R[tn];
      const StepRec rc = R[max(t, 0)];
      const bool last_step = last_seg && t == n_s - 1;
      const bool clip = last_step && clipped;
      float lam_ne = 0.f, lam_te = 0.f, lalpha = 0.f, lLnM = 0.f, lk_node = 0.f, lTbar = 0.f;
      float dkn, dkt;
      kappa_partials(rn.ne, rn.te, kap_c, ln_f, dkn, dkt);
      if (!P.emission) { dkn = 0.f; dkt = 0.f; }
      if (t >= 0) {
        // (A) transfer of segment m (Eq. 2 front to back, differentiated)
        const float al = clip ? alpha : 1.f;
        const float kap_sum = rc.kap + rn.kap;
        const float dt = 0.5f * kap_sum * P.hrsun * al;
        const float tbar = 0.5f * (rc.te + rn.te);
        const float qv = __expf(rc.lns_next - rc.tau);
        const float ed = __expf(-dt);
        const float om = one_minus_exp_neg(dt);
        const float W = tbar * om * qv;
        const float lDt = lamT * (tbar * ed * qv - Wsuf);
        lTbar = lamT * om * qv;
        lLnM = lamT * (W + Wsuf);
        Wsuf += W;
        lk_node = 0.5f * P.hrsun * al * lDt;
        const float lkap_n = lkap + lk_node;
        const float lte_n = lte + 0.5f * lTbar;
        lalpha = 0.5f * kap_sum * P.hrsun * lDt;
        lam_ne = lkap_n * dkn;
        lam_te = lte_n + lkap_n * dkt;
      } else {
        // node 0 on the outer sphere: its transfer values and k0 = n(r0) (-o)
        lam_ne = lkap * dkn;
        lam_te = lte + lkap * dkt;
        const Vec k0{rn.k[0], rn.k[1], rn.k[2]};
        const float n0 = sqrtf(dot3(k0, k0));
        if (n0 > 0.f) lam_ne += dot3(Lk, k0) / n0 * kn2 / (2.f * n0);
      }
      const Vec lpos = value_adjoint(P.G, rn.r[0], rn.r[1], rn.r[2], lam_ne, lam_te, P.dne, P.dte);
      if (t < 0) break;
      Vec lpc{0.f, 0.f, 0.f};
      if (clip) {
        lpc = lpos;   // the crossing point closes the path
      } else {
        Lr = {Lr.x + lpos.x, Lr.y + lpos.y, Lr.z + lpos.z};  // node m+1's full adjoint
      }
      lkap = lk_node;  // node m, completed by segment m - 1
      lte = 0.5f * lTbar;

      // tube area of step m (Eqs. 9-11, differentiated)
      const Vec dr{rc.dr[0], rc.dr[1], rc.dr[2]};
      Vec slp{0.f, 0.f, 0.f}, slk{0.f, 0.f, 0.f};   // sums of the seed adjoints
      Vec lt{0.f, 0.f, 0.f}, le1{0.f, 0.f, 0.f}, le2{0.f, 0.f, 0.f};
      float leps = 0.f;
      Vec t3{0.f, 0.f, 0.f}, e1{0.f, 0.f, 0.f}, e2{0.f, 0.f, 0.f}, lc1{0.f, 0.f, 0.f}, lc2{0.f, 0.f, 0.f};
      float eps = 0.f, sc = 0.f;
      if (NB > 0) {
        const float d2n = dot3(dr, dr);
        const float ids = rsqrtf(d2n);
        t3 = {dr.x * ids, dr.y * ids, dr.z * ids};
        basis(t3, e1, e2);
        eps = (P.eps_fixed > 0.f) ? P.eps_fixed : P.eta * (d2n * ids);
        const Vec c1{rc.c1[0], rc.c1[1], rc.c1[2]}, c2{rc.c2[0], rc.c2[1], rc.c2[2]};
        const float lm1 = lLnM * __expf(-rc.lnm);  // d ln(1 + m1) / d m1 = 1 / M
        const Vec c2xt{c2.y * t3.z - c2.z * t3.y, c2.z * t3.x - c2.x * t3.z, c2.x * t3.y - c2.y * t3.x};
        const Vec txc1{t3.y * c1.z - t3.z * c1.y, t3.z * c1.x - t3.x * c1.z, t3.x * c1.y - t3.y * c1.x};
        lc1 = {lm1 * (e1.x + c2xt.x), lm1 * (e1.y + c2xt.y), lm1 * (e1.z + c2xt.z)};
        lc2 = {lm1 * (e2.x + txc1.x), lm1 * (e2.y + txc1.y), lm1 * (e2.z + txc1.z)};
        le1 = {lm1 * c1.x, lm1 * c1.y, lm1 * c1.z};
        le2 = {lm1 * c2.x, lm1 * c2.y, lm1 * c2.z};
        lt = {lm1 * (c1.y * c2.z - c1.z * c2.y), lm1 * (c1.z * c2.x - c1.x * c2.z), lm1 * (c1.x * c2.y - c1.y * c2.x)};
        leps = -(dot3(c1, lc1) + dot3(c2, lc2)) / eps;
        sc = P.h2_12 / eps;
      }

      // (B) the neighbours' retraces (q < NB), then (C) the central step (q = NB)
      const Vec rr{rc.r[0], rc.r[1], rc.r[2]}, rk{rc.k[0], rc.k[1], rc.k[2]};
#pragma unroll 1
      for (int q = (NB > 0 ? 0 : NB); q <= NB; ++q) {
        Vec base = rr, lr_in{0.f, 0.f, 0.f}, lk_in{0.f, 0.f, 0.f}, lg{0.f, 0.f, 0.f};
        Vec lp_o{0.f, 0.f, 0.f}, lk_o{0.f, 0.f, 0.f};
        const bool first = q < 2;
        const float sgn = (q & 1) ? -1.f : 1.f;
        const Vec ev = first ? e1 : e2;
        if (q < NB) {
          // seed r_m +- eps e_j with k = k_m; its G enters D_j with the seed's sign
          const Vec lc = first ? lc1 : lc2;
          base = {rr.x + sgn * eps * ev.x, rr.y + sgn * eps * ev.y, rr.z + sgn * eps * ev.z};
          lg = {sgn * sc * lc.x, sgn * sc * lc.y, sgn * sc * lc.z};
        } else {
          Vec ldr{0.f, 0.f, 0.f};
          if (NB > 0) {
            // e2 = t x e1
            lt = {lt.x + (e1.y * le2.z - e1.z * le2.y), lt.y + (e1.z * le2.x - e1.x * le2.z),
                  lt.z + (e1.x * le2.y - e1.y * le2.x)};
            le1 = {le1.x + (le2.y * t3.z - le2.z * t3.y), le1.y + (le2.z * t3.x - le2.x * t3.z),
                   le1.z + (le2.x * t3.y - le2.y * t3.x)};
            // e1 = c / |c|, c = a x t
            const Vec av = (fabsf(t3.z) <= 0.9f) ? Vec{0.f, 0.f, 1.f} : Vec{0.f, 1.f, 0.f};
            const Vec cv{av.y * t3.z - av.z * t3.y, av.z * t3.x - av.x * t3.z, av.x * t3.y - av.y * t3.x};
            const float ic = rsqrtf(dot3(cv, cv));
            const float pe = dot3(e1, le1);
            const Vec lc{(le1.x - pe * e1.x) * ic, (le1.y - pe * e1.y) * ic, (le1.z - pe * e1.z) * ic};
            lt = {lt.x + (lc.y * av.z - lc.z * av.y), lt.y + (lc.z * av.x - lc.x * av.z),
                  lt.z + (lc.x * av.y - lc.y * av.x)};
            // eps = eta |dr| (Eq. 8); t = dr / |dr| (Eq. 5)
            const float ids = rsqrtf(dot3(dr, dr));
            const float lds = (P.eps_fixed > 0.f) ? 0.f : P.eta * leps;
            const float pt = dot3(t3, lt);
            ldr = {(lt.x - pt * t3.x) * ids + t3.x * lds, (lt.y - pt * t3.y) * ids + t3.y * lds,
                   (lt.z - pt * t3.z) * ids + t3.z * lds};
          }
          lp_o = slp;
          lk_o = slk;
          Vec lr_next = Lr;
          if (clip) {
            // crossing point pc = r_m + alpha dr with |pc| = R:
            // d alpha = -(pc . (d r_m + alpha d dr)) / (pc . dr)
            const Vec pc{rn.r[0], rn.r[1], rn.r[2]};
            const float den = dot3(pc, dr);
            const float la = lalpha + dot3(lpc, dr);
            const float g = (den != 0.f) ? la / den : 0.f;
            lp_o = {lp_o.x + lpc.x - g * pc.x, lp_o.y + lpc.y - g * pc.y, lp_o.z + lpc.z - g * pc.z};
            ldr = {ldr.x + alpha * (lpc.x - g * pc.x), ldr.y + alpha * (lpc.y - g * pc.y),
                   ldr.z + alpha * (lpc.z - g * pc.z)};
            lr_next = {0.f, 0.f, 0.f};  // the unclipped node is used only through the chord
          }
          // dr = r' - r_m
          lr_in = {lr_next.x + ldr.x, lr_next.y + ldr.y, lr_next.z + ldr.z};
          lp_o = {lp_o.x - ldr.x, lp_o.y - ldr.y, lp_o.z - ldr.z};
          lk_in = Lk;
        }
        rk4_reverse_any(P.G, kf, h, base, rk, lr_in, lk_in, lg, (q < NB) ? 3 : 4, lp_o, lk_o, P.dne, A);
        if (q < NB) {
          slp = {slp.x + lp_o.x, slp.y + lp_o.y, slp.z + lp_o.z};
          slk = {slk.x + lk_o.x, slk.y + lk_o.y, slk.z + lk_o.z};
          leps += sgn * dot3(ev, lp_o);
          if (first) le1 = {fmaf(sgn * eps, lp_o.x, le1.x), fmaf(sgn * eps, lp_o.y, le1.y), fmaf(sgn * eps, lp_o.z, le1.z)};
          else le2 = {fmaf(sgn * eps, lp_o.x, le2.x), fmaf(sgn * eps, lp_o.y, le2.y), fmaf(sgn * eps, lp_o.z, le2.z)};
        } else {
          Lr = lp_o;  // node m (its value adjoint joins in the next step back)
          Lk = lk_o;
        }
      }
    }

    // ------------------------------------------------ next segment / done
    if (seg == 0) {
      acc_flush(P.G, A, P.dne);
      active = false;
    } else {
      seg -= 1;
      if (P.ck_prev) slot = P.ck_prev[slot];
    }
  }
}

}  // namespace rt
