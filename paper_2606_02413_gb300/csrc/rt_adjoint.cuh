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
#include "rt_bundle.cuh"

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
  const float tt = (atan2_grid(rho, z) - G.t0) * G.t_inv;
  if (tt > 0.f && tt < G.t_last) {
    c.j = min(__float2int_rd(tt), G.n_t - 2);
    c.v = tt - (float)c.j;
    c.tsel = 1.f;
  } else if (tt <= 0.f) {
    c.j = 0; c.v = 0.f; c.tsel = 0.f;
  } else {
    c.j = G.n_t - 2; c.v = 1.f; c.tsel = 0.f;
  }
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

// Force adjoint at one RK4 stage: the force is a = kf grad n_e(p).  Given
// lam = dL/da, scatters kf lam . grad w_c to the n_e nodes and returns
// kf H(p) lam (the position adjoint), H from dual numbers with the cell fixed.
__device__ __forceinline__ Vec force_adjoint(const GridDev& G, float kf, float x, float y, float z, const Vec& lam,
                                             float* dne) {
  const CellGeom c = cell_geom(G, x, y, z);
  if (c.vac || (lam.x == 0.f && lam.y == 0.f && lam.z == 0.f)) return {0.f, 0.f, 0.f};
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
        atomicAdd(dne + node_index(G, c, a, b, cc), kf * coef);
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
  const int cell = (c.i * (G.n_t - 1) + c.j) * G.n_p + c.k;
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

// Reverse of one RK4 step from (p, k) (see rk4_step), given the adjoints of
// its outputs: lr = dL/dr', lk = dL/dk', and extra adjoints lg on
// G = a1 + a2 + a3 (the neighbours' separations enter only through G).
// Accumulates dL/dp and dL/dk into lp, lk_out and scatters the n_e nodes.
__device__ __forceinline__ void rk4_reverse(const GridDev& G, float kf, float h, const Vec& p, const Vec& k,
                                            const Vec& lr, const Vec& lk, const Vec& lg, Vec& lp, Vec& lk_out,
                                            float* dne) {
  const float hh = 0.5f * h;
  // forward stages
  const Sample s1 = eval_field(G, p.x, p.y, p.z, false);
  const Vec a1{kf * s1.gx, kf * s1.gy, kf * s1.gz};
  const Vec p2{fmaf(hh, k.x, p.x), fmaf(hh, k.y, p.y), fmaf(hh, k.z, p.z)};
  const Vec k2{fmaf(hh, a1.x, k.x), fmaf(hh, a1.y, k.y), fmaf(hh, a1.z, k.z)};
  const Sample s2 = eval_field(G, p2.x, p2.y, p2.z, false);
  const Vec a2{kf * s2.gx, kf * s2.gy, kf * s2.gz};
  const Vec p3{fmaf(hh, k2.x, p.x), fmaf(hh, k2.y, p.y), fmaf(hh, k2.z, p.z)};
  const Vec k3{fmaf(hh, a2.x, k.x), fmaf(hh, a2.y, k.y), fmaf(hh, a2.z, k.z)};
  const Vec p4{fmaf(h, k3.x, p.x), fmaf(h, k3.y, p.y), fmaf(h, k3.z, p.z)};
  // output adjoints: r' = r + h/6 (k + 2k2 + 2k3 + k4), k' = k + h/6 (a1 + 2a2 + 2a3 + a4)
  const float h6 = h / 6.f, h3 = h / 3.f;
  Vec Lp = lr;
  Vec Lk{lk.x + h6 * lr.x, lk.y + h6 * lr.y, lk.z + h6 * lr.z};
  Vec Lk2{h3 * lr.x, h3 * lr.y, h3 * lr.z};
  Vec Lk3 = Lk2;
  const Vec Lk4{h6 * lr.x, h6 * lr.y, h6 * lr.z};
  Vec La1{h6 * lk.x + lg.x, h6 * lk.y + lg.y, h6 * lk.z + lg.z};
  Vec La2{h3 * lk.x + lg.x, h3 * lk.y + lg.y, h3 * lk.z + lg.z};
  Vec La3{h3 * lk.x + lg.x, h3 * lk.y + lg.y, h3 * lk.z + lg.z};
  const Vec La4{h6 * lk.x, h6 * lk.y, h6 * lk.z};
  // stage 4: a4 = A(p4), p4 = p + h k3, k4 = k + h a3
  Vec Lp4 = force_adjoint(G, kf, p4.x, p4.y, p4.z, La4, dne);
  Lp = {Lp.x + Lp4.x, Lp.y + Lp4.y, Lp.z + Lp4.z};
  Lk3 = {fmaf(h, Lp4.x, Lk3.x), fmaf(h, Lp4.y, Lk3.y), fmaf(h, Lp4.z, Lk3.z)};
  Lk = {Lk.x + Lk4.x, Lk.y + Lk4.y, Lk.z + Lk4.z};
  La3 = {fmaf(h, Lk4.x, La3.x), fmaf(h, Lk4.y, La3.y), fmaf(h, Lk4.z, La3.z)};
  // stage 3: a3 = A(p3), p3 = p + hh k2, k3 = k + hh a2
  const Vec Lp3 = force_adjoint(G, kf, p3.x, p3.y, p3.z, La3, dne);
  Lp = {Lp.x + Lp3.x, Lp.y + Lp3.y, Lp.z + Lp3.z};
  Lk2 = {fmaf(hh, Lp3.x, Lk2.x), fmaf(hh, Lp3.y, Lk2.y), fmaf(hh, Lp3.z, Lk2.z)};
  Lk = {Lk.x + Lk3.x, Lk.y + Lk3.y, Lk.z + Lk3.z};
  La2 = {fmaf(hh, Lk3.x, La2.x), fmaf(hh, Lk3.y, La2.y), fmaf(hh, Lk3.z, La2.z)};
  // stage 2: a2 = A(p2), p2 = p + hh k, k2 = k + hh a1
  const Vec Lp2 = force_adjoint(G, kf, p2.x, p2.y, p2.z, La2, dne);
  Lp = {Lp.x + Lp2.x, Lp.y + Lp2.y, Lp.z + Lp2.z};
  Lk = {fmaf(hh, Lp2.x, Lk.x + Lk2.x), fmaf(hh, Lp2.y, Lk.y + Lk2.y), fmaf(hh, Lp2.z, Lk.z + Lk2.z)};
  La1 = {fmaf(hh, Lk2.x, La1.x), fmaf(hh, Lk2.y, La1.y), fmaf(hh, Lk2.z, La1.z)};
  // stage 1: a1 = A(p)
  const Vec Lp1 = force_adjoint(G, kf, p.x, p.y, p.z, La1, dne);
  lp = {lp.x + Lp.x + Lp1.x, lp.y + Lp.y + Lp1.y, lp.z + Lp.z + Lp1.z};
  lk_out = {lk_out.x + Lk.x, lk_out.y + Lk.y, lk_out.z + Lk.z};
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
// Per-step record of one recomputed segment (node m = m0 + j).
struct StepRec {
  float r[3], k[3], dr[3];     // node state and the chord increment of step m
  float kap, te, ne, tau;      // node transfer values; tau before segment m
  float lns_next, lnm;         // ln S at node m+1 and ln M^{m+1}
  float c1[3], c2[3];          // scaled tube separations of step m
  float t[3], e1[3], e2[3];    // chord direction and transverse basis of step m
  float eps;
  int axis;                    // basis reference: 0 z, 1 y
};

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
  const unsigned long long* ck_off;
  StepRec* rec;                // [slots][kCkptEvery + 1]
  float* dne;
  float* dte;
  unsigned int* counter;
  unsigned int total;
  unsigned long long* mismatch;  // rays whose step count does not match their checkpoint allocation
};

struct AdjState {
  int N, status, seg, clipped;
  float kf, kn2, kap_c, ln_f, lamT, alpha;
  float Wsuf;
  float lr[3], lk[3];          // adjoint of the node state at the end of the step being reversed
  float lkap, lte;             // partial adjoints of kappa and T_e at that node
  // per-step adjoints handed from the transfer/tube part (A) and the
  // neighbours (B) of step m to the central reverse (C) of the same step one
  // iteration later; double-buffered by the parity of m
  struct {
    float lt[3], le1[3], le2[3], leps, lalpha;  // chord, basis and eps adjoints
    float lpc[3];                                // the clip point (clipped last step)
    float slp[3], slk[3];                        // sum of the neighbour seed adjoints
  } st[2];
  float lpos[3];               // value adjoint of the node A just completed
};

#ifndef RT_ADJ_MIN_BLOCKS
#define RT_ADJ_MIN_BLOCKS 5
#endif
constexpr int kAdjMinBlocks = RT_ADJ_MIN_BLOCKS;  // occupancy target: 5 x 128 threads per SM

template <int NB>
__global__ void __launch_bounds__(kThreads, kAdjMinBlocks) adjoint_bundles(const __grid_constant__ AdjParams P) {
  constexpr int L = NB + 1;
  constexpr int BPW = 32 / L;
  constexpr int K = kCkptEvery;
  __shared__ AdjState S[kThreads / 32][BPW];
  const int lane = threadIdx.x & 31;
  const int q = lane % L;
  const bool used = (lane / L) < BPW;
  const int base = used ? lane - q : lane;
  const bool central = used && q == 0;
  const int bundle = used ? lane / L : 0;
  AdjState& A = S[threadIdx.x >> 5][bundle];
  const long slot = ((long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5)) * BPW + bundle;
  StepRec* R = P.rec + slot * (K + 1);
  const float h = P.h;
  bool active = false, exhausted = !central;
  unsigned int item = 0;

  while (true) {
    // ---------------------------------------------------------- refill
    bool need = central && !active && !exhausted;
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
          const float lamT = P.dL_dTb[o];
          // the checkpoints were sized from a step count: it must be this ray's
          const unsigned long long n_ck = (d.steps > 0) ? (unsigned long long)((d.steps - 1) / K + 1) : 0ull;
          const bool fits = P.ck_off[item + 1] - P.ck_off[item] == n_ck;
          if (!fits) atomicAdd(P.mismatch, 1ull);
          const bool has = fits && d.steps > 0 && d.status >= kExitOuter && d.status <= kStepLimit && lamT != 0.f;
          if (has) {
            A.N = d.steps;
            A.status = d.status;
            A.clipped = (d.status == kExitOuter || d.status == kHitInner) ? 1 : 0;
            A.seg = (d.steps - 1) / K;
            A.kf = F.kf; A.kn2 = F.kn2; A.kap_c = F.kap_c; A.ln_f = F.ln_f;
            A.lamT = lamT;
            A.alpha = 1.f;
            A.Wsuf = 0.f;
            A.lr[0] = A.lr[1] = A.lr[2] = A.lk[0] = A.lk[1] = A.lk[2] = 0.f;
            A.lkap = A.lte = 0.f;
            active = true;
            need = false;
          }
        }
      }
      needmask = __ballot_sync(kFull, need);
    }
    if (!__any_sync(kFull, active)) break;

    // ---------------------------------------------- recompute the segment
    // Pipelined as the forward: in iteration j the central lane steps node
    // m0 + j while its neighbours retrace step m0 + j - 1 from the seeds
    // broadcast one iteration earlier, all in one RK4 pass.
    const int m0 = active ? A.seg * K : 0;
    const int n_s = active ? min(K, A.N - m0) : 0;
    const bool last_seg = active && (m0 + n_s == A.N);
    const int ns_b = __shfl_sync(kFull, n_s, base);      // the bundle's segment length, on every lane
    const int ns_w = __reduce_max_sync(kFull, ns_b);     // the warp's longest
    float px = 0.f, py = 0.f, pz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
    float rlx = 0.f, rly = 0.f, rlz = 0.f, klx = 0.f, kly = 0.f, klz = 0.f;
    float tau = 0.f, lns = 0.f;
    bool has_seed = false;  // neighbour lanes: a retrace is pending
    if (central && active) {
      const Ckpt& c = P.ckpt[P.ck_off[item] + A.seg];
      px = c.r[0]; py = c.r[1]; pz = c.r[2];
      kx = c.k[0]; ky = c.k[1]; kz = c.k[2];
      rlx = c.rl[0]; rly = c.rl[1]; rlz = c.rl[2];
      klx = c.kl[0]; kly = c.kl[1]; klz = c.kl[2];
      tau = c.tau_hi + c.tau_lo;
      lns = c.lns_hi + c.lns_lo;
    }
    const float kf_lane = __shfl_sync(kFull, (central && active) ? A.kf : 0.f, base);
    for (int j = 0; j <= ns_w; ++j) {
      const bool cw = central && j < n_s;
      Rk4Out o;
      o.Gx = o.Gy = o.Gz = o.Ax = o.Ay = o.Az = 0.f;
      o.ne1 = o.te1 = 0.f;
      if (cw || (NB > 0 && has_seed)) o = rk4_step(P.G, kf_lane, h, px, py, pz, kx, ky, kz, cw);
      if (NB > 0) {
        // separations of the retraced step m0 + j - 1: D_j = G_{+j} - G_{-j}
        const float dx = o.Gx - __shfl_down_sync(kFull, o.Gx, 1);
        const float dy = o.Gy - __shfl_down_sync(kFull, o.Gy, 1);
        const float dz = o.Gz - __shfl_down_sync(kFull, o.Gz, 1);
        const Vec d1{__shfl_sync(kFull, dx, base + 1), __shfl_sync(kFull, dy, base + 1), __shfl_sync(kFull, dz, base + 1)};
        const Vec d2{__shfl_sync(kFull, dx, base + 3), __shfl_sync(kFull, dy, base + 3), __shfl_sync(kFull, dz, base + 3)};
        if (central && j >= 1 && j - 1 < n_s) {
          StepRec& rc = R[j - 1];
          const float sc = P.h2_12 / rc.eps;
          const Vec c1{sc * d1.x, sc * d1.y, sc * d1.z}, c2{sc * d2.x, sc * d2.y, sc * d2.z};
          const Vec tp{rc.t[0], rc.t[1], rc.t[2]}, e1p{rc.e1[0], rc.e1[1], rc.e1[2]}, e2p{rc.e2[0], rc.e2[1], rc.e2[2]};
          const float lm = ln_m(c1, c2, e1p, e2p, tp);
          rc.c1[0] = c1.x; rc.c1[1] = c1.y; rc.c1[2] = c1.z;
          rc.c2[0] = c2.x; rc.c2[1] = c2.y; rc.c2[2] = c2.z;
          rc.lnm = lm;
          lns += lm;
          rc.lns_next = lns;
        }
      } else if (central && j >= 1 && j - 1 < n_s) {
        R[j - 1].lnm = 0.f;
        R[j - 1].lns_next = lns;
      }
      Vec sr{0.f, 0.f, 0.f}, sk{0.f, 0.f, 0.f}, sa{0.f, 0.f, 0.f}, sb{0.f, 0.f, 0.f};
      if (cw) {
        const float kap = P.emission ? kappa_vac(o.ne1, o.te1, A.kap_c, A.ln_f) : 0.f;
        if (j > 0) tau += 0.5f * (R[j - 1].kap + kap) * P.hrsun;
        StepRec& rc = R[j];
        rc.r[0] = px; rc.r[1] = py; rc.r[2] = pz;
        rc.k[0] = kx; rc.k[1] = ky; rc.k[2] = kz;
        rc.kap = kap; rc.te = o.te1; rc.ne = o.ne1; rc.tau = tau;
        const Vec dr{fmaf(h, kx + klx, P.h2_6 * o.Gx), fmaf(h, ky + kly, P.h2_6 * o.Gy),
                     fmaf(h, kz + klz, P.h2_6 * o.Gz)};
        const Vec dk{P.h_6 * o.Ax, P.h_6 * o.Ay, P.h_6 * o.Az};
        rc.dr[0] = dr.x; rc.dr[1] = dr.y; rc.dr[2] = dr.z;
        const float d2n = dot3(dr, dr);
        const float ids = rsqrtf(d2n);
        const Vec tp{dr.x * ids, dr.y * ids, dr.z * ids};
        rc.t[0] = tp.x; rc.t[1] = tp.y; rc.t[2] = tp.z;
        if (NB > 0) {
          Vec e1p, e2p;
          basis(tp, e1p, e2p);
          const float eps = (P.eps_fixed > 0.f) ? P.eps_fixed : P.eta * (d2n * ids);
          rc.e1[0] = e1p.x; rc.e1[1] = e1p.y; rc.e1[2] = e1p.z;
          rc.e2[0] = e2p.x; rc.e2[1] = e2p.y; rc.e2[2] = e2p.z;
          rc.eps = eps;
          rc.axis = (fabsf(tp.z) <= 0.9f) ? 0 : 1;
          sr = {px, py, pz};
          sk = {kx, ky, kz};
          sa = {eps * e1p.x, eps * e1p.y, eps * e1p.z};
          sb = {eps * e2p.x, eps * e2p.y, eps * e2p.z};
        }
        float e;
        float nx, ny, nz;
        fast_two_sum(px, dr.x + rlx, nx, e); rlx = e;
        fast_two_sum(py, dr.y + rly, ny, e); rly = e;
        fast_two_sum(pz, dr.z + rlz, nz, e); rlz = e;
        px = nx; py = ny; pz = nz;
        float mx, my, mz;
        fast_two_sum(kx, dk.x + klx, mx, e); klx = e;
        fast_two_sum(ky, dk.y + kly, my, e); kly = e;
        fast_two_sum(kz, dk.z + klz, mz, e); klz = e;
        kx = mx; ky = my; kz = mz;
      }
      if (NB > 0) {
        // seeds of step m0 + j for the next iteration: +-eps e1 (roles 1, 2), +-eps e2 (3, 4)
        const bool e = __shfl_sync(kFull, cw ? 1 : 0, base) != 0;
        const float bx = __shfl_sync(kFull, sr.x, base), by = __shfl_sync(kFull, sr.y, base),
                    bz = __shfl_sync(kFull, sr.z, base);
        const float bkx = __shfl_sync(kFull, sk.x, base), bky = __shfl_sync(kFull, sk.y, base),
                    bkz = __shfl_sync(kFull, sk.z, base);
        const float ax = __shfl_sync(kFull, sa.x, base), ay = __shfl_sync(kFull, sa.y, base),
                    az = __shfl_sync(kFull, sa.z, base);
        const float cx = __shfl_sync(kFull, sb.x, base), cy = __shfl_sync(kFull, sb.y, base),
                    cz = __shfl_sync(kFull, sb.z, base);
        if (used && q > 0) {
          has_seed = e;
          const float sgn = (q & 1) ? 1.f : -1.f;
          px = bx + sgn * ((q <= 2) ? ax : cx);
          py = by + sgn * ((q <= 2) ? ay : cy);
          pz = bz + sgn * ((q <= 2) ? az : cz);
          kx = bkx; ky = bky; kz = bkz;
        }
      }
    }
    // the closing node of the segment: node m0 + n_s (the clip point on a clipped final step)
    if (central && active) {
      StepRec& rl = R[n_s];
      float qx = px, qy = py, qz = pz;
      if (last_seg && A.clipped) {
        const StepRec& rp = R[n_s - 1];
        const Vec rr{rp.r[0], rp.r[1], rp.r[2]}, dr{rp.dr[0], rp.dr[1], rp.dr[2]};
        const float a = (A.status == kHitInner) ? chord_crossing(rr, dr, P.G.r_min, false)
                                                 : chord_crossing(rr, dr, P.G.r_max, true);
        A.alpha = a;
        qx = fmaf(a, dr.x, rr.x); qy = fmaf(a, dr.y, rr.y); qz = fmaf(a, dr.z, rr.z);
      }
      const Sample s = eval_field(P.G, qx, qy, qz, true);
      const float kap = P.emission ? kappa_vac(s.ne, s.te, A.kap_c, A.ln_f) : 0.f;
      rl.r[0] = qx; rl.r[1] = qy; rl.r[2] = qz;
      rl.kap = kap; rl.te = s.te; rl.ne = s.ne;
      if (last_seg) {
        const float alpha = A.clipped ? A.alpha : 1.f;
        const float tauN = tau + 0.5f * (R[n_s - 1].kap + kap) * P.hrsun * alpha;
        rl.tau = tauN;
        const float sN = __expf(lns - tauN);
        float tbc = 0.f;
        if (A.status == kHitInner) tbc = (P.tbc_mode == 1) ? P.tbc_K : s.te;
        A.Wsuf = tbc * sN;  // the boundary term
        if (A.status == kHitInner && P.tbc_mode == 0) A.lte = A.lamT * sN;
      }
    }

    // ------------------------------------------------ reverse the segment
    // Pipelined: in iteration t the central lane runs the transfer and
    // tube-area adjoint of step m0 + t (A) and the reverse of its own RK4
    // step m0 + t + 1 (C), while its neighbours reverse their retrace of step
    // m0 + t (B); B and C share one rk4_reverse pass.  C of step t + 1 needs
    // A and B of step t + 1, which the previous iteration left in the
    // bundle's shared state.
    for (int t = ns_w - 1; t >= -1; --t) {
      const bool a_ok = central && t >= 0 && t < n_s;
      const bool c_ok = central && t + 1 < n_s;
      const bool b_ok = NB > 0 && used && q > 0 && t >= 0 && t < ns_b;
      // A: transfer of segment m = m0 + t (Eq. 2 front to back, differentiated)
      float lD1x = 0.f, lD1y = 0.f, lD1z = 0.f, lD2x = 0.f, lD2y = 0.f, lD2z = 0.f;
      if (a_ok) {
        auto& S = A.st[t & 1];
        const bool last_step = last_seg && t == n_s - 1;
        const StepRec& rc = R[t];
        const StepRec& rn = R[t + 1];
        const float alpha = (last_step && A.clipped) ? A.alpha : 1.f;
        const float kap_sum = rc.kap + rn.kap;
        const float dt = 0.5f * kap_sum * P.hrsun * alpha;
        const float tbar = 0.5f * (rc.te + rn.te);
        const float qv = __expf(rc.lns_next - rc.tau);
        const float ed = __expf(-dt);
        const float om = one_minus_exp_neg(dt);
        const float W = tbar * om * qv;
        const float lDt = A.lamT * (tbar * ed * qv - A.Wsuf);
        const float lTbar = A.lamT * om * qv;
        const float lLnM = A.lamT * (W + A.Wsuf);
        A.Wsuf += W;
        const float lk_node = 0.5f * P.hrsun * alpha * lDt;
        const float lkap_n = A.lkap + lk_node;
        const float lte_n = A.lte + 0.5f * lTbar;
        S.lalpha = 0.5f * kap_sum * P.hrsun * lDt;
        // node m+1 is complete: scatter its value adjoints
        float dkn, dkt;
        kappa_partials(rn.ne, rn.te, A.kap_c, A.ln_f, dkn, dkt);
        if (!P.emission) { dkn = 0.f; dkt = 0.f; }
        const Vec lpos = value_adjoint(P.G, rn.r[0], rn.r[1], rn.r[2], lkap_n * dkn, lte_n + lkap_n * dkt,
                                       P.dne, P.dte);
        if (last_step && A.clipped) {
          S.lpc[0] = lpos.x; S.lpc[1] = lpos.y; S.lpc[2] = lpos.z;
          A.lpos[0] = A.lpos[1] = A.lpos[2] = 0.f;
        } else {
          A.lpos[0] = lpos.x; A.lpos[1] = lpos.y; A.lpos[2] = lpos.z;
        }
        A.lkap = lk_node;  // node m, completed by segment m - 1
        A.lte = 0.5f * lTbar;
        // tube area of step m (Eqs. 9-11, differentiated); the neighbour
        // seeds add their parts after B
        S.lt[0] = S.lt[1] = S.lt[2] = 0.f;
        S.le1[0] = S.le1[1] = S.le1[2] = 0.f;
        S.le2[0] = S.le2[1] = S.le2[2] = 0.f;
        S.leps = 0.f;
        S.slp[0] = S.slp[1] = S.slp[2] = S.slk[0] = S.slk[1] = S.slk[2] = 0.f;
        if (NB > 0) {
          const Vec c1{rc.c1[0], rc.c1[1], rc.c1[2]}, c2{rc.c2[0], rc.c2[1], rc.c2[2]};
          const Vec t3{rc.t[0], rc.t[1], rc.t[2]}, e1{rc.e1[0], rc.e1[1], rc.e1[2]}, e2{rc.e2[0], rc.e2[1], rc.e2[2]};
          const float lm1 = lLnM * __expf(-rc.lnm);  // d ln(1 + m1) / d m1 = 1 / M
          const Vec c2xt{c2.y * t3.z - c2.z * t3.y, c2.z * t3.x - c2.x * t3.z, c2.x * t3.y - c2.y * t3.x};
          const Vec txc1{t3.y * c1.z - t3.z * c1.y, t3.z * c1.x - t3.x * c1.z, t3.x * c1.y - t3.y * c1.x};
          const Vec lc1{lm1 * (e1.x + c2xt.x), lm1 * (e1.y + c2xt.y), lm1 * (e1.z + c2xt.z)};
          const Vec lc2{lm1 * (e2.x + txc1.x), lm1 * (e2.y + txc1.y), lm1 * (e2.z + txc1.z)};
          S.le1[0] = lm1 * c1.x; S.le1[1] = lm1 * c1.y; S.le1[2] = lm1 * c1.z;
          S.le2[0] = lm1 * c2.x; S.le2[1] = lm1 * c2.y; S.le2[2] = lm1 * c2.z;
          S.lt[0] = lm1 * (c1.y * c2.z - c1.z * c2.y);
          S.lt[1] = lm1 * (c1.z * c2.x - c1.x * c2.z);
          S.lt[2] = lm1 * (c1.x * c2.y - c1.y * c2.x);
          S.leps = -(dot3(c1, lc1) + dot3(c2, lc2)) / rc.eps;
          const float sc = P.h2_12 / rc.eps;
          lD1x = sc * lc1.x; lD1y = sc * lc1.y; lD1z = sc * lc1.z;
          lD2x = sc * lc2.x; lD2y = sc * lc2.y; lD2z = sc * lc2.z;
        }
      } else if (central) {
        A.lpos[0] = A.lpos[1] = A.lpos[2] = 0.f;
      }
      // B and C in one rk4_reverse pass: the neighbours reverse their
      // retrace of step t (G enters the separations only), the central lane
      // its own step t + 1
      Vec rp{0.f, 0.f, 0.f}, rk{0.f, 0.f, 0.f}, lr_in{0.f, 0.f, 0.f}, lk_in{0.f, 0.f, 0.f}, lg{0.f, 0.f, 0.f};
      Vec lp_o{0.f, 0.f, 0.f}, lk_o{0.f, 0.f, 0.f};
      if (NB > 0) {
        const float g1x = __shfl_sync(kFull, lD1x, base), g1y = __shfl_sync(kFull, lD1y, base),
                    g1z = __shfl_sync(kFull, lD1z, base);
        const float g2x = __shfl_sync(kFull, lD2x, base), g2y = __shfl_sync(kFull, lD2y, base),
                    g2z = __shfl_sync(kFull, lD2z, base);
        if (b_ok) {
          const StepRec& rc = R[t];
          const float sgn = (q & 1) ? 1.f : -1.f;
          const bool first = q <= 2;
          const float* ev = first ? rc.e1 : rc.e2;
          rp = {rc.r[0] + sgn * rc.eps * ev[0], rc.r[1] + sgn * rc.eps * ev[1], rc.r[2] + sgn * rc.eps * ev[2]};
          rk = {rc.k[0], rc.k[1], rc.k[2]};
          lg = first ? Vec{sgn * g1x, sgn * g1y, sgn * g1z} : Vec{sgn * g2x, sgn * g2y, sgn * g2z};
        }
      }
      if (c_ok) {
        // C's inputs: the output adjoints of central step t + 1 and its seed/chord terms
        const auto& S = A.st[(t + 1) & 1];
        const bool last_step = last_seg && t + 1 == n_s - 1;
        const StepRec& rc = R[t + 1];
        Vec ldr{0.f, 0.f, 0.f};
        if (NB > 0) {
          const Vec e1{rc.e1[0], rc.e1[1], rc.e1[2]}, t3{rc.t[0], rc.t[1], rc.t[2]};
          lp_o = {S.slp[0], S.slp[1], S.slp[2]};
          lk_o = {S.slk[0], S.slk[1], S.slk[2]};
          Vec le1{S.le1[0], S.le1[1], S.le1[2]}, lt{S.lt[0], S.lt[1], S.lt[2]};
          const Vec le2{S.le2[0], S.le2[1], S.le2[2]};
          // e2 = t x e1
          lt = {lt.x + (e1.y * le2.z - e1.z * le2.y), lt.y + (e1.z * le2.x - e1.x * le2.z),
                lt.z + (e1.x * le2.y - e1.y * le2.x)};
          le1 = {le1.x + (le2.y * t3.z - le2.z * t3.y), le1.y + (le2.z * t3.x - le2.x * t3.z),
                 le1.z + (le2.x * t3.y - le2.y * t3.x)};
          // e1 = c / |c|, c = a x t
          const Vec av = (rc.axis == 0) ? Vec{0.f, 0.f, 1.f} : Vec{0.f, 1.f, 0.f};
          const Vec cv{av.y * t3.z - av.z * t3.y, av.z * t3.x - av.x * t3.z, av.x * t3.y - av.y * t3.x};
          const float ic = rsqrtf(dot3(cv, cv));
          const float pe = dot3(e1, le1);
          const Vec lc{(le1.x - pe * e1.x) * ic, (le1.y - pe * e1.y) * ic, (le1.z - pe * e1.z) * ic};
          lt = {lt.x + (lc.y * av.z - lc.z * av.y), lt.y + (lc.z * av.x - lc.x * av.z),
                lt.z + (lc.x * av.y - lc.y * av.x)};
          // eps = eta |dr| (Eq. 8); t = dr / |dr| (Eq. 5)
          const Vec dr{rc.dr[0], rc.dr[1], rc.dr[2]};
          const float ids = rsqrtf(dot3(dr, dr));
          const float lds = (P.eps_fixed > 0.f) ? 0.f : P.eta * S.leps;
          const float pt = dot3(t3, lt);
          ldr = {(lt.x - pt * t3.x) * ids + t3.x * lds, (lt.y - pt * t3.y) * ids + t3.y * lds,
                 (lt.z - pt * t3.z) * ids + t3.z * lds};
        }
        Vec lr_next{A.lr[0], A.lr[1], A.lr[2]};
        if (last_step && A.clipped) {
          // clip point pc = r_m + alpha dr with |pc| = R: d alpha = -(pc . (d r_m + alpha d dr)) / (pc . dr)
          const StepRec& rn = R[t + 2];
          const Vec pc{rn.r[0], rn.r[1], rn.r[2]}, dr{rc.dr[0], rc.dr[1], rc.dr[2]};
          const Vec lpc{S.lpc[0], S.lpc[1], S.lpc[2]};
          const float den = dot3(pc, dr);
          const float la = S.lalpha + dot3(lpc, dr);
          const float g = (den != 0.f) ? la / den : 0.f;
          lp_o = {lp_o.x + lpc.x - g * pc.x, lp_o.y + lpc.y - g * pc.y, lp_o.z + lpc.z - g * pc.z};
          ldr = {ldr.x + A.alpha * (lpc.x - g * pc.x), ldr.y + A.alpha * (lpc.y - g * pc.y),
                 ldr.z + A.alpha * (lpc.z - g * pc.z)};
          lr_next = {0.f, 0.f, 0.f};  // the unclipped node is used only through the chord
        }
        // dr = r' - r_m
        lr_in = {lr_next.x + ldr.x, lr_next.y + ldr.y, lr_next.z + ldr.z};
        lp_o = {lp_o.x - ldr.x, lp_o.y - ldr.y, lp_o.z - ldr.z};
        lk_in = {A.lk[0], A.lk[1], A.lk[2]};
        rp = {rc.r[0], rc.r[1], rc.r[2]};
        rk = {rc.k[0], rc.k[1], rc.k[2]};
      }
      if (c_ok || b_ok) rk4_reverse(P.G, kf_lane, h, rp, rk, lr_in, lk_in, lg, lp_o, lk_o, P.dne);
      // gather the neighbours' seed adjoints of step t to the central lane
      if (NB > 0) {
        Vec lps[4], lks[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const int src = base + 1 + n;
          lps[n] = {__shfl_sync(kFull, lp_o.x, src), __shfl_sync(kFull, lp_o.y, src), __shfl_sync(kFull, lp_o.z, src)};
          lks[n] = {__shfl_sync(kFull, lk_o.x, src), __shfl_sync(kFull, lk_o.y, src), __shfl_sync(kFull, lk_o.z, src)};
        }
        if (a_ok) {
          // seeds r_m +- eps e_j with k = k_m: node, eps and basis adjoints of step t
          auto& S = A.st[t & 1];
          const StepRec& rc = R[t];
          const Vec e1{rc.e1[0], rc.e1[1], rc.e1[2]}, e2{rc.e2[0], rc.e2[1], rc.e2[2]};
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            S.slp[0] += lps[n].x; S.slp[1] += lps[n].y; S.slp[2] += lps[n].z;
            S.slk[0] += lks[n].x; S.slk[1] += lks[n].y; S.slk[2] += lks[n].z;
          }
          S.leps += dot3(e1, lps[0]) - dot3(e1, lps[1]) + dot3(e2, lps[2]) - dot3(e2, lps[3]);
          S.le1[0] += rc.eps * (lps[0].x - lps[1].x);
          S.le1[1] += rc.eps * (lps[0].y - lps[1].y);
          S.le1[2] += rc.eps * (lps[0].z - lps[1].z);
          S.le2[0] += rc.eps * (lps[2].x - lps[3].x);
          S.le2[1] += rc.eps * (lps[2].y - lps[3].y);
          S.le2[2] += rc.eps * (lps[2].z - lps[3].z);
        }
      }
      // the adjoints at node m0 + t + 1: C's output plus A's value term
      if (c_ok) {
        A.lr[0] = lp_o.x + A.lpos[0]; A.lr[1] = lp_o.y + A.lpos[1]; A.lr[2] = lp_o.z + A.lpos[2];
        A.lk[0] = lk_o.x; A.lk[1] = lk_o.y; A.lk[2] = lk_o.z;
      } else if (a_ok) {
        A.lr[0] += A.lpos[0]; A.lr[1] += A.lpos[1]; A.lr[2] += A.lpos[2];
      }
    }

    // ------------------------------------------------ next segment / launch
    if (central && active) {
      if (A.seg == 0) {
        // node 0 on the outer sphere: its transfer values and k0 = n(r0) (-o)
        const StepRec& r0 = R[0];
        float dkn, dkt;
        kappa_partials(r0.ne, r0.te, A.kap_c, A.ln_f, dkn, dkt);
        if (!P.emission) { dkn = 0.f; dkt = 0.f; }
        float lam_ne = A.lkap * dkn;
        const float lam_te = A.lte + A.lkap * dkt;
        const Vec k0{r0.k[0], r0.k[1], r0.k[2]};
        const float n0 = sqrtf(dot3(k0, k0));
        if (n0 > 0.f) {
          const float ln0 = (A.lk[0] * k0.x + A.lk[1] * k0.y + A.lk[2] * k0.z) / n0;
          lam_ne += ln0 * A.kn2 / (2.f * n0);
        }
        value_adjoint(P.G, r0.r[0], r0.r[1], r0.r[2], lam_ne, lam_te, P.dne, P.dte);
        active = false;
      } else {
        A.seg -= 1;
      }
    }
  }
}

}  // namespace rt

