// The persistent one-thread-per-bundle ray kernel (step-wise magnification
// with 0, 2, 4 or 8 neighbours; Sec. 2.1 Eqs. 4-12, Sec. 3.2).
//
// Each thread owns one ray bundle at a time: the central ray of a (pixel,
// frequency) and its NB step-wise neighbours.  Per central step i it
//   (a) advances the central ray one RK4 step from node i (Eq. 4), with the
//       stage-1 sample giving n_e and T_e at node i;
//   (b) settles the transfer of segment i-1 -> i (Eq. 2 with Eq. 12, front to
//       back) and the TAU_STOP / STEP_LIMIT terminations;
//   (c) completes step i: chord t^i, transverse basis and eps (Eqs. 5, 6, 8),
//       the new node, and the clip tests against the inner and outer spheres;
//   (d) retraces step i for every neighbour seeded at r^i +- eps e_j with the
//       central k^i (Eq. 7) and accumulates ln M^{i+1} (Eqs. 9-11);
//   (e) on a clipped last step, closes the path at the crossing point.
// This is the order of the paper's per-step description; the lane-parallel
// bundle kernel (rt_bundle.cuh) computes the same quantities with the
// neighbours one step behind the central lane.
//
// Why one thread per bundle.  The per-step bookkeeping (basis, ln M,
// absorption, transfer, termination, compensated updates) is scalar per
// bundle; with the bundle spread over NB + 1 lanes it ran on one lane of
// NB + 1 and took a third of the warp's issue slots.  Here every lane of a
// warp does useful work in every instruction, and a neighbour needs only the
// first three RK4 stages (its separation depends on its end position, which
// does not involve the fourth stage), so a step costs 4 + 3 NB field
// evaluations instead of 4 (NB + 1).
//
// Precision (kMixed) and the offset form of the separations are those of
// rt_bundle.cuh: d_j = eps e_j + h^2/12 (G_{+j} - G_{-j}) for a +-e_j pair,
// ln M = log1p(c1.e1 + c2.e2 + t.(c1 x c2)) with c_j = (d_j - eps e_j) / eps.
#pragma once
#include "rt_bundle.cuh"

namespace rt {

// __launch_bounds__ occupancy target (128-thread blocks).  At 4 blocks (16
// warps per SM, up to 128 registers) the step keeps its values in registers
// instead of recomputing or spilling them; the kernel is bound by issue, not
// latency, and 4 measured faster than 6, 5, 3 or 2.
#ifndef RT_RAY_MIN_BLOCKS
#define RT_RAY_MIN_BLOCKS 4
#endif
constexpr int kRayMinBlocks = RT_RAY_MIN_BLOCKS;

// The sum G = a1 + a2 + a3 of the first three RK4 stages from (p, k): a
// neighbour's end position is p + h k + h^2/6 G (the fourth stage enters only
// the wave vector).  The arithmetic is that of rk4_step's G.
__device__ __forceinline__ Vec rk4_g3(const GridDev& G, float kf, float h, float px, float py, float pz, float kx,
                                      float ky, float kz) {
  const float hh = 0.5f * h;
  // stages 1 and 2 are independent (stage 2 sits at p + h/2 k)
  Sample s1 = eval_field_t<false>(G, px, py, pz, false);
  Sample s2 = eval_field_t<false>(G, fmaf(hh, kx, px), fmaf(hh, ky, py), fmaf(hh, kz, pz), false);
  const float a1x = kf * s1.gx, a1y = kf * s1.gy, a1z = kf * s1.gz;
  const float a2x = kf * s2.gx, a2y = kf * s2.gy, a2z = kf * s2.gz;
  Vec g{a1x, a1y, a1z};
  g.x += a2x; g.y += a2y; g.z += a2z;
  // stage 3 at p + h/2 (k + h/2 a1)
  const float qx = fmaf(hh, a1x, kx), qy = fmaf(hh, a1y, ky), qz = fmaf(hh, a1z, kz);
  const Sample s3 = eval_field_t<false>(G, fmaf(hh, qx, px), fmaf(hh, qy, py), fmaf(hh, qz, pz), false);
  g.x += kf * s3.gx; g.y += kf * s3.gy; g.z += kf * s3.gz;
  return g;
}

// One central RK4 step (see rk4_step) with the stage-1 sample including T_e;
// stages 1 and 2, and then 3 and 4, are independent of each other.
__device__ __forceinline__ Rk4Out rk4_central(const GridDev& G, float kf, float h, float px, float py, float pz,
                                              float kx, float ky, float kz) {
  Rk4Out o;
  const float hh = 0.5f * h;
  const Sample s1 = eval_field_t<true>(G, px, py, pz, true);
  const Sample s2 = eval_field_t<false>(G, fmaf(hh, kx, px), fmaf(hh, ky, py), fmaf(hh, kz, pz), false);
  o.ne1 = s1.ne;
  o.te1 = s1.te;
  const float a1x = kf * s1.gx, a1y = kf * s1.gy, a1z = kf * s1.gz;
  const float a2x = kf * s2.gx, a2y = kf * s2.gy, a2z = kf * s2.gz;
  o.Gx = a1x; o.Gy = a1y; o.Gz = a1z;
  o.Ax = a1x; o.Ay = a1y; o.Az = a1z;
  o.Gx += a2x; o.Gy += a2y; o.Gz += a2z;
  o.Ax = fmaf(2.f, a2x, o.Ax); o.Ay = fmaf(2.f, a2y, o.Ay); o.Az = fmaf(2.f, a2z, o.Az);
  // stage 3 at p + h/2 (k + h/2 a1), stage 4 at p + h (k + h/2 a2)
  const float qx = fmaf(hh, a1x, kx), qy = fmaf(hh, a1y, ky), qz = fmaf(hh, a1z, kz);
  const float q3x = fmaf(hh, a2x, kx), q3y = fmaf(hh, a2y, ky), q3z = fmaf(hh, a2z, kz);
  const Sample s3 = eval_field_t<false>(G, fmaf(hh, qx, px), fmaf(hh, qy, py), fmaf(hh, qz, pz), false);
  const Sample s4 = eval_field_t<false>(G, fmaf(h, q3x, px), fmaf(h, q3y, py), fmaf(h, q3z, pz), false);
  const float a3x = kf * s3.gx, a3y = kf * s3.gy, a3z = kf * s3.gz;
  o.Gx += a3x; o.Gy += a3y; o.Gz += a3z;
  o.Ax = fmaf(2.f, a3x, o.Ax); o.Ay = fmaf(2.f, a3y, o.Ay); o.Az = fmaf(2.f, a3z, o.Az);
  o.Ax = fmaf(kf, s4.gx, o.Ax); o.Ay = fmaf(kf, s4.gy, o.Ay); o.Az = fmaf(kf, s4.gz, o.Az);
  return o;
}

// "+" seed offset of neighbour pair j from the node: eps e1, eps e2, and (8
// neighbours) eps (e1 + e2)/sqrt2, eps (e2 - e1)/sqrt2; the "-" member of the
// pair sits at minus that offset.  a = eps e1, b = eps e2.
__device__ __forceinline__ Vec pair_offset(int j, const Vec& a, const Vec& b) {
  const float s2 = 0.70710678118654752f;
  if (j == 0) return a;
  if (j == 1) return b;
  if (j == 2) return {s2 * (a.x + b.x), s2 * (a.y + b.y), s2 * (a.z + b.z)};
  return {s2 * (b.x - a.x), s2 * (b.y - a.y), s2 * (b.z - a.z)};
}

// Completes a central RK4 step from node (p, k) (Eq. 4 in increment form):
// the chord dr = h (k + kl) + h^2/6 G, dk = h/6 A, and the next node
// (rn, kn).  kMixed carries the rounding of both updates in (rl, kl)
// (Fast2Sum); the plain form leaves them at zero.  The forward kernel and the
// adjoint's recomputation share it, so both follow the same path.
template <bool kMixed>
__device__ __forceinline__ void complete_step(float h, float h2_6, float h_6, const Rk4Out& o, float px, float py,
                                              float pz, float kx, float ky, float kz, float& rlx, float& rly,
                                              float& rlz, float& klx, float& kly, float& klz, Vec& dr, Vec& rn,
                                              Vec& kn) {
  dr = {fmaf(h, kx + klx, h2_6 * o.Gx), fmaf(h, ky + kly, h2_6 * o.Gy), fmaf(h, kz + klz, h2_6 * o.Gz)};
  const Vec dk{h_6 * o.Ax, h_6 * o.Ay, h_6 * o.Az};
  if (kMixed) {
    fast_two_sum(px, dr.x + rlx, rn.x, rlx);
    fast_two_sum(py, dr.y + rly, rn.y, rly);
    fast_two_sum(pz, dr.z + rlz, rn.z, rlz);
    fast_two_sum(kx, dk.x + klx, kn.x, klx);
    fast_two_sum(ky, dk.y + kly, kn.y, kly);
    fast_two_sum(kz, dk.z + klz, kn.z, klz);
  } else {
    rn = {px + dr.x, py + dr.y, pz + dr.z};
    kn = {kx + dk.x, ky + dk.y, kz + dk.z};
  }
}

// The step-wise retrace of one central step (Eqs. 5-11): chord direction t,
// transverse basis (e1, e2), eps, the scaled separations c1, c2 of the
// +-e1, +-e2 pairs (2 neighbours: one-sided against the central G0), and
// ln M.  With 8 neighbours the 45-degree pairs give a second estimate and M
// is the mean of the two.
struct Retrace {
  Vec t, e1, e2, c1, c2;
  float eps, lm;
};

template <int NB>
__device__ __forceinline__ Retrace retrace_step(const GridDev& G, float kf, float h, float h2_6, float h2_12,
                                                float eta, float eps_fixed, float px, float py, float pz, float kx,
                                                float ky, float kz, const Vec& dr, const Vec& G0) {
  Retrace R;
  const float d2n = dot3(dr, dr);
  const float ids = rsqrtf(d2n);
  R.t = {dr.x * ids, dr.y * ids, dr.z * ids};  // chord direction (Eq. 5)
  basis(R.t, R.e1, R.e2);                      // transverse basis (Eq. 6)
  R.eps = (eps_fixed > 0.f) ? eps_fixed : eta * (d2n * ids);  // Eq. 8
  const Vec sa{R.eps * R.e1.x, R.eps * R.e1.y, R.eps * R.e1.z}, sb{R.eps * R.e2.x, R.eps * R.e2.y, R.eps * R.e2.z};
  // raw separations: NB >= 4: D_j = G_{+j} - G_{-j} over the +-pair j
  // (neighbour q is the "+" (even q) or "-" (odd q) member of pair q / 2);
  // NB == 2: D_j = G_j.  One retrace per loop trip keeps the code small.
  constexpr int NP = (NB >= 4) ? NB / 2 : 2;
  Vec D[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) D[m] = {0.f, 0.f, 0.f};
#pragma unroll 1
  for (int q = 0; q < NB; ++q) {
    const int j = (NB >= 4) ? (q >> 1) : q;
    const float sgn = (NB >= 4 && (q & 1)) ? -1.f : 1.f;
    const Vec off = (NB >= 4) ? pair_offset(j, sa, sb) : ((j == 0) ? sa : sb);
    const Vec g = rk4_g3(G, kf, h, fmaf(sgn, off.x, px), fmaf(sgn, off.y, py), fmaf(sgn, off.z, pz), kx, ky, kz);
#pragma unroll
    for (int m = 0; m < NP; ++m)
      if (m == j) D[m] = {fmaf(sgn, g.x, D[m].x), fmaf(sgn, g.y, D[m].y), fmaf(sgn, g.z, D[m].z)};
  }
  if (NB == 2) {  // one-sided: d_j = eps e_j + h^2/6 (G_j - G_0)
    const float sc = h2_6 / R.eps;
    R.c1 = {sc * (D[0].x - G0.x), sc * (D[0].y - G0.y), sc * (D[0].z - G0.z)};
    R.c2 = {sc * (D[1].x - G0.x), sc * (D[1].y - G0.y), sc * (D[1].z - G0.z)};
  } else {        // central difference: d = eps e + h^2/12 (G_+ - G_-)
    const float sc = h2_12 / R.eps;
    R.c1 = {sc * D[0].x, sc * D[0].y, sc * D[0].z};
    R.c2 = {sc * D[1].x, sc * D[1].y, sc * D[1].z};
  }
  R.lm = ln_m(R.c1, R.c2, R.e1, R.e2, R.t);
  if (NB == 8) {
    const float s2 = 0.70710678118654752f, sc = h2_12 / R.eps;
    const Vec g1{s2 * (R.e1.x + R.e2.x), s2 * (R.e1.y + R.e2.y), s2 * (R.e1.z + R.e2.z)};
    const Vec g2{s2 * (R.e2.x - R.e1.x), s2 * (R.e2.y - R.e1.y), s2 * (R.e2.z - R.e1.z)};
    const Vec c3{sc * D[2 % NP].x, sc * D[2 % NP].y, sc * D[2 % NP].z};
    const Vec c4{sc * D[3 % NP].x, sc * D[3 % NP].y, sc * D[3 % NP].z};
    const float lm2 = ln_m(c3, c4, g1, g2, R.t);
    // M = (M_e + M_g) / 2
    R.lm = fmaxf(R.lm, lm2) + log1p_small(__expf(-fabsf(R.lm - lm2))) - 0.69314718055994531f;
  }
  return R;
}

template <int NB, bool kMixed>
__global__ void __launch_bounds__(kThreads, kRayMinBlocks) trace_rays(const __grid_constant__ TraceParams P) {
  const int lane = threadIdx.x & 31;
  const float h = P.h;

  // per-ray state; what is touched only when a ray starts or ends lives in
  // shared memory (it would otherwise hold registers through every step)
  struct Cold {
    float* out;
    RayDiag* dg;
    unsigned long long steps_done, rays_done;
    unsigned int item;
    int ck_last;  // tape: the ray's last checkpoint slot (-1: none)
  };
  __shared__ Cold cold[kThreads];
  Cold& C = cold[threadIdx.x];
  C.out = nullptr;
  C.dg = nullptr;
  C.steps_done = 0;
  C.rays_done = 0;
  C.item = 0;
  C.ck_last = -1;
  int step = 0;
  bool active = false, exhausted = false;
  float px = 0.f, py = 0.f, pz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
  float rlx = 0.f, rly = 0.f, rlz = 0.f, klx = 0.f, kly = 0.f, klz = 0.f;  // compensation (kMixed)
  float kf = 0.f, kap_c = 0.f, ln_f = 0.f;
  float tau_hi = 0.f, tau_lo = 0.f, lns_hi = 0.f, lns_lo = 0.f, tb_hi = 0.f, tb_lo = 0.f;
  float kap_prev = 0.f, te_prev = 0.f;

  auto finish = [&](int st, float ex, float ey, float ez) {
    *C.out = tb_hi + tb_lo;
    RayDiag* dg = C.dg;
    if (dg) {
      RayDiag d;
      d.exit_pos[0] = ex; d.exit_pos[1] = ey; d.exit_pos[2] = ez;
      d.tau = tau_hi + tau_lo;
      d.ln_s = lns_hi + lns_lo;
      d.steps = step;
      d.status = st;
      *dg = d;
    }
    if (P.ck_last) P.ck_last[C.item] = C.ck_last;
    C.steps_done += (unsigned long long)step;
    C.rays_done += 1;
    active = false;
  };

  // One central step of this thread's bundle.  Every lane of the warp runs
  // it while any lane holds a ray: a lane without one (only when the ticket
  // pool is exhausted) computes on its stale state, whose lookups stay in
  // bounds, and writes nothing.  Keeping the evaluations out of divergent
  // branches lets warp-uniform values (grid and step parameters) live in
  // uniform registers.
  auto step_once = [&]() {
    // ---------------------------------------------- (a) central RK4 step
    const Rk4Out o = rk4_central(P.G, kf, h, px, py, pz, kx, ky, kz);
    const float kap = P.emission ? kappa_vac(o.ne1, o.te1, kap_c, ln_f) : 0.f;

    // ---------------------------------------------- (b) segment step-1 -> step
    int stop = 0;  // TAU_STOP or STEP_LIMIT: the path ends at node `step`
    if (step >= 1) {
      const float dt = 0.5f * (kap_prev + kap) * P.hrsun;
      const float tbar = 0.5f * (te_prev + o.te1);
      const float tau0 = tau_hi + tau_lo;
      acc_add<kMixed>(tb_hi, tb_lo, tbar * one_minus_exp_neg(dt) * __expf((lns_hi + lns_lo) - tau0));
      acc_add<kMixed>(tau_hi, tau_lo, dt);
      if (P.tau_stop > 0.f && tau_hi + tau_lo >= P.tau_stop) stop = kTauStop;
      else if (step >= P.max_steps) stop = kStepLimit;
    }
    if (active && stop == 0 && P.ckpt && (step % kCkptEvery) == 0) {
      // state at node `step` for the adjoint's recomputation: in the ray's
      // own slots, or (a tape) in the next pool slot, linked to its previous
      unsigned long long slot;
      bool ok;
      if (P.ck_prev) {
        slot = atomicAdd(P.pool_counter, 1ull);
        ok = slot < P.pool_cap;  // an overflowing tape is detected from the counter
      } else {
        const unsigned int item = C.item;
        slot = P.ck_off[item] + (unsigned long long)(step / kCkptEvery);
        ok = slot < P.ck_off[item + 1];
      }
      if (ok) {
        Ckpt& c = P.ckpt[slot];
        c.r[0] = px; c.r[1] = py; c.r[2] = pz;
        c.k[0] = kx; c.k[1] = ky; c.k[2] = kz;
        c.rl[0] = rlx; c.rl[1] = rly; c.rl[2] = rlz;
        c.kl[0] = klx; c.kl[1] = kly; c.kl[2] = klz;
        c.tau_hi = tau_hi; c.tau_lo = tau_lo;
        c.lns_hi = lns_hi; c.lns_lo = lns_lo;
        c.step = step;
        if (P.ck_prev) {
          P.ck_prev[slot] = C.ck_last;
          C.ck_last = (int)slot;
        }
      }
    }

    // ---------------------------------------------- (c) complete step `step`
    const float qx = px, qy = py, qz = pz;  // node `step` (a stopped path ends there)
    Vec dr, rn, kn;
    complete_step<kMixed>(h, P.h2_6, P.h_6, o, px, py, pz, kx, ky, kz, rlx, rly, rlz, klx, kly, klz, dr, rn, kn);
    kap_prev = kap;
    te_prev = o.te1;
    const float rr2 = dot3(rn, rn);
    int term = 0;  // 0: carry on; else the status of a last step
    if (rr2 < P.G.r_min * P.G.r_min) term = kHitInner;
    else if (rr2 > P.G.r_max * P.G.r_max && dot3(rn, kn) > 0.f) term = kExitOuter;
    else if (!isfinite(rr2 + kn.x + kn.y + kn.z)) term = kNan;

    // ---------------------------------------------- (d) neighbour retrace of step `step`
    if (NB > 0) {
      const Retrace R = retrace_step<NB>(P.G, kf, h, P.h2_6, P.h2_12, P.eta, P.eps_fixed, px, py, pz, kx, ky, kz,
                                         dr, Vec{o.Gx, o.Gy, o.Gz});
      if (stop == 0 && term != kNan) acc_add<kMixed>(lns_hi, lns_lo, R.lm);
    }
    if (!active) return;

    // ---------------------------------------------- (e) next node, or the end of the path
    if (stop != 0) {
      finish(stop, qx, qy, qz);
    } else if (term == 0) {
      px = rn.x; py = rn.y; pz = rn.z;
      kx = kn.x; ky = kn.y; kz = kn.z;
      step += 1;
    } else if (term == kNan) {
      step += 1;
      finish(kNan, rn.x, rn.y, rn.z);
    } else {
      // clipped last segment + boundary term (Eq. 2 front to back); the
      // crossing point closes the path
      const Vec here{px, py, pz};
      const float a = chord_crossing(here, dr, (term == kHitInner) ? P.G.r_min : P.G.r_max, term == kExitOuter);
      const float cx = fmaf(a, dr.x, px), cy = fmaf(a, dr.y, py), cz = fmaf(a, dr.z, pz);
      const Sample s = eval_field_t<true>(P.G, cx, cy, cz, true);
      const float kap_e = P.emission ? kappa_vac(s.ne, s.te, kap_c, ln_f) : 0.f;
      const float dt = 0.5f * (kap_prev + kap_e) * P.hrsun * a;
      const float tbar = 0.5f * (te_prev + s.te);
      const float lns = lns_hi + lns_lo;
      acc_add<kMixed>(tb_hi, tb_lo, tbar * one_minus_exp_neg(dt) * __expf(lns - (tau_hi + tau_lo)));
      acc_add<kMixed>(tau_hi, tau_lo, dt);
      float tbc = 0.f;
      if (term == kHitInner) tbc = (P.tbc_mode == 1) ? P.tbc_K : s.te;
      if (tbc != 0.f) acc_add<kMixed>(tb_hi, tb_lo, tbc * __expf(lns - (tau_hi + tau_lo)));
      step += 1;
      finish(term, cx, cy, cz);
    }
  };

  while (true) {
    // ------------------------------------------------------------ refill
    bool need = !active && !exhausted;
    unsigned needmask = __ballot_sync(kFull, need);
    while (needmask) {
      const int leader = __ffs(needmask) - 1;
      unsigned int first = 0;
      if (lane == leader) first = atomicAdd(P.counter, (unsigned)__popc(needmask));
      first = __shfl_sync(kFull, first, leader);
      if (need) {
        const unsigned int item = first + __popc(needmask & ((1u << lane) - 1u));
        if (item >= P.total) {
          exhausted = true;
          need = false;
        } else {
          const RayStart rs = start_ray(P, item);
          C.item = item;
          C.out = rs.out;
          C.dg = rs.dg;
          C.ck_last = -1;
          if (rs.valid) {  // a ragged chunk tail has no ray behind the ticket: take another
            kf = P.straight ? 0.f : rs.F->kf;
            kap_c = rs.F->kap_c;
            ln_f = rs.F->ln_f;
            step = 0;
            tau_hi = tau_lo = lns_hi = lns_lo = tb_hi = tb_lo = 0.f;
            rlx = rly = rlz = klx = kly = klz = 0.f;
            kap_prev = te_prev = 0.f;
            if (!rs.enter) {
              finish(kMiss, rs.px, rs.py, rs.pz);
            } else {
              px = rs.px; py = rs.py; pz = rs.pz;
              kx = rs.kx; ky = rs.ky; kz = rs.kz;
              active = true;
              need = false;
            }
          }
        }
      }
      needmask = __ballot_sync(kFull, need);
    }
    if (!__any_sync(kFull, active)) break;
    step_once();
  }

  // ---- statistics
  unsigned long long steps_done = C.steps_done, rays_done = C.rays_done;
  for (int off = 16; off > 0; off >>= 1) {
    steps_done += __shfl_down_sync(kFull, steps_done, off);
    rays_done += __shfl_down_sync(kFull, rays_done, off);
  }
  if (lane == 0 && P.stats) {
    atomicAdd(P.stats, steps_done);
    atomicAdd(P.stats + 1, rays_done);
  }
}

}  // namespace rt

namespace rt {

// One node of a recorded ray path (rt_path_node).
struct PathNode {
  float r[3];
  float ln_s;     // ln(S / S_0) at the node
  float dlns_ds;  // ln M of the step arriving at the node over its chord length (0 at node 0)
  float tau;      // optical depth from the entry to the node
  float ne, te;   // the interpolated n_e and T_e at the node
};

// Ray-fan diagnostics (Sec. 3.2, Figs. 4 and 6): the rays of the given pixels
// at one frequency, one thread each, stepped exactly as trace_rays steps
// them (the same step code in the same order), recording every node.
// The first `cap` nodes of ray i go to path[i * cap ...], its node count to
// count[i], and its T_b and diagnostics to tb[i] and diag[i].
template <int NB, bool kMixed>
__global__ void __launch_bounds__(64) trace_paths(const __grid_constant__ TraceParams P, const int* __restrict__ pix,
                                                  int n, int cap, PathNode* __restrict__ path, int* __restrict__ count,
                                                  float* __restrict__ tb, RayDiag* __restrict__ diag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = P.h;
  RayStart rs;
  rs.V = &P.view;
  rs.F = &P.freq[0];
  ray_entry(P, rs.V, rs.F, pix[i], rs);
  PathNode* out = path + (size_t)i * cap;
  int nodes = 0;
  auto record = [&](float x, float y, float z, float lns, float dls, float tau, float ne, float te) {
    if (nodes < cap) {
      PathNode& q = out[nodes];
      q.r[0] = x; q.r[1] = y; q.r[2] = z;
      q.ln_s = lns; q.dlns_ds = dls; q.tau = tau; q.ne = ne; q.te = te;
    }
    ++nodes;
  };
  float tb_hi = 0.f, tb_lo = 0.f, tau_hi = 0.f, tau_lo = 0.f, lns_hi = 0.f, lns_lo = 0.f;
  int step = 0, status = kMiss;
  float ex = rs.px, ey = rs.py, ez = rs.pz;
  if (rs.enter) {
    const float kf = P.straight ? 0.f : rs.F->kf, kap_c = rs.F->kap_c, ln_f = rs.F->ln_f;
    float px = rs.px, py = rs.py, pz = rs.pz, kx = rs.kx, ky = rs.ky, kz = rs.kz;
    float rlx = 0.f, rly = 0.f, rlz = 0.f, klx = 0.f, kly = 0.f, klz = 0.f;
    float kap_prev = 0.f, te_prev = 0.f, dls = 0.f;
    while (true) {
      const Rk4Out o = rk4_central(P.G, kf, h, px, py, pz, kx, ky, kz);
      const float kap = P.emission ? kappa_vac(o.ne1, o.te1, kap_c, ln_f) : 0.f;
      if (step >= 1) {
        const float dt = 0.5f * (kap_prev + kap) * P.hrsun;
        const float tbar = 0.5f * (te_prev + o.te1);
        const float tau0 = tau_hi + tau_lo;
        acc_add<kMixed>(tb_hi, tb_lo, tbar * one_minus_exp_neg(dt) * __expf((lns_hi + lns_lo) - tau0));
        acc_add<kMixed>(tau_hi, tau_lo, dt);
      }
      record(px, py, pz, lns_hi + lns_lo, dls, tau_hi + tau_lo, o.ne1, o.te1);
      ex = px; ey = py; ez = pz;
      if (step >= 1 && P.tau_stop > 0.f && tau_hi + tau_lo >= P.tau_stop) { status = kTauStop; break; }
      if (step >= 1 && step >= P.max_steps) { status = kStepLimit; break; }
      Vec dr, rn, kn;
      complete_step<kMixed>(h, P.h2_6, P.h_6, o, px, py, pz, kx, ky, kz, rlx, rly, rlz, klx, kly, klz, dr, rn, kn);
      kap_prev = kap;
      te_prev = o.te1;
      const float rr2 = dot3(rn, rn);
      int term = 0;
      if (rr2 < P.G.r_min * P.G.r_min) term = kHitInner;
      else if (rr2 > P.G.r_max * P.G.r_max && dot3(rn, kn) > 0.f) term = kExitOuter;
      else if (!isfinite(rr2 + kn.x + kn.y + kn.z)) term = kNan;
      dls = 0.f;
      if (NB > 0 && term != kNan) {
        const Retrace R = retrace_step<(NB > 0 ? NB : 4)>(P.G, kf, h, P.h2_6, P.h2_12, P.eta, P.eps_fixed, px, py,
                                                          pz, kx, ky, kz, dr, Vec{o.Gx, o.Gy, o.Gz});
        acc_add<kMixed>(lns_hi, lns_lo, R.lm);
        dls = R.lm * rsqrtf(dot3(dr, dr));
      }
      if (term == 0) {
        px = rn.x; py = rn.y; pz = rn.z;
        kx = kn.x; ky = kn.y; kz = kn.z;
        step += 1;
        continue;
      }
      step += 1;
      status = term;
      if (term == kNan) { ex = rn.x; ey = rn.y; ez = rn.z; break; }
      const Vec here{px, py, pz};
      const float a = chord_crossing(here, dr, (term == kHitInner) ? P.G.r_min : P.G.r_max, term == kExitOuter);
      const float cx = fmaf(a, dr.x, px), cy = fmaf(a, dr.y, py), cz = fmaf(a, dr.z, pz);
      const Sample s = eval_field(P.G, cx, cy, cz, true);
      const float kap_e = P.emission ? kappa_vac(s.ne, s.te, kap_c, ln_f) : 0.f;
      const float dt = 0.5f * (kap_prev + kap_e) * P.hrsun * a;
      const float tbar = 0.5f * (te_prev + s.te);
      const float lns = lns_hi + lns_lo;
      acc_add<kMixed>(tb_hi, tb_lo, tbar * one_minus_exp_neg(dt) * __expf(lns - (tau_hi + tau_lo)));
      acc_add<kMixed>(tau_hi, tau_lo, dt);
      float tbc = 0.f;
      if (term == kHitInner) tbc = (P.tbc_mode == 1) ? P.tbc_K : s.te;
      if (tbc != 0.f) acc_add<kMixed>(tb_hi, tb_lo, tbc * __expf(lns - (tau_hi + tau_lo)));
      record(cx, cy, cz, lns, dls, tau_hi + tau_lo, s.ne, s.te);
      ex = cx; ey = cy; ez = cz;
      break;
    }
  }
  count[i] = nodes;
  tb[i] = tb_hi + tb_lo;
  if (diag) {
    RayDiag d;
    d.exit_pos[0] = ex; d.exit_pos[1] = ey; d.exit_pos[2] = ez;
    d.tau = tau_hi + tau_lo;
    d.ln_s = lns_hi + lns_lo;
    d.steps = step;
    d.status = status;
    diag[i] = d;
  }
}

}  // namespace rt
