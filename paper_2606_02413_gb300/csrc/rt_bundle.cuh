// The persistent warp-cooperative ray-bundle kernel.
//
// One bundle = the central ray of a (pixel, frequency) plus NB step-wise
// neighbour rays (Sec. 2.1, Eqs. 5-11) on NB + 1 adjacent lanes; 32 / (NB+1)
// bundles share a warp.  The neighbours of step i can only start once the
// central step i is known (they need its chord t^i, Eqs. 5-8), so the two are
// pipelined: in every iteration the central lane takes step i while its
// neighbours retrace step i - 1, and the magnification M^i and the transfer
// of segment i - 1 are settled at the end of that iteration.
//
// Precision (template kMixed):
//   - neighbour separations are never formed as differences of absolute
//     positions.  A neighbour started at r^i + s eps e with the central k^i
//     ends at r^i + s eps e + h k^i + h^2/6 G_s, so the central difference
//     of a +-e pair is d = eps e + h^2/12 (G_+ - G_-) exactly, and with
//     c_j = (d_j - eps e_j) / eps,
//       |det[d1, d2, t]| / eps^2 = |1 + c1.e1 + c2.e2 + t.(c1 x c2)|
//     for the orthonormal right-handed (e1, e2, t).  ln M = log1p of that.
//   - kMixed keeps the central position / wave vector and the tau, ln S, T_b
//     sums as compensated float pairs (TwoSum), which holds them near double
//     precision over 10^4-step rays at FP32 instruction cost (FP64 runs at
//     a small fraction of the FP32 rate on this GPU).
//
// Work distribution: each bundle takes a ticket from a global atomic queue
// when it finishes (warp-aggregated), so rays of very uneven length keep
// every warp busy; consecutive tickets are adjacent pixels of one frequency.
#pragma once
#include "rt_device.cuh"

namespace rt {

struct Vec {
  float x, y, z;
};

__device__ __forceinline__ float dot3(const Vec& a, const Vec& b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// Transverse basis of Eq. 6: a = z unless |t_z| > 0.9, then y.
__device__ __forceinline__ void basis(const Vec& t, Vec& e1, Vec& e2) {
  Vec c;
  if (fabsf(t.z) <= 0.9f) {  // z x t
    c = {-t.y, t.x, 0.f};
  } else {                   // y x t
    c = {t.z, 0.f, -t.x};
  }
  const float inv = rsqrtf(dot3(c, c));
  e1 = {c.x * inv, c.y * inv, c.z * inv};
  e2 = {t.y * e1.z - t.z * e1.y, t.z * e1.x - t.x * e1.z, t.x * e1.y - t.y * e1.x};
}

// ln |1 + c1.e1 + c2.e2 + t.(c1 x c2)| (see the file comment).
__device__ __forceinline__ float ln_m(const Vec& c1, const Vec& c2, const Vec& e1, const Vec& e2,
                                      const Vec& t) {
  const float cx = c1.y * c2.z - c1.z * c2.y, cy = c1.z * c2.x - c1.x * c2.z, cz = c1.x * c2.y - c1.y * c2.x;
  const float m1 = dot3(c1, e1) + dot3(c2, e2) + fmaf(t.x, cx, fmaf(t.y, cy, t.z * cz));
  return log1p_small(m1);
}

// Root alpha in [0, 1] of |r + alpha dr| = R on the chord (stable form).
__device__ __forceinline__ float chord_crossing(const Vec& r, const Vec& dr, float R, bool leaving) {
  const float A = dot3(dr, dr), B = 2.f * dot3(r, dr), C = fmaf(-R, R, dot3(r, r));
  const float disc = fmaxf(fmaf(B, B, -4.f * A * C), 0.f);
  const float sq = sqrtf(disc);
  float a;
  if (leaving) {  // larger root
    a = (B >= 0.f) ? (2.f * C) / (-B - sq) : (-B + sq) / (2.f * A);
  } else {        // smaller root
    a = (B <= 0.f) ? (2.f * C) / (-B + sq) : (-B - sq) / (2.f * A);
  }
  if (!(a >= 0.f)) a = 0.f;
  return fminf(a, 1.f);
}

template <int NB, bool kMixed>
__global__ void __launch_bounds__(kThreads, kMinBlocks) trace_bundles(const __grid_constant__ TraceParams P) {
  constexpr int L = NB + 1;
  constexpr int BPW = 32 / L;
  const int lane = threadIdx.x & 31;
  const int q = lane % L;
  const bool used = (lane / L) < BPW;
  const int base = used ? lane - q : lane;
  const bool central = used && q == 0;
  const float h = P.h;

  // ---- per-lane RK4 start state
  float px = 0.f, py = 0.f, pz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
  bool has_seed = false;  // neighbour lanes: a retrace is pending
  // ---- central-lane bundle state
  int phase = 0;          // 0 needs work, 1 stepping, 2 final (clipped) segment
  bool exhausted = !used || !central;
  unsigned int item = 0;
  int fi = 0, pix = 0;
  float kf = 0.f;
  int step = 0;
  Acc<kMixed> tau, lns, tb;
  tau.zero(); lns.zero(); tb.zero();
  float rlx = 0.f, rly = 0.f, rlz = 0.f, klx = 0.f, kly = 0.f, klz = 0.f;  // compensation terms
  float kap_prev = 0.f, te_prev = 0.f;
  Vec tp{0.f, 0.f, 1.f}, e1p{1.f, 0.f, 0.f}, e2p{0.f, 1.f, 0.f};  // basis of the step being retraced
  float epsp = 1.f;
  Vec g0p{0.f, 0.f, 0.f};  // central G of that step (one-sided 2-neighbour form)
  bool emitted = false;    // neighbours retrace a step in this iteration
  float alpha = 1.f;
  Vec pc{0.f, 0.f, 0.f};
  int status = 0;
  unsigned long long my_steps = 0, my_rays = 0;

  auto finish = [&](int st, const Vec& endp, float tb_val) {
    const FreqDev& F = P.freq[fi];
    const size_t o = (size_t)F.out_slab * P.npix + pix;
    P.tb_out[o] = tb_val;
    if (P.diag) {
      RayDiag d;
      d.exit_pos[0] = endp.x; d.exit_pos[1] = endp.y; d.exit_pos[2] = endp.z;
      d.tau = tau.val();
      d.ln_s = lns.val();
      d.steps = step;
      d.status = st;
      P.diag[o] = d;
    }
    my_steps += (unsigned long long)step;
    my_rays += 1;
    phase = 0;
  };

  while (true) {
    // ------------------------------------------------------------ refill
    bool need = central && phase == 0 && !exhausted;
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
          // launch (Sec. 3.2): entry point on the outer sphere, k = n(r0) (-o)
          fi = item / P.npix;
          pix = item - fi * P.npix;
          const FreqDev& F = P.freq[fi];
          kf = P.straight ? 0.f : F.kf;
          const int ix = pix % P.nx, iy = pix / P.nx;
          const float u = fmaf((float)ix + 0.5f, P.dx, P.x0);
          const float v = fmaf((float)iy + 0.5f, P.dy, P.y0);
          const float R = P.G.r_max;
          const float b2 = fmaf(u, u, v * v);
          step = 0;
          tau.zero(); lns.zero(); tb.zero();
          rlx = rly = rlz = klx = kly = klz = 0.f;
          emitted = false;
          bool ok = b2 < R * R;
          float nn = 1.f;
          Vec r0{0.f, 0.f, 0.f};
          if (ok) {
            const float s = sqrtf(fmaf(R, R, -b2));
            r0 = {fmaf(u, P.eux, fmaf(v, P.evx, s * P.ox)), fmaf(u, P.euy, fmaf(v, P.evy, s * P.oy)),
                  fmaf(u, P.euz, fmaf(v, P.evz, s * P.oz))};
            if (!P.straight) {
              const Sample s0 = eval_field<false>(P.G, r0.x, r0.y, r0.z);
              const float n2 = fmaf(F.kn2, s0.ne, 1.f);
              ok = n2 > 0.f;
              nn = ok ? sqrtf(n2) : 0.f;
            }
          }
          if (!ok) {
            finish(kMiss, r0, 0.f);
          } else {
            px = r0.x; py = r0.y; pz = r0.z;
            kx = -nn * P.ox; ky = -nn * P.oy; kz = -nn * P.oz;
            phase = 1;
            need = false;
          }
        }
      }
      needmask = __ballot_sync(kFull, need);
    }
    if (!__any_sync(kFull, phase != 0)) break;

    // ------------------------------------------------------------ RK4
    // central lanes step (phase 1); neighbour lanes retrace (has_seed)
    const bool work = central ? (phase == 1) : has_seed;
    Rk4Out o;
    o.Gx = o.Gy = o.Gz = o.Ax = o.Ay = o.Az = 0.f;
    o.ne1 = o.te1 = 0.f;
    const float kf_lane = __shfl_sync(kFull, kf, base);
    if (work) o = rk4_step(P.G, kf_lane, h, px, py, pz, kx, ky, kz, central);
    if (central && phase == 2) {  // the clip point closes the path
      const Sample s = eval_field<true>(P.G, pc.x, pc.y, pc.z);
      o.ne1 = s.ne;
      o.te1 = s.te;
    }

    // ------------------------------------------------- neighbour exchange
    Vec c1{0.f, 0.f, 0.f}, c2{0.f, 0.f, 0.f}, c3{0.f, 0.f, 0.f}, c4{0.f, 0.f, 0.f};
    if (NB == 2) {
      const float gx1 = __shfl_sync(kFull, o.Gx, base + 1), gy1 = __shfl_sync(kFull, o.Gy, base + 1),
                  gz1 = __shfl_sync(kFull, o.Gz, base + 1);
      const float gx2 = __shfl_sync(kFull, o.Gx, base + 2), gy2 = __shfl_sync(kFull, o.Gy, base + 2),
                  gz2 = __shfl_sync(kFull, o.Gz, base + 2);
      const float s = P.h2_6 / epsp;  // one-sided: d_j = eps e_j + h^2/6 (G_j - G_0)
      c1 = {s * (gx1 - g0p.x), s * (gy1 - g0p.y), s * (gz1 - g0p.z)};
      c2 = {s * (gx2 - g0p.x), s * (gy2 - g0p.y), s * (gz2 - g0p.z)};
    } else if (NB >= 4) {
      // "+" members (odd roles) form G_+ - G_- with their "-" partner
      const float dx = o.Gx - __shfl_down_sync(kFull, o.Gx, 1);
      const float dy = o.Gy - __shfl_down_sync(kFull, o.Gy, 1);
      const float dz = o.Gz - __shfl_down_sync(kFull, o.Gz, 1);
      const float s = P.h2_12 / epsp;  // central difference: d = eps e + h^2/12 (G_+ - G_-)
      c1 = {s * __shfl_sync(kFull, dx, base + 1), s * __shfl_sync(kFull, dy, base + 1),
            s * __shfl_sync(kFull, dz, base + 1)};
      c2 = {s * __shfl_sync(kFull, dx, base + 3), s * __shfl_sync(kFull, dy, base + 3),
            s * __shfl_sync(kFull, dz, base + 3)};
      if (NB == 8) {
        c3 = {s * __shfl_sync(kFull, dx, base + 5), s * __shfl_sync(kFull, dy, base + 5),
              s * __shfl_sync(kFull, dz, base + 5)};
        c4 = {s * __shfl_sync(kFull, dx, base + 7), s * __shfl_sync(kFull, dy, base + 7),
              s * __shfl_sync(kFull, dz, base + 7)};
      }
    }

    // ------------------------------------------------- central bookkeeping
    bool emit = false;
    Vec sr{0.f, 0.f, 0.f}, sk{0.f, 0.f, 0.f}, sa{0.f, 0.f, 0.f}, sb{0.f, 0.f, 0.f};
    if (central && phase != 0) {
      const FreqDev& F = P.freq[fi];
      if (emitted && NB > 0) {  // M of the step the neighbours just retraced (Eqs. 9-11)
        float lm = ln_m(c1, c2, e1p, e2p, tp);
        if (NB == 8) {
          const float s2 = 0.70710678118654752f;
          const Vec g1{s2 * (e1p.x + e2p.x), s2 * (e1p.y + e2p.y), s2 * (e1p.z + e2p.z)};
          const Vec g2{s2 * (e2p.x - e1p.x), s2 * (e2p.y - e1p.y), s2 * (e2p.z - e1p.z)};
          const float lm2 = ln_m(c3, c4, g1, g2, tp);
          // M = (M_e + M_g) / 2
          lm = fmaxf(lm, lm2) + log1p_small(__expf(-fabsf(lm - lm2))) - 0.69314718055994531f;
        }
        lns.add(lm);
      }
      const float kap = P.emission ? kappa_vac(o.ne1, o.te1, F) : 0.f;
      bool done = false;
      if (phase == 2) {
        // clipped last segment + boundary term (Eq. 2 front to back)
        const float dt = 0.5f * (kap_prev + kap) * P.hrsun * alpha;
        const float tbar = 0.5f * (te_prev + o.te1);
        tb.add(tbar * one_minus_exp_neg(dt) * __expf(lns.val() - tau.val()));
        tau.add(dt);
        float tbc = 0.f;
        if (status == kHitInner) tbc = (P.tbc_mode == 1) ? P.tbc_K : o.te1;
        if (tbc != 0.f) tb.add(tbc * __expf(lns.val() - tau.val()));
        step += 1;
        finish(status, pc, tb.val());
        done = true;
      } else {
        if (step >= 1) {
          // segment step-1 -> step (Eq. 2 with Eq. 12, front to back)
          const float dt = 0.5f * (kap_prev + kap) * P.hrsun;
          const float tbar = 0.5f * (te_prev + o.te1);
          tb.add(tbar * one_minus_exp_neg(dt) * __expf(lns.val() - tau.val()));
          tau.add(dt);
          const Vec here{px, py, pz};
          if (P.tau_stop > 0.f && tau.val() >= P.tau_stop) {
            finish(kTauStop, here, tb.val());
            done = true;
          } else if (step >= P.max_steps) {
            finish(kStepLimit, here, tb.val());
            done = true;
          }
        }
        if (!done) {
          // complete central step `step` (Eq. 4, RK4 increment form)
          const float kxx = kx + klx, kyy = ky + kly, kzz = kz + klz;
          const Vec dr{fmaf(h, kxx, P.h2_6 * o.Gx), fmaf(h, kyy, P.h2_6 * o.Gy), fmaf(h, kzz, P.h2_6 * o.Gz)};
          const Vec dk{P.h_6 * o.Ax, P.h_6 * o.Ay, P.h_6 * o.Az};
          sr = {px, py, pz};
          sk = {kx, ky, kz};
          // chord, basis and eps of this step (Eqs. 5, 6, 8)
          const float d2 = dot3(dr, dr);
          const float ids = rsqrtf(d2);
          const float ds = d2 * ids;
          tp = {dr.x * ids, dr.y * ids, dr.z * ids};
          if (NB > 0) {
            basis(tp, e1p, e2p);
            epsp = (P.eps_fixed > 0.f) ? P.eps_fixed : P.eta * ds;
            sa = {epsp * e1p.x, epsp * e1p.y, epsp * e1p.z};
            sb = {epsp * e2p.x, epsp * e2p.y, epsp * e2p.z};
            g0p = {o.Gx, o.Gy, o.Gz};
            emit = true;
          }
          Vec rn, kn;
          if (kMixed) {
            float e;
            two_sum(px, dr.x + rlx, rn.x, e); rlx = e;
            two_sum(py, dr.y + rly, rn.y, e); rly = e;
            two_sum(pz, dr.z + rlz, rn.z, e); rlz = e;
            two_sum(kx, dk.x + klx, kn.x, e); klx = e;
            two_sum(ky, dk.y + kly, kn.y, e); kly = e;
            two_sum(kz, dk.z + klz, kn.z, e); klz = e;
          } else {
            rn = {px + dr.x, py + dr.y, pz + dr.z};
            kn = {kx + dk.x, ky + dk.y, kz + dk.z};
          }
          const Vec here{px, py, pz};
          const float rr2 = dot3(rn, rn);
          kap_prev = kap;
          te_prev = o.te1;
          if (rr2 < P.G.r_min * P.G.r_min) {
            status = kHitInner;
            alpha = chord_crossing(here, dr, P.G.r_min, false);
            pc = {fmaf(alpha, dr.x, px), fmaf(alpha, dr.y, py), fmaf(alpha, dr.z, pz)};
            phase = 2;
          } else if (rr2 > P.G.r_max * P.G.r_max && dot3(rn, kn) > 0.f) {
            status = kExitOuter;
            alpha = chord_crossing(here, dr, P.G.r_max, true);
            pc = {fmaf(alpha, dr.x, px), fmaf(alpha, dr.y, py), fmaf(alpha, dr.z, pz)};
            phase = 2;
          } else if (!isfinite(rr2 + kn.x + kn.y + kn.z)) {
            step += 1;
            finish(kNan, rn, tb.val());
            emit = false;
          } else {
            px = rn.x; py = rn.y; pz = rn.z;
            kx = kn.x; ky = kn.y; kz = kn.z;
            step += 1;
          }
        }
      }
      emitted = emit;
    }

    // ------------------------------------------------- seed broadcast
    if (NB > 0) {
      const bool e = __shfl_sync(kFull, emit ? 1 : 0, base) != 0;
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
        // role -> offset: 1 +e1, 2 -e1 (or +e2 with 2 neighbours), 3 +e2, 4 -e2,
        // 5 +g1, 6 -g1, 7 +g2, 8 -g2 with g1 = (e1+e2)/sqrt2, g2 = (e2-e1)/sqrt2
        float ox, oy, oz;
        if (NB == 2) {
          ox = (q == 1) ? ax : cx; oy = (q == 1) ? ay : cy; oz = (q == 1) ? az : cz;
        } else if (q <= 4) {
          const float sgn = (q & 1) ? 1.f : -1.f;
          ox = sgn * ((q <= 2) ? ax : cx);
          oy = sgn * ((q <= 2) ? ay : cy);
          oz = sgn * ((q <= 2) ? az : cz);
        } else {
          const float s2 = 0.70710678118654752f;
          const float sgn = (q & 1) ? 1.f : -1.f;
          const bool g1 = q <= 6;
          ox = sgn * s2 * (g1 ? (ax + cx) : (cx - ax));
          oy = sgn * s2 * (g1 ? (ay + cy) : (cy - ay));
          oz = sgn * s2 * (g1 ? (az + cz) : (cz - az));
        }
        px = bx + ox; py = by + oy; pz = bz + oz;
        kx = bkx; ky = bky; kz = bkz;
      }
    }
  }

  // ---- statistics
  for (int off = 16; off > 0; off >>= 1) {
    my_steps += __shfl_down_sync(kFull, my_steps, off);
    my_rays += __shfl_down_sync(kFull, my_rays, off);
  }
  if (lane == 0 && P.stats) {
    atomicAdd(P.stats, my_steps);
    atomicAdd(P.stats + 1, my_rays);
  }
}

}  // namespace rt
