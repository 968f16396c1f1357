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

// A ticket decoded into its ray (Sec. 3.2): the view, frequency, pixel and
// outputs, and the launch state.  valid = false for a ticket past a ragged
// chunk or tile edge (no ray behind it); enter = false for a MISS (the line
// misses the outer sphere, or n^2 <= 0 at the entry point).
struct RayStart {
  const ViewDev* V;
  const FreqDev* F;
  float* out;
  RayDiag* dg;
  bool valid, enter;
  float px, py, pz, kx, ky, kz;  // entry point on the outer sphere, k = n(r0) (-o)
  float u, v, sc, nc, nec;       // image-plane point, entry depth, n and n_e at the entry (tube launch)
};

// The launch of the ray of pixel pix (Sec. 3.2): its image-plane point, the
// entry point on the outer sphere and k = n(r0) (-o); enter = false for a
// MISS.
__device__ __forceinline__ void ray_entry(const TraceParams& P, const ViewDev* V, const FreqDev* F, int pix,
                                          RayStart& s) {
  s.enter = false;
  s.px = s.py = s.pz = s.kx = s.ky = s.kz = 0.f;
  s.sc = s.nec = 0.f;
  s.nc = 1.f;
  const int ix = pix % V->nx, iy = pix / V->nx;
  s.u = fmaf((float)ix + 0.5f, V->dx, V->x0);
  s.v = fmaf((float)iy + 0.5f, V->dy, V->y0);
  const float R = P.G.r_max;
  const float b2 = fmaf(s.u, s.u, s.v * s.v);
  bool ok = b2 < R * R;
  if (ok) {
    s.sc = sqrtf(fmaf(R, R, -b2));
    s.px = fmaf(s.u, V->eux, fmaf(s.v, V->evx, s.sc * V->ox));
    s.py = fmaf(s.u, V->euy, fmaf(s.v, V->evy, s.sc * V->oy));
    s.pz = fmaf(s.u, V->euz, fmaf(s.v, V->evz, s.sc * V->oz));
    if (!P.straight) {
      const Sample s0 = eval_field(P.G, s.px, s.py, s.pz, false);
      s.nec = s0.ne;
      const float n2 = fmaf(F->kn2, s0.ne, 1.f);
      ok = n2 > 0.f;
      s.nc = ok ? sqrtf(n2) : 0.f;
    }
  }
  s.enter = ok;
  if (ok) {
    s.kx = -s.nc * V->ox;
    s.ky = -s.nc * V->oy;
    s.kz = -s.nc * V->oz;
  }
}

__device__ __forceinline__ RayStart start_ray(const TraceParams& P, unsigned int item) {
  RayStart s;
  int pix;
  s.valid = true;
  if (P.chunks) {
    const ChunkDev c = P.chunks[item >> kChunkShift];
    const int off = (int)(item & (kChunk - 1));
    s.valid = off < c.count;
    const MapDev& M = P.maps[c.map];
    pix = c.pix0 + off;
    s.V = &P.views[M.view];
    s.F = &M.f;
    s.out = M.out + pix;
    s.dg = M.diag ? M.diag + pix : nullptr;
  } else {
    const int fi = item / P.view.tickets;
    const int t = item - fi * P.view.tickets;
    if (P.view.tile > 0) {  // tile-major walk; tickets past the image edge carry no ray
      const int T = P.view.tile, tt = T * T;
      const int tile = t / tt, w = t - tile * tt;
      const int ix = (tile % P.view.tiles_x) * T + w % T, iy = (tile / P.view.tiles_x) * T + w / T;
      s.valid = ix < P.view.nx && iy < P.view.ny;
      pix = s.valid ? iy * P.view.nx + ix : 0;
    } else {
      pix = t;
    }
    s.V = &P.view;
    s.F = &P.freq[fi];
    const size_t o = (size_t)s.F->out_slab * P.view.npix + pix;
    s.out = P.tb_out + o;
    s.dg = P.diag ? P.diag + o : nullptr;
    if (s.valid && P.skip_zero && P.skip_zero[o] == 0.f) {  // not traced: T_b 0, zero diagnostics
      *s.out = 0.f;
      if (s.dg) *s.dg = RayDiag{{0.f, 0.f, 0.f}, 0.f, 0.f, 0, 0};
      s.valid = false;
    }
  }
  s.enter = false;
  if (!s.valid) return s;
  ray_entry(P, s.V, s.F, pix, s);
  return s;
}

// Per-bundle state of the central lane, kept in shared memory so that only
// the RK4 state lives in registers across the four field evaluations.
struct BundleState {
  unsigned int item;                                    // ticket of this ray
  float* out;                                           // T_b of this ray
  RayDiag* dg;                                          // its diagnostics or null
  int step, status;
  float kf, kap_c, ln_f;                                // frequency constants
  float tau_hi, tau_lo, lns_hi, lns_lo, tb_hi, tb_lo;  // running sums (lo: compensation)
  float rl[3], kl[3];                                   // compensation of r and k
  float kap_prev, te_prev;                              // node i-1 transfer values
  float t[3], e1[3], e2[3], eps;                        // basis of the retraced step
  float g0[3];                                          // central G of that step (2 neighbours)
  float alpha, pc[3];                                   // clipped last step
  // tube mode: launch data the neighbour lanes read to start their rays
  const ViewDev* view;
  float u, v, sc, nc, nec, kn2;
  int tube_ok;
  unsigned long long steps_done, rays_done;
};

// Tube-mode image-plane offset of neighbour role q (Sec. 2 persistent
// reading): +-e_u, +-e_v, and with 8 neighbours the 45-degree diagonals.
template <int NB>
__device__ __forceinline__ void tube_offset(int q, float& a, float& b) {
  const float s2 = 0.70710678118654752f;
  if (NB == 2) {
    a = (q == 1) ? 1.f : 0.f;
    b = (q == 1) ? 0.f : 1.f;
    return;
  }
  switch (q) {
    case 1: a = 1.f; b = 0.f; break;
    case 2: a = -1.f; b = 0.f; break;
    case 3: a = 0.f; b = 1.f; break;
    case 4: a = 0.f; b = -1.f; break;
    case 5: a = s2; b = s2; break;
    case 6: a = -s2; b = -s2; break;
    case 7: a = -s2; b = s2; break;
    default: a = s2; b = -s2; break;
  }
}

template <bool kComp>
__device__ __forceinline__ void acc_add(float& hi, float& lo, float x) {
  if (kComp) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  } else {
    hi += x;
  }
}

// kTube: the neighbours are persistent rays launched at image-plane offsets
// +-delta and integrated in lock-step with the central ray; each neighbour
// lane carries its offset (dr, dk) from the central ray, updated with the
// difference of RK4 increments, and S = |det[d1, d2, t]| is taken after every
// step with central differences d_j of those offsets (S_0 = delta^2).
template <int NB, bool kMixed, bool kTube>
__global__ void __launch_bounds__(kThreads, kTube ? kMinBlocksTube : kMinBlocks) trace_bundles(const __grid_constant__ TraceParams P) {
  constexpr int L = NB + 1;
  constexpr int BPW = 32 / L;
  __shared__ BundleState S[kThreads / 32][BPW];
  const int lane = threadIdx.x & 31;
  const int q = lane % L;
  const bool used = (lane / L) < BPW;
  const int base = used ? lane - q : lane;
  const bool central = used && q == 0;
  BundleState& B = S[threadIdx.x >> 5][used ? lane / L : 0];
  const float h = P.h;

  if (central) {
    B.steps_done = 0;
    B.rays_done = 0;
  }
  // ---- per-lane RK4 start state (central: its node; neighbour: its seed)
  float px = 0.f, py = 0.f, pz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
  bool has_seed = false;  // neighbour lanes: a retrace is pending
  int phase = 0;          // central: 0 needs work, 1 stepping, 2 final (clipped) segment
  bool emitted = false;   // central: its neighbours retrace a step this iteration
  bool exhausted = !central;
  bool fresh = false;     // central (tube mode): a ray started in this iteration
  // tube neighbours (mixed form): rounding carried by the offset accumulation
  float lpx = 0.f, lpy = 0.f, lpz = 0.f, lkx = 0.f, lky = 0.f, lkz = 0.f;

  auto finish = [&](int st, float ex, float ey, float ez, float tb_val) {
    *B.out = tb_val;
    if (B.dg) {
      RayDiag d;
      d.exit_pos[0] = ex; d.exit_pos[1] = ey; d.exit_pos[2] = ez;
      d.tau = B.tau_hi + B.tau_lo;
      d.ln_s = B.lns_hi + B.lns_lo;
      d.steps = B.step;
      d.status = st;
      *B.dg = d;
    }
    B.steps_done += (unsigned long long)B.step;
    B.rays_done += 1;
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
        const unsigned int item = first + __popc(needmask & ((1u << lane) - 1u));
        if (item >= P.total) {
          exhausted = true;
          need = false;
        } else {
          const RayStart rs = start_ray(P, item);
          B.out = rs.out;
          B.dg = rs.dg;
          if (rs.valid) {  // a ragged chunk tail has no ray behind the ticket: take another
            B.item = item;
            B.kf = P.straight ? 0.f : rs.F->kf;
            B.kap_c = rs.F->kap_c;
            B.ln_f = rs.F->ln_f;
            B.step = 0;
            B.tau_hi = B.tau_lo = B.lns_hi = B.lns_lo = B.tb_hi = B.tb_lo = 0.f;
            B.rl[0] = B.rl[1] = B.rl[2] = B.kl[0] = B.kl[1] = B.kl[2] = 0.f;
            emitted = false;
            if (!rs.enter) {
              finish(kMiss, rs.px, rs.py, rs.pz, 0.f);
            } else {
              px = rs.px; py = rs.py; pz = rs.pz;
              kx = rs.kx; ky = rs.ky; kz = rs.kz;
              phase = 1;
              need = false;
              if (kTube) {
                B.view = rs.V;
                B.u = rs.u; B.v = rs.v;
                B.sc = rs.sc;
                B.nc = rs.nc;
                B.nec = rs.nec;
                B.kn2 = rs.F->kn2;
                fresh = true;
              }
            }
          }
        }
      }
      needmask = __ballot_sync(kFull, need);
    }
    if (!__any_sync(kFull, phase != 0)) break;

    if (kTube) {
      // neighbours of a new bundle launch from their offset pixel positions:
      // entry offsets and wave-vector offsets formed without cancellation
      const bool fr = __shfl_sync(kFull, fresh ? 1 : 0, base) != 0;
      const float ex = __shfl_sync(kFull, px, base), ey = __shfl_sync(kFull, py, base),
                  ez = __shfl_sync(kFull, pz, base);  // the central entry point
      __syncwarp();
      bool ok = true;
      if (used && q > 0 && fr) {
        float a, b;
        tube_offset<NB>(q, a, b);
        const ViewDev& V = *B.view;
        const float du = P.tube_delta * a, dv = P.tube_delta * b;
        const float R = P.G.r_max;
        const float un = B.u + du, vn = B.v + dv;
        const float b2n = fmaf(un, un, vn * vn);
        ok = b2n < R * R;
        if (ok) {
          const float sn = sqrtf(fmaf(R, R, -b2n));
          const float dsv = -(2.f * fmaf(B.u, du, B.v * dv) + fmaf(du, du, dv * dv)) / (sn + B.sc);
          const float ox = fmaf(du, V.eux, fmaf(dv, V.evx, dsv * V.ox));
          const float oy = fmaf(du, V.euy, fmaf(dv, V.evy, dsv * V.oy));
          const float oz = fmaf(du, V.euz, fmaf(dv, V.evz, dsv * V.oz));
          px = ox; py = oy; pz = oz;
          lpx = lpy = lpz = lkx = lky = lkz = 0.f;
          float nn = 1.f;
          if (!P.straight) {
            const Sample s0 = eval_field_off(P.G, base_point(P.G, ex, ey, ez), ox, oy, oz, false);
            const float n2 = fmaf(B.kn2, s0.ne, 1.f);
            ok = n2 > 0.f;
            nn = ok ? sqrtf(n2) : 0.f;
            const float dn = ok ? B.kn2 * (s0.ne - B.nec) / (nn + B.nc) : 0.f;
            kx = -dn * V.ox; ky = -dn * V.oy; kz = -dn * V.oz;
          } else {
            kx = ky = kz = 0.f;
          }
        }
        has_seed = ok;
      }
      const unsigned okmask = __ballot_sync(kFull, ok);
      if (central && fresh) {
        const unsigned mine = ((1u << (NB + 1)) - 1u) << lane;
        B.tube_ok = ((okmask & mine) == mine) ? 1 : 0;
        fresh = false;
      }
    }

    // ------------------------------------------------------------ RK4
    // central lanes step (phase 1); neighbour lanes retrace (has_seed), or
    // in tube mode step their own rays from the central state + offsets
    const float kf_lane = __shfl_sync(kFull, (central && phase != 0) ? B.kf : 0.f, base);
    const int bphase = __shfl_sync(kFull, phase, base);
    const bool work = central ? (phase == 1) : (kTube ? (has_seed && bphase == 1) : has_seed);
    Rk4Out o;
    o.Gx = o.Gy = o.Gz = o.Ax = o.Ay = o.Az = 0.f;
    o.ne1 = o.te1 = 0.f;
    if (kTube) {
      // every ray of the bundle steps about the central node (b, its low part l)
      float lx = 0.f, ly = 0.f, lz = 0.f;
      if (kMixed && central) { lx = B.rl[0]; ly = B.rl[1]; lz = B.rl[2]; }
      const float cpx = __shfl_sync(kFull, px, base), cpy = __shfl_sync(kFull, py, base),
                  cpz = __shfl_sync(kFull, pz, base);
      const float ckx = __shfl_sync(kFull, kx, base), cky = __shfl_sync(kFull, ky, base),
                  ckz = __shfl_sync(kFull, kz, base);
      lx = __shfl_sync(kFull, lx, base); ly = __shfl_sync(kFull, ly, base); lz = __shfl_sync(kFull, lz, base);
      if (work) {
        const BasePoint bp = base_point(P.G, cpx, cpy, cpz);
        o = rk4_step_base(P.G, kf_lane, h, bp, lx, ly, lz, ckx, cky, ckz, central ? 0.f : px, central ? 0.f : py,
                          central ? 0.f : pz, central ? 0.f : kx, central ? 0.f : ky, central ? 0.f : kz, central);
      }
    } else if (work) {
      o = rk4_step(P.G, kf_lane, h, px, py, pz, kx, ky, kz, central);
    }
    if (central && phase == 2) {  // the clip point closes the path
      const Sample s = eval_field(P.G, B.pc[0], B.pc[1], B.pc[2], true);
      o.ne1 = s.ne;
      o.te1 = s.te;
    }

    // ------------------------------------------------- neighbour exchange
    // raw separations: NB >= 4: D_j = G_{+j} - G_{-j}; NB == 2: G_j
    // (tube mode: the offsets after this step; central differences for 4, 8)
    Vec d1{0.f, 0.f, 0.f}, d2{0.f, 0.f, 0.f}, d3{0.f, 0.f, 0.f}, d4{0.f, 0.f, 0.f};
    if (kTube) {
      const float gcx = __shfl_sync(kFull, o.Gx, base), gcy = __shfl_sync(kFull, o.Gy, base),
                  gcz = __shfl_sync(kFull, o.Gz, base);
      const float acx = __shfl_sync(kFull, o.Ax, base), acy = __shfl_sync(kFull, o.Ay, base),
                  acz = __shfl_sync(kFull, o.Az, base);
      if (work && !central) {
        // offset update: d(dr) = h dk + h^2/6 (G_nb - G_c), d(dk) = h/6 (A_nb - A_c); the
        // increments are ~1e-6 of the offsets, so the mixed form carries their rounding
        const float ipx = fmaf(h, kx, P.h2_6 * (o.Gx - gcx)), ipy = fmaf(h, ky, P.h2_6 * (o.Gy - gcy)),
                    ipz = fmaf(h, kz, P.h2_6 * (o.Gz - gcz));
        const float ikx = P.h_6 * (o.Ax - acx), iky = P.h_6 * (o.Ay - acy), ikz = P.h_6 * (o.Az - acz);
        if (kMixed) {
          float t;
          two_sum(px, ipx + lpx, t, lpx); px = t;
          two_sum(py, ipy + lpy, t, lpy); py = t;
          two_sum(pz, ipz + lpz, t, lpz); pz = t;
          two_sum(kx, ikx + lkx, t, lkx); kx = t;
          two_sum(ky, iky + lky, t, lky); ky = t;
          two_sum(kz, ikz + lkz, t, lkz); kz = t;
        } else {
          px += ipx; py += ipy; pz += ipz;
          kx += ikx; ky += iky; kz += ikz;
        }
      }
      if (NB == 2) {
        d1 = {__shfl_sync(kFull, px, base + 1), __shfl_sync(kFull, py, base + 1), __shfl_sync(kFull, pz, base + 1)};
        d2 = {__shfl_sync(kFull, px, base + 2), __shfl_sync(kFull, py, base + 2), __shfl_sync(kFull, pz, base + 2)};
      } else {
        const float dx = 0.5f * (px - __shfl_down_sync(kFull, px, 1));
        const float dy = 0.5f * (py - __shfl_down_sync(kFull, py, 1));
        const float dz = 0.5f * (pz - __shfl_down_sync(kFull, pz, 1));
        d1 = {__shfl_sync(kFull, dx, base + 1), __shfl_sync(kFull, dy, base + 1), __shfl_sync(kFull, dz, base + 1)};
        d2 = {__shfl_sync(kFull, dx, base + 3), __shfl_sync(kFull, dy, base + 3), __shfl_sync(kFull, dz, base + 3)};
        if (NB == 8) {
          d3 = {__shfl_sync(kFull, dx, base + 5), __shfl_sync(kFull, dy, base + 5), __shfl_sync(kFull, dz, base + 5)};
          d4 = {__shfl_sync(kFull, dx, base + 7), __shfl_sync(kFull, dy, base + 7), __shfl_sync(kFull, dz, base + 7)};
        }
      }
    } else if (NB == 2) {
      d1 = {__shfl_sync(kFull, o.Gx, base + 1), __shfl_sync(kFull, o.Gy, base + 1), __shfl_sync(kFull, o.Gz, base + 1)};
      d2 = {__shfl_sync(kFull, o.Gx, base + 2), __shfl_sync(kFull, o.Gy, base + 2), __shfl_sync(kFull, o.Gz, base + 2)};
    } else if (NB >= 4) {
      // "+" members (odd roles) form G_+ - G_- with their "-" partner
      const float dx = o.Gx - __shfl_down_sync(kFull, o.Gx, 1);
      const float dy = o.Gy - __shfl_down_sync(kFull, o.Gy, 1);
      const float dz = o.Gz - __shfl_down_sync(kFull, o.Gz, 1);
      d1 = {__shfl_sync(kFull, dx, base + 1), __shfl_sync(kFull, dy, base + 1), __shfl_sync(kFull, dz, base + 1)};
      d2 = {__shfl_sync(kFull, dx, base + 3), __shfl_sync(kFull, dy, base + 3), __shfl_sync(kFull, dz, base + 3)};
      if (NB == 8) {
        d3 = {__shfl_sync(kFull, dx, base + 5), __shfl_sync(kFull, dy, base + 5), __shfl_sync(kFull, dz, base + 5)};
        d4 = {__shfl_sync(kFull, dx, base + 7), __shfl_sync(kFull, dy, base + 7), __shfl_sync(kFull, dz, base + 7)};
      }
    }

    // ------------------------------------------------- central bookkeeping
    bool emit = false;
    Vec sr{0.f, 0.f, 0.f}, sk{0.f, 0.f, 0.f}, sa{0.f, 0.f, 0.f}, sb{0.f, 0.f, 0.f};
    if (central && phase != 0) {
      if (!kTube && emitted && NB > 0) {  // M of the step the neighbours just retraced (Eqs. 9-11)
        const Vec tp{B.t[0], B.t[1], B.t[2]};
        const Vec e1p{B.e1[0], B.e1[1], B.e1[2]}, e2p{B.e2[0], B.e2[1], B.e2[2]};
        Vec c1, c2;
        if (NB == 2) {  // one-sided: d_j = eps e_j + h^2/6 (G_j - G_0)
          const float sc = P.h2_6 / B.eps;
          c1 = {sc * (d1.x - B.g0[0]), sc * (d1.y - B.g0[1]), sc * (d1.z - B.g0[2])};
          c2 = {sc * (d2.x - B.g0[0]), sc * (d2.y - B.g0[1]), sc * (d2.z - B.g0[2])};
        } else {        // central difference: d = eps e + h^2/12 (G_+ - G_-)
          const float sc = P.h2_12 / B.eps;
          c1 = {sc * d1.x, sc * d1.y, sc * d1.z};
          c2 = {sc * d2.x, sc * d2.y, sc * d2.z};
        }
        float lm = ln_m(c1, c2, e1p, e2p, tp);
        if (NB == 8) {
          const float s2 = 0.70710678118654752f, sc = P.h2_12 / B.eps;
          const Vec g1{s2 * (e1p.x + e2p.x), s2 * (e1p.y + e2p.y), s2 * (e1p.z + e2p.z)};
          const Vec g2{s2 * (e2p.x - e1p.x), s2 * (e2p.y - e1p.y), s2 * (e2p.z - e1p.z)};
          const Vec c3{sc * d3.x, sc * d3.y, sc * d3.z}, c4{sc * d4.x, sc * d4.y, sc * d4.z};
          const float lm2 = ln_m(c3, c4, g1, g2, tp);
          // M = (M_e + M_g) / 2
          lm = fmaxf(lm, lm2) + log1p_small(__expf(-fabsf(lm - lm2))) - 0.69314718055994531f;
        }
        acc_add<kMixed>(B.lns_hi, B.lns_lo, lm);
      }
      const float kap = P.emission ? kappa_vac(o.ne1, o.te1, B.kap_c, B.ln_f) : 0.f;
      bool done = false;
      if (phase == 2) {
        // clipped last segment + boundary term (Eq. 2 front to back)
        const float dt = 0.5f * (B.kap_prev + kap) * P.hrsun * B.alpha;
        const float tbar = 0.5f * (B.te_prev + o.te1);
        const float lns = B.lns_hi + B.lns_lo;
        acc_add<kMixed>(B.tb_hi, B.tb_lo, tbar * one_minus_exp_neg(dt) * __expf(lns - (B.tau_hi + B.tau_lo)));
        acc_add<kMixed>(B.tau_hi, B.tau_lo, dt);
        float tbc = 0.f;
        if (B.status == kHitInner) tbc = (P.tbc_mode == 1) ? P.tbc_K : o.te1;
        if (tbc != 0.f) acc_add<kMixed>(B.tb_hi, B.tb_lo, tbc * __expf(lns - (B.tau_hi + B.tau_lo)));
        B.step += 1;
        finish(B.status, B.pc[0], B.pc[1], B.pc[2], B.tb_hi + B.tb_lo);
        done = true;
      } else {
        const int step = B.step;
        if (step >= 1) {
          // segment step-1 -> step (Eq. 2 with Eq. 12, front to back)
          const float dt = 0.5f * (B.kap_prev + kap) * P.hrsun;
          const float tbar = 0.5f * (B.te_prev + o.te1);
          const float tau0 = B.tau_hi + B.tau_lo;
          acc_add<kMixed>(B.tb_hi, B.tb_lo, tbar * one_minus_exp_neg(dt) * __expf((B.lns_hi + B.lns_lo) - tau0));
          acc_add<kMixed>(B.tau_hi, B.tau_lo, dt);
          if (P.tau_stop > 0.f && B.tau_hi + B.tau_lo >= P.tau_stop) {
            finish(kTauStop, px, py, pz, B.tb_hi + B.tb_lo);
            done = true;
          } else if (step >= P.max_steps) {
            finish(kStepLimit, px, py, pz, B.tb_hi + B.tb_lo);
            done = true;
          }
        }
        if (!done && P.ckpt && (step % kCkptEvery) == 0) {
          // state at node `step` for the adjoint's recomputation (bounded by the ray's allocation)
          const unsigned long long slot = P.ck_off[B.item] + (unsigned long long)(step / kCkptEvery);
          if (slot < P.ck_off[B.item + 1]) {
            Ckpt& c = P.ckpt[slot];
            c.r[0] = px; c.r[1] = py; c.r[2] = pz;
            c.k[0] = kx; c.k[1] = ky; c.k[2] = kz;
            c.rl[0] = B.rl[0]; c.rl[1] = B.rl[1]; c.rl[2] = B.rl[2];
            c.kl[0] = B.kl[0]; c.kl[1] = B.kl[1]; c.kl[2] = B.kl[2];
            c.tau_hi = B.tau_hi; c.tau_lo = B.tau_lo;
            c.lns_hi = B.lns_hi; c.lns_lo = B.lns_lo;
          }
        }
        if (!done) {
          // complete central step `step` (Eq. 4, RK4 increment form)
          float rlx = B.rl[0], rly = B.rl[1], rlz = B.rl[2];
          float klx = B.kl[0], kly = B.kl[1], klz = B.kl[2];
          const Vec dr{fmaf(h, kx + klx, P.h2_6 * o.Gx), fmaf(h, ky + kly, P.h2_6 * o.Gy),
                       fmaf(h, kz + klz, P.h2_6 * o.Gz)};
          const Vec dk{P.h_6 * o.Ax, P.h_6 * o.Ay, P.h_6 * o.Az};
          sr = {px, py, pz};
          sk = {kx, ky, kz};
          // chord, basis and eps of this step (Eqs. 5, 6, 8)
          const float d2n = dot3(dr, dr);
          const float ids = rsqrtf(d2n);
          const Vec tp{dr.x * ids, dr.y * ids, dr.z * ids};
          if (kTube) {
            // S_{i+1} = |det[d1, d2, t^i]| (8: mean of the two pairs), ln(S / delta^2)
            if (B.tube_ok) {
              const float cx = d1.y * d2.z - d1.z * d2.y, cy = d1.z * d2.x - d1.x * d2.z, cz = d1.x * d2.y - d1.y * d2.x;
              float S = fabsf(fmaf(tp.x, cx, fmaf(tp.y, cy, tp.z * cz)));
              if (NB == 8) {
                const float gx = d3.y * d4.z - d3.z * d4.y, gy = d3.z * d4.x - d3.x * d4.z, gz = d3.x * d4.y - d3.y * d4.x;
                S = 0.5f * (S + fabsf(fmaf(tp.x, gx, fmaf(tp.y, gy, tp.z * gz))));
              }
              B.lns_hi = __logf(S * P.inv_delta2);
              B.lns_lo = 0.f;
            }
          } else if (NB > 0) {
            Vec e1p, e2p;
            basis(tp, e1p, e2p);
            const float eps = (P.eps_fixed > 0.f) ? P.eps_fixed : P.eta * (d2n * ids);
            B.t[0] = tp.x; B.t[1] = tp.y; B.t[2] = tp.z;
            B.e1[0] = e1p.x; B.e1[1] = e1p.y; B.e1[2] = e1p.z;
            B.e2[0] = e2p.x; B.e2[1] = e2p.y; B.e2[2] = e2p.z;
            B.eps = eps;
            sa = {eps * e1p.x, eps * e1p.y, eps * e1p.z};
            sb = {eps * e2p.x, eps * e2p.y, eps * e2p.z};
            if (NB == 2) { B.g0[0] = o.Gx; B.g0[1] = o.Gy; B.g0[2] = o.Gz; }
            emit = true;
          }
          Vec rn, kn;
          if (kMixed) {
            float e;
            fast_two_sum(px, dr.x + rlx, rn.x, e); rlx = e;
            fast_two_sum(py, dr.y + rly, rn.y, e); rly = e;
            fast_two_sum(pz, dr.z + rlz, rn.z, e); rlz = e;
            fast_two_sum(kx, dk.x + klx, kn.x, e); klx = e;
            fast_two_sum(ky, dk.y + kly, kn.y, e); kly = e;
            fast_two_sum(kz, dk.z + klz, kn.z, e); klz = e;
            B.rl[0] = rlx; B.rl[1] = rly; B.rl[2] = rlz;
            B.kl[0] = klx; B.kl[1] = kly; B.kl[2] = klz;
          } else {
            rn = {px + dr.x, py + dr.y, pz + dr.z};
            kn = {kx + dk.x, ky + dk.y, kz + dk.z};
          }
          const float rr2 = dot3(rn, rn);
          B.kap_prev = kap;
          B.te_prev = o.te1;
          const Vec here{px, py, pz};
          if (rr2 < P.G.r_min * P.G.r_min) {
            B.status = kHitInner;
            const float a = chord_crossing(here, dr, P.G.r_min, false);
            B.alpha = a;
            B.pc[0] = fmaf(a, dr.x, px); B.pc[1] = fmaf(a, dr.y, py); B.pc[2] = fmaf(a, dr.z, pz);
            phase = 2;
          } else if (rr2 > P.G.r_max * P.G.r_max && dot3(rn, kn) > 0.f) {
            B.status = kExitOuter;
            const float a = chord_crossing(here, dr, P.G.r_max, true);
            B.alpha = a;
            B.pc[0] = fmaf(a, dr.x, px); B.pc[1] = fmaf(a, dr.y, py); B.pc[2] = fmaf(a, dr.z, pz);
            phase = 2;
          } else if (!isfinite(rr2 + kn.x + kn.y + kn.z)) {
            B.step = step + 1;
            finish(kNan, rn.x, rn.y, rn.z, B.tb_hi + B.tb_lo);
            emit = false;
          } else {
            px = rn.x; py = rn.y; pz = rn.z;
            kx = kn.x; ky = kn.y; kz = kn.z;
            B.step = step + 1;
          }
        }
      }
      emitted = emit;
    }

    // ------------------------------------------------- seed broadcast
    if (!kTube && NB > 0) {
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
  unsigned long long my_steps = central ? B.steps_done : 0ull, my_rays = central ? B.rays_done : 0ull;
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
