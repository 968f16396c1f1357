// C-ABI host side of librt: contexts, grid loading and repacking, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "rt.h"
#include "rt_adjoint.cuh"
#include "rt_rays.cuh"

using namespace rt;

namespace {

constexpr double kPi = 3.14159265358979323846;
// CODATA 2018, CGS: f_pe^2 = n_e e^2 / (pi m_e)
constexpr double kElectronCharge = 4.803204712570263e-10;  // statC
constexpr double kElectronMass = 9.1093837015e-28;         // g
constexpr double kRsunCm = 6.957e10;                       // IAU nominal
constexpr double kSpeedOfLightCmS = 2.99792458e10;
constexpr double kAuRsun = 1.495978707e13 / 6.957e10;      // 1 AU in R_sun (IAU)
constexpr double kOuterBand = 1e-6;                        // vacuum beyond r_max (1 + band)

thread_local std::string g_err;

rt_status fail(rt_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define RT_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
    }                                                                                   \
  } while (0)

double c_pe() { return kElectronCharge * kElectronCharge / (kPi * kElectronMass); }

}  // namespace

struct rt_ctx {
  int device = 0;
  int sm_count = 0;
  unsigned int* d_counter = nullptr;        // work-queue ticket
  unsigned long long* d_stats = nullptr;    // [2]
  // pinned staging of rt_trace_image's work tables; stage_done follows the
  // last copy out of it (the next call waits for it before refilling)
  std::mutex stage_mu;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;
};

struct rt_grid {
  GridDev dev{};
  int device = 0;                // CUDA device that holds the grid
  float4* ne = nullptr;
  float4* te = nullptr;
  RadBin* lut = nullptr;
  float2* rcell = nullptr;
  int n_r = 0, n_t = 0, n_p = 0;
  std::vector<double> r;         // radial nodes
  std::vector<double> shell_ne;  // mean n_e over each r shell (work estimates)
};

struct rt_batch_plan {
  rt_ctx* ctx = nullptr;
  ChunkDev* chunks = nullptr;
  MapDev* maps = nullptr;
  ViewDev* views = nullptr;
  unsigned int* counter = nullptr;
  unsigned long long* stats = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// A forward with its checkpoints kept for the reverse sweep.
struct rt_tape {
  rt_ctx* ctx = nullptr;
  const rt_grid* g = nullptr;
  rt_view view{};
  std::vector<double> freqs;
  rt_options opt{};
  int nb = 0;
  bool mixed = true;
  TraceParams P{};                  // the forward's parameters (frequency order, view)
  Ckpt* pool = nullptr;
  int* prev = nullptr;
  int* last = nullptr;
  unsigned long long* counter = nullptr;  // [0] pool slots taken, [1] the adjoint's mismatch count
  unsigned long long cap = 0;
  RayDiag* diag = nullptr;
  bool own_diag = false;
  long total = 0;
};

// --------------------------------------------------------------- kernels
namespace {

template <class T>
__global__ void pack_cells(const T* __restrict__ ne, const T* __restrict__ te, float4* cne, float4* cte,
                           int n_r, int n_t, int n_p) {
  const long ncell = (long)(n_r - 1) * (n_t - 1) * n_p;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell; c += (long)gridDim.x * blockDim.x) {
    const int k = (int)(c % n_p);
    const long ij = c / n_p;
    const int j = (int)(ij % (n_t - 1));
    const int i = (int)(ij / (n_t - 1));
    const int k1 = (k + 1 == n_p) ? 0 : k + 1;
    float vn[8], vt[8];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int cc = 0; cc < 2; ++cc) {
          const long id = ((long)(i + a) * n_t + (j + b)) * n_p + (cc ? k1 : k);
          vn[a * 4 + b * 2 + cc] = (float)ne[id];
          vt[a * 4 + b * 2 + cc] = (float)te[id];
        }
    cne[2 * c] = make_float4(vn[0], vn[1], vn[2], vn[3]);
    cne[2 * c + 1] = make_float4(vn[4], vn[5], vn[6], vn[7]);
    cte[2 * c] = make_float4(vt[0], vt[1], vt[2], vt[3]);
    cte[2 * c + 1] = make_float4(vt[4], vt[5], vt[6], vt[7]);
  }
}

// Mean n_e over each radial shell (one block per shell).
template <class T>
__global__ void shell_mean(const T* __restrict__ ne, int n_tp, double* out) {
  __shared__ double part[256];
  double acc = 0.0;
  const T* row = ne + (long)blockIdx.x * n_tp;
  for (int i = threadIdx.x; i < n_tp; i += blockDim.x) acc += (double)row[i];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = part[0] / n_tp;
}

// Flags non-finite or negative n_e and non-finite or non-positive T_e.
template <class T>
__global__ void check_values(const T* __restrict__ ne, const T* __restrict__ te, long n, unsigned int* bad) {
  unsigned int flag = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double a = (double)ne[i], b = (double)te[i];
    if (!(a >= 0.0) || !std::isfinite(a)) flag |= 1u;
    if (!(b > 0.0) || !std::isfinite(b)) flag |= 2u;
  }
  if (flag) atomicOr(bad, flag);
}

__global__ void probe_field(const GridDev G, const float* __restrict__ xyz, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Sample s = eval_field(G, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], true);
  out[5 * i] = s.ne;
  out[5 * i + 1] = s.te;
  out[5 * i + 2] = s.gx;
  out[5 * i + 3] = s.gy;
  out[5 * i + 4] = s.gz;
}

// Mean T_b over the pixels whose centre lies within `radius` of the image
// centre (Sec. 3.4: the near-centre quiet-Sun spectrum); one block per
// frequency, FP64 sums in a fixed order (deterministic).
// Beam convolution (Sec. 3.3: maps seen by an interferometer of maximum
// baseline B): each map is convolved with a circular Gaussian beam of
// FWHM lambda / B (in R_sun on the image plane at 1 AU), separably, rows then
// columns, with zero outside the image; the weights of one map are the
// normalised samples exp(-d^2 / 2 sigma^2) at the pixel offsets within 4 sigma.
// One thread per output pixel; pass 0 reads src along rows, pass 1 along
// columns.
constexpr int kBeamThreads = 256;
struct BeamParams {
  int nx, ny;
  float inv2s2[kMaxFreq];  // 1 / (2 sigma^2), sigma in pixels
  float norm[kMaxFreq];    // 1 / sum of the map's samples
  int half[kMaxFreq];      // taps each side (ceil(4 sigma))
};

__global__ void __launch_bounds__(kBeamThreads) beam_pass(const float* __restrict__ src, float* __restrict__ dst,
                                                          const __grid_constant__ BeamParams B, int col) {
  const int f = blockIdx.y;
  const int n = B.nx * B.ny;
  const int p = blockIdx.x * kBeamThreads + threadIdx.x;
  if (p >= n) return;
  const float* m = src + (size_t)f * n;
  const int hw = B.half[f];
  const float a = B.inv2s2[f];
  const int ix = p % B.nx, iy = p / B.nx;
  double acc = 0.0;
  for (int d = -hw; d <= hw; ++d) {
    const int jx = col ? ix : ix + d, jy = col ? iy + d : iy;
    if (jx < 0 || jx >= B.nx || jy < 0 || jy >= B.ny) continue;
    acc += (double)expf(-(float)(d * d) * a) * (double)m[jy * B.nx + jx];
  }
  dst[(size_t)f * n + p] = (float)(acc * (double)B.norm[f]);
}

constexpr int kDiskThreads = 512;
__global__ void __launch_bounds__(kDiskThreads) disk_mean(const float* __restrict__ tb, int nx, int ny, double x0,
                                                          double dx, double y0, double dy, double r2,
                                                          double* __restrict__ out) {
  __shared__ double sum[kDiskThreads];
  __shared__ long long cnt[kDiskThreads];
  const float* map = tb + (size_t)blockIdx.x * nx * ny;
  double s = 0.0;
  long long c = 0;
  for (long p = threadIdx.x; p < (long)nx * ny; p += kDiskThreads) {
    const int ix = (int)(p % nx), iy = (int)(p / nx);
    const double u = x0 + (ix + 0.5) * dx, v = y0 + (iy + 0.5) * dy;
    if (u * u + v * v < r2) {
      s += (double)map[p];
      c += 1;
    }
  }
  sum[threadIdx.x] = s;
  cnt[threadIdx.x] = c;
  __syncthreads();
  for (int w = kDiskThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sum[threadIdx.x] += sum[threadIdx.x + w];
      cnt[threadIdx.x] += cnt[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = cnt[0] > 0 ? sum[0] / (double)cnt[0] : 0.0;
}

template <int NB, bool M, bool T>
int blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_bundles<NB, M, T>, kThreads, 0) != cudaSuccess || b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

template <int NB, bool M>
int adj_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, adjoint_rays<NB, M>, kThreads, 0) != cudaSuccess || b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

template <int NB, bool M>
int ray_blocks_per_sm() {
  static int cached = -1;
  if (cached < 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_rays<NB, M>, kThreads, 0) != cudaSuccess || b < 1)
      b = 1;
    cached = b;
  }
  return cached;
}

// tube mode: the lane-parallel bundle kernel (persistent neighbours)
template <int NB, bool M>
cudaError_t launch_tube(const TraceParams& P, int sm_count, cudaStream_t s) {
  const int fit = blocks_per_sm<NB, M, true>();
  const int per_sm = (P.blocks_per_sm > 0) ? std::min(P.blocks_per_sm, fit) : fit;
  trace_bundles<NB, M, true><<<sm_count * per_sm, kThreads, 0, s>>>(P);
  return cudaGetLastError();
}

// step-wise magnification (or none): one thread per bundle
template <int NB, bool M>
cudaError_t launch_rays(const TraceParams& P, int sm_count, cudaStream_t s) {
  const int fit = ray_blocks_per_sm<NB, M>();
  const int per_sm = (P.blocks_per_sm > 0) ? std::min(P.blocks_per_sm, fit) : fit;
  trace_rays<NB, M><<<sm_count * per_sm, kThreads, 0, s>>>(P);
  return cudaGetLastError();
}

// nb: neighbour rays per bundle (0 = magnification off); tube: persistent
// neighbours (tube mode) instead of the step-wise retrace
cudaError_t dispatch_trace(int nb, bool mixed, const TraceParams& P, int sm, cudaStream_t s, bool tube = false) {
  if (tube) {
    switch (nb) {
      case 2: return mixed ? launch_tube<2, true>(P, sm, s) : launch_tube<2, false>(P, sm, s);
      case 4: return mixed ? launch_tube<4, true>(P, sm, s) : launch_tube<4, false>(P, sm, s);
      case 8: return mixed ? launch_tube<8, true>(P, sm, s) : launch_tube<8, false>(P, sm, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (nb) {
    case 0: return mixed ? launch_rays<0, true>(P, sm, s) : launch_rays<0, false>(P, sm, s);
    case 2: return mixed ? launch_rays<2, true>(P, sm, s) : launch_rays<2, false>(P, sm, s);
    case 4: return mixed ? launch_rays<4, true>(P, sm, s) : launch_rays<4, false>(P, sm, s);
    case 8: return mixed ? launch_rays<8, true>(P, sm, s) : launch_rays<8, false>(P, sm, s);
    default: return cudaErrorInvalidValue;
  }
}

bool strictly_increasing(const double* a, int n) {
  for (int i = 0; i + 1 < n; ++i)
    if (!(a[i + 1] > a[i]) || !std::isfinite(a[i]) || !std::isfinite(a[i + 1])) return false;
  return true;
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

void rt_default_options(rt_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->dtau = 2e-3;
  o->s_mode = RT_STEPWISE;
  o->n_nb = 4;
  o->eps_mode = 0;
  o->eta = 0.5;
  o->delta = 1e-3;
  o->tau_stop = 30.0;
  o->max_steps = 0;
  o->tbc_mode = 0;
  o->tbc_K = 0.0;
  o->emission = 1;
  o->straight = 0;
  o->precision = RT_PLAIN_F32;
}

const char* rt_status_string(rt_status s) {
  switch (s) {
    case RT_OK: return "RT_OK";
    case RT_ERR_ARG: return "RT_ERR_ARG";
    case RT_ERR_GRID: return "RT_ERR_GRID";
    case RT_ERR_CUDA: return "RT_ERR_CUDA";
    case RT_ERR_OOM: return "RT_ERR_OOM";
    case RT_ERR_TIMEOUT: return "RT_ERR_TIMEOUT";
    case RT_ERR_CHECKED: return "RT_ERR_CHECKED";
    case RT_ERR_UNSUPPORTED: return "RT_ERR_UNSUPPORTED";
    default: return "RT_ERR_UNKNOWN";
  }
}

const char* rt_last_error(void) { return g_err.c_str(); }

rt_status rt_create(rt_ctx** out, int device) {
  if (!out) return fail(RT_ERR_ARG, "rt_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  RT_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(RT_ERR_ARG, "rt_create: device %d of %d", device, ndev);
  RT_CUDA(cudaSetDevice(device));
  rt_ctx* c = new rt_ctx;
  c->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, 64);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_stats, 64);
  if (e != cudaSuccess) {
    cudaFree(c->d_counter);
    cudaFree(c->d_stats);
    delete c;
    return fail(RT_ERR_CUDA, "rt_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return RT_OK;
}

rt_status rt_destroy(rt_ctx* ctx) {
  if (!ctx) return fail(RT_ERR_ARG, "rt_destroy: ctx is NULL");
  cudaSetDevice(ctx->device);
  if (ctx->stage_done) {
    cudaEventSynchronize(ctx->stage_done);
    cudaEventDestroy(ctx->stage_done);
  }
  cudaFreeHost(ctx->stage);
  cudaFree(ctx->d_counter);
  cudaFree(ctx->d_stats);
  delete ctx;
  return RT_OK;
}

rt_status rt_load_grid(rt_ctx* ctx, const rt_grid_desc* d, const void* ne, const void* te, void* stream,
                       rt_grid** out) {
  if (!ctx || !d || !ne || !te || !out) return fail(RT_ERR_ARG, "rt_load_grid: NULL argument");
  *out = nullptr;
  if (d->dtype != RT_F32 && d->dtype != RT_F64) return fail(RT_ERR_ARG, "rt_load_grid: dtype %d", d->dtype);
  const int nr = d->n_r, nt = d->n_theta, np = d->n_phi;
  if (nr < 2 || nt < 2 || np < 2) return fail(RT_ERR_GRID, "rt_load_grid: need >= 2 nodes per axis");
  if (!d->r_nodes || !d->theta_nodes || !d->phi_nodes) return fail(RT_ERR_ARG, "rt_load_grid: NULL node array");
  const long nodes = (long)nr * nt * np;
  // cells, with the vacuum shell, must index as 2 * cell in 32 bits
  if ((long)nr * (nt - 1) * np > (1L << 31) / 2) return fail(RT_ERR_GRID, "rt_load_grid: grid too large");
  const double* R = d->r_nodes;
  const double* T = d->theta_nodes;
  const double* Ph = d->phi_nodes;
  if (!strictly_increasing(R, nr) || !(R[0] > 0.0))
    return fail(RT_ERR_GRID, "rt_load_grid: r nodes must be positive and strictly increasing");
  if (!strictly_increasing(T, nt) || T[0] < 0.0 || T[nt - 1] > kPi + 1e-12)
    return fail(RT_ERR_GRID, "rt_load_grid: theta nodes must increase strictly within [0, pi]");
  const double dth = (T[nt - 1] - T[0]) / (nt - 1);
  for (int j = 0; j < nt; ++j)
    if (std::fabs(T[j] - (T[0] + j * dth)) > 1e-9)
      return fail(RT_ERR_GRID, "rt_load_grid: theta nodes must be uniformly spaced");
  if (!strictly_increasing(Ph, np)) return fail(RT_ERR_GRID, "rt_load_grid: phi nodes must increase strictly");
  const double dph = 2.0 * kPi / np;
  for (int k = 0; k < np; ++k)
    if (std::fabs(Ph[k] - (Ph[0] + k * dph)) > 1e-9)
      return fail(RT_ERR_GRID, "rt_load_grid: phi nodes must be uniform with n_phi * dphi = 2 pi");

  // radial lookup: bins no wider than the narrowest cell hold at most one node;
  // they start at r = 0, so the bin index of any radius is non-negative
  std::vector<float> Rf(nr);
  for (int i = 0; i < nr; ++i) Rf[i] = (float)R[i];
  double wmin = 1e300;
  for (int i = 0; i + 1 < nr; ++i) wmin = std::min(wmin, (double)Rf[i + 1] - (double)Rf[i]);
  if (!(wmin > 0)) return fail(RT_ERR_GRID, "rt_load_grid: r nodes collapse in FP32");
  const double span = (double)Rf[nr - 1];
  const double nb_d = std::ceil(span / wmin) + 1.0;
  if (nb_d > (double)(1 << 22)) return fail(RT_ERR_GRID, "rt_load_grid: radial spacing too uneven for the lookup table");
  const int nb = (int)nb_d;
  const double bw = span / nb;
  std::vector<float2> rcell(nr - 1);
  for (int i = 0; i + 1 < nr; ++i)
    rcell[i] = make_float2(Rf[i], (float)(1.0 / ((double)Rf[i + 1] - (double)Rf[i])));
  // vacuum beyond r_vac: the lookup's "up" test r >= r_vac_split holds exactly for r > r_vac
  const float r_vac_f = (float)(R[nr - 1] * (1.0 + kOuterBand));
  const float r_vac_split = std::nextafter(r_vac_f, std::numeric_limits<float>::infinity());
  std::vector<RadBin> lut(nb);
  for (int b = 0; b < nb; ++b) {
    const double lo = b * bw, hi = lo + bw;
    int base = (int)(std::upper_bound(Rf.begin(), Rf.end(), (float)lo) - Rf.begin()) - 1;
    base = std::min(std::max(base, 0), nr - 2);
    while (base > 0 && (double)Rf[base] > lo) --base;
    RadBin e{};
    e.base = base;
    e.split = std::numeric_limits<float>::infinity();
    e.r0 = rcell[base].x;
    e.inv0 = rcell[base].y;
    e.inv1 = 0.f;
    if (base + 1 <= nr - 2 && (double)Rf[base + 1] < hi) {
      e.split = Rf[base + 1];
      e.inv1 = rcell[base + 1].y;
    } else if (base == nr - 2) {
      // the last cell's bins (and, by the index clamp, every radius beyond
      // them) switch to the all-zero shell nr - 1 above r_vac: vacuum
      e.split = r_vac_split;
      e.inv1 = 0.f;
    }
    lut[b] = e;
  }

  RT_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  rt_grid* g = new rt_grid;
  g->device = ctx->device;
  g->n_r = nr; g->n_t = nt; g->n_p = np;
  const long ncell = (long)(nr - 1) * (nt - 1) * np;
  const size_t esz = d->dtype == RT_F64 ? 8 : 4;
  void* tmp_ne = nullptr;
  void* tmp_te = nullptr;
  unsigned int* d_bad = nullptr;
  unsigned int h_bad = 0;
  double* d_shell = nullptr;
  g->shell_ne.assign(nr, 0.0);
  g->r.assign(R, R + nr);
  auto cleanup = [&](bool keep) {
    if (d->on_device == 0) {
      cudaFree(tmp_ne);
      cudaFree(tmp_te);
    }
    cudaFree(d_bad);
    cudaFree(d_shell);
    if (!keep) {
      cudaFree(g->ne); cudaFree(g->te); cudaFree(g->lut); cudaFree(g->rcell);
      delete g;
    }
  };
  cudaError_t e = cudaSuccess;
  const long nshell = (long)(nt - 1) * np;  // cells of one radial shell
  if (e == cudaSuccess) e = cudaMalloc(&g->ne, sizeof(float4) * 2 * (ncell + nshell));
  if (e == cudaSuccess) e = cudaMalloc(&g->te, sizeof(float4) * 2 * (ncell + nshell));
  if (e == cudaSuccess) e = cudaMalloc(&g->lut, sizeof(RadBin) * nb);
  if (e == cudaSuccess) e = cudaMalloc(&g->rcell, sizeof(float2) * (nr - 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&d_shell, sizeof(double) * nr);
  if (e == cudaSuccess && d->on_device == 0) {
    e = cudaMalloc(&tmp_ne, esz * nodes);
    if (e == cudaSuccess) e = cudaMalloc(&tmp_te, esz * nodes);
  }
  if (e != cudaSuccess) {
    cleanup(false);
    return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_load_grid: %s", cudaGetErrorString(e));
  }
  const void* src_ne = ne;
  const void* src_te = te;
  if (d->on_device == 0) {
    e = cudaMemcpyAsync(tmp_ne, ne, esz * nodes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp_te, te, esz * nodes, cudaMemcpyHostToDevice, s);
    src_ne = tmp_ne;
    src_te = tmp_te;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->lut, lut.data(), sizeof(RadBin) * nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->rcell, rcell.data(), sizeof(float2) * (nr - 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned int), s);
  // the vacuum shell (cells nr - 1): all corners zero
  if (e == cudaSuccess) e = cudaMemsetAsync(g->ne + 2 * ncell, 0, sizeof(float4) * 2 * nshell, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->te + 2 * ncell, 0, sizeof(float4) * 2 * nshell, s);
  const int blocks = ctx->sm_count * 8;
  if (e == cudaSuccess) {
    if (d->dtype == RT_F64) {
      check_values<double><<<blocks, 256, 0, s>>>((const double*)src_ne, (const double*)src_te, nodes, d_bad);
      pack_cells<double><<<blocks, 256, 0, s>>>((const double*)src_ne, (const double*)src_te, g->ne, g->te, nr, nt, np);
      shell_mean<double><<<nr, 256, 0, s>>>((const double*)src_ne, nt * np, d_shell);
    } else {
      check_values<float><<<blocks, 256, 0, s>>>((const float*)src_ne, (const float*)src_te, nodes, d_bad);
      pack_cells<float><<<blocks, 256, 0, s>>>((const float*)src_ne, (const float*)src_te, g->ne, g->te, nr, nt, np);
      shell_mean<float><<<nr, 256, 0, s>>>((const float*)src_ne, nt * np, d_shell);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof h_bad, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->shell_ne.data(), d_shell, sizeof(double) * nr, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup(false);
    return fail(RT_ERR_CUDA, "rt_load_grid: %s", cudaGetErrorString(e));
  }
  if (h_bad) {
    cleanup(false);
    return fail(RT_ERR_GRID, "rt_load_grid: %s%s", (h_bad & 1) ? "n_e must be finite and >= 0; " : "",
                (h_bad & 2) ? "T_e must be finite and > 0" : "");
  }
  cleanup(true);

  GridDev& G = g->dev;
  G.ne = g->ne;
  G.te = g->te;
  G.r_bins = g->lut;
  G.r_cell = g->rcell;
  G.n_r = nr; G.n_t = nt; G.n_p = np;
  G.r_lut_n = nb;
  G.r_lut_inv = (float)(nb / span);
  G.r_min = Rf[0];
  G.r_max = Rf[nr - 1];
  G.r_vac = r_vac_f;
  G.t0 = (float)T[0];
  G.t_inv = (float)(1.0 / dth);
  G.t_last = (float)(nt - 1);
  G.p0 = (float)Ph[0];
  G.p_inv = (float)(np / (2.0 * kPi));
  *out = g;
  return RT_OK;
}

rt_status rt_free_grid(rt_ctx* ctx, rt_grid* g) {
  if (!ctx || !g) return fail(RT_ERR_ARG, "rt_free_grid: NULL argument");
  cudaSetDevice(ctx->device);
  cudaFree(g->ne);
  cudaFree(g->te);
  cudaFree(g->lut);
  cudaFree(g->rcell);
  delete g;
  return RT_OK;
}

static rt_status check_options(const rt_options* o, int* nb_out) {
  if (!o) return fail(RT_ERR_ARG, "options are NULL");
  if (!(o->dtau > 0.0) || !std::isfinite(o->dtau)) return fail(RT_ERR_ARG, "dtau must be > 0");
  if (o->s_mode != RT_STEPWISE && o->s_mode != RT_TUBE && o->s_mode != RT_MAG_OFF)
    return fail(RT_ERR_ARG, "s_mode %d", o->s_mode);
  if (o->n_nb != 2 && o->n_nb != 4 && o->n_nb != 8) return fail(RT_ERR_ARG, "n_nb must be 2, 4 or 8");
  if (o->eps_mode == 0 && !(o->eta > 0.0)) return fail(RT_ERR_ARG, "eta must be > 0");
  if (o->eps_mode == 1 && !(o->delta > 0.0)) return fail(RT_ERR_ARG, "delta must be > 0");
  if (o->eps_mode != 0 && o->eps_mode != 1) return fail(RT_ERR_ARG, "eps_mode %d", o->eps_mode);
  if (o->precision != RT_PLAIN_F32 && o->precision != RT_MIXED) return fail(RT_ERR_ARG, "precision %d", o->precision);
  if (o->tbc_mode != 0 && o->tbc_mode != 1) return fail(RT_ERR_ARG, "tbc_mode %d", o->tbc_mode);
  if (o->tile != 0 && (o->tile < 2 || o->tile > 32)) return fail(RT_ERR_ARG, "tile %d (0 or 2..32)", o->tile);
  if (o->blocks_per_sm < 0) return fail(RT_ERR_ARG, "blocks_per_sm %d", o->blocks_per_sm);
  if (o->s_mode == RT_TUBE && !(o->delta > 0.0)) return fail(RT_ERR_ARG, "tube mode needs delta > 0");
  *nb_out = (o->straight || o->s_mode == RT_MAG_OFF) ? 0 : o->n_nb;
  return RT_OK;
}

static rt_status check_view(const rt_view* v) {
  if (!v) return fail(RT_ERR_ARG, "view is NULL");
  if (v->nx < 1 || v->ny < 1) return fail(RT_ERR_ARG, "image size %d x %d", v->nx, v->ny);
  if ((long)v->nx * v->ny > (1L << 30)) return fail(RT_ERR_ARG, "image too large");
  if (!std::isfinite(v->lon_rad) || !std::isfinite(v->lat_rad) || !std::isfinite(v->x0) || !std::isfinite(v->x1) ||
      !std::isfinite(v->y0) || !std::isfinite(v->y1))
    return fail(RT_ERR_ARG, "view has non-finite fields");
  return RT_OK;
}

}  // extern "C"

namespace {

ViewDev make_view(const rt_view& v) {
  ViewDev V;
  const double cl = std::cos(v.lon_rad), sl = std::sin(v.lon_rad), cb = std::cos(v.lat_rad), sb = std::sin(v.lat_rad);
  V.ox = (float)(cb * cl); V.oy = (float)(cb * sl); V.oz = (float)sb;
  V.eux = (float)(-sl); V.euy = (float)cl; V.euz = 0.f;
  V.evx = (float)(-sb * cl); V.evy = (float)(-sb * sl); V.evz = (float)cb;
  V.x0 = (float)v.x0; V.dx = (float)((v.x1 - v.x0) / v.nx);
  V.y0 = (float)v.y0; V.dy = (float)((v.y1 - v.y0) / v.ny);
  V.nx = v.nx;
  V.ny = v.ny;
  V.npix = v.nx * v.ny;
  V.tile = 0;
  V.tiles_x = 0;
  V.tickets = V.npix;
  return V;
}

void set_tiles(ViewDev& V, int tile) {
  if (tile <= 0) return;
  V.tile = tile;
  V.tiles_x = (V.nx + tile - 1) / tile;
  V.tickets = V.tiles_x * ((V.ny + tile - 1) / tile) * tile * tile;
}

FreqDev make_freq(double f, int slab) {
  const double cpe = c_pe();
  FreqDev F;
  F.kf = (float)(-cpe / (2.0 * f * f));
  F.kn2 = (float)(-cpe / (f * f));
  F.kap_c = (float)(9.78e-3 / (f * f));
  F.ln_f = (float)std::log(f);
  F.out_slab = slab;
  return F;
}

void fill_common(TraceParams& P, const rt_grid* g, const rt_options* o) {
  P.G = g->dev;
  const double h = o->dtau;
  P.h = (float)h;
  P.h2_6 = (float)(h * h / 6.0);
  P.h_6 = (float)(h / 6.0);
  P.h2_12 = (float)(h * h / 12.0);
  P.hrsun = (float)(h * kRsunCm);
  P.eta = (float)o->eta;
  P.eps_fixed = o->eps_mode == 1 ? (float)o->delta : 0.f;
  P.tau_stop = (float)o->tau_stop;
  P.max_steps = o->max_steps > 0 ? o->max_steps : (int)std::ceil(40.0 * g->dev.r_max / h);
  P.tbc_mode = o->tbc_mode;
  P.tbc_K = (float)o->tbc_K;
  P.emission = o->emission;
  P.straight = o->straight;
  P.blocks_per_sm = o->blocks_per_sm;
  P.tube_delta = (float)o->delta;
  P.inv_delta2 = (float)(1.0 / (o->delta * o->delta));
}

bool bad_freq(double f) { return !(f > 0.0) || !std::isfinite(f); }

bool is_tube(const rt_options* o) { return o->s_mode == RT_TUBE && !o->straight; }

// Estimated RK4 steps of a ray with impact parameter b (in units of h):
// the entry chord, cut at the turning radius r_c where the shell-mean
// plasma frequency equals f, or at the inner sphere.
double path_estimate(double b, double rc, double rmin, double rmax) {
  if (b >= rmax) return 1.0;
  const double out = std::sqrt(rmax * rmax - b * b);
  const double stop = std::max(rc, rmin);
  if (b >= stop) return 2.0 * out;
  const double in = std::sqrt(stop * stop - b * b);
  return (rc > rmin) ? 2.0 * (out - in) : out - in;
}

double turning_radius(const rt_grid* g, double f) {
  const double nc = f * f / c_pe();
  for (int i = g->n_r - 1; i >= 0; --i)
    if (g->shell_ne[i] >= nc) return g->r[i];
  return 0.0;
}

struct ChunkCand {
  double cost;  // estimated steps of the chunk's rays (every 8th pixel sampled)
  ChunkDev c;
};

// The maps (one per frequency) and 64-pixel chunks of one image request, as
// view q of a work table; chunk costs from path_estimate.
void request_chunks(const rt_grid* g, const rt_view& V, const double* freqs, int nf, int q, float* tb_out,
                    rt_ray_diag* diag, std::vector<MapDev>& maps, std::vector<ChunkCand>& cands) {
  const double rmin = g->r.front(), rmax = g->r.back();
  const int npix = V.nx * V.ny;
  const double du = (V.x1 - V.x0) / V.nx, dv = (V.y1 - V.y0) / V.ny;
  for (int fi = 0; fi < nf; ++fi) {
    MapDev M;
    M.f = make_freq(freqs[fi], fi);
    M.view = q;
    M.out = tb_out + (size_t)fi * npix;
    M.diag = diag ? reinterpret_cast<RayDiag*>(diag) + (size_t)fi * npix : nullptr;
    const int m = (int)maps.size();
    maps.push_back(M);
    const double rc = turning_radius(g, freqs[fi]);
    for (int p0 = 0; p0 < npix; p0 += kChunk) {
      const int cnt = std::min(kChunk, npix - p0);
      double cost = 0.0;
      for (int k = 0; k < cnt; k += 8) {
        const int pix = p0 + k, ix = pix % V.nx, iy = pix / V.nx;
        const double u = V.x0 + (ix + 0.5) * du, v = V.y0 + (iy + 0.5) * dv;
        cost += path_estimate(std::sqrt(u * u + v * v), rc, rmin, rmax);
      }
      cands.push_back({cost, ChunkDev{m, p0, cnt, 0}});
    }
  }
}

void sort_longest_first(std::vector<ChunkCand>& cands) {
  std::stable_sort(cands.begin(), cands.end(), [](const ChunkCand& a, const ChunkCand& b) { return a.cost > b.cost; });
}


}  // namespace

extern "C" {

rt_status rt_trace_image(rt_ctx* ctx, const rt_grid* g, const rt_view* v, const double* freqs, int nf,
                         const rt_options* o, float* tb_out, rt_ray_diag* diag, void* stream) {
  if (!ctx || !g || !freqs || !tb_out) return fail(RT_ERR_ARG, "rt_trace_image: NULL argument");
  rt_status st = check_view(v);
  if (st != RT_OK) return st;
  int nb = 0;
  st = check_options(o, &nb);
  if (st != RT_OK) return st;
  if (nf < 1 || nf > kMaxFreq) return fail(RT_ERR_ARG, "rt_trace_image: nf = %d (1..%d)", nf, kMaxFreq);
  for (int i = 0; i < nf; ++i)
    if (bad_freq(freqs[i])) return fail(RT_ERR_ARG, "frequency %d is not > 0", i);
  const long total = (long)nf * v->nx * v->ny;
  if (total >= (1L << 31)) return fail(RT_ERR_ARG, "rt_trace_image: too many rays");

  TraceParams P;
  std::memset(&P, 0, sizeof P);
  fill_common(P, g, o);
  P.view = make_view(*v);
  set_tiles(P.view, o->tile);
  if ((long)nf * P.view.tickets >= (1L << 31)) return fail(RT_ERR_ARG, "rt_trace_image: too many rays");
  P.nf = nf;
  // lowest frequencies first: their rays turn high and tend to be longest
  std::vector<int> order(nf);
  for (int i = 0; i < nf; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return freqs[a] < freqs[b]; });
  for (int i = 0; i < nf; ++i) P.freq[i] = make_freq(freqs[order[i]], order[i]);
  P.tb_out = tb_out;
  P.diag = reinterpret_cast<RayDiag*>(diag);
  P.counter = ctx->d_counter;
  P.stats = ctx->d_stats;
  P.total = (unsigned int)((long)nf * P.view.tickets);

  RT_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void* d_tables = nullptr;
  if (o->tile <= 0) {
    // row order: the 64-pixel chunks of all frequencies, longest first (the
    // batch plans' order; a ray's arithmetic does not depend on it), through
    // a work table uploaded from the context's pinned staging
    std::vector<MapDev> maps;
    std::vector<ChunkCand> cands;
    request_chunks(g, *v, freqs, nf, 0, tb_out, diag, maps, cands);
    sort_longest_first(cands);
    const size_t off_maps = (sizeof(ViewDev) + 15) / 16 * 16;
    const size_t off_chunks = off_maps + (sizeof(MapDev) * maps.size() + 15) / 16 * 16;
    const size_t bytes = off_chunks + sizeof(ChunkDev) * cands.size();
    std::lock_guard<std::mutex> lock(ctx->stage_mu);
    cudaError_t e = cudaSuccess;
    if (ctx->stage_pending) e = cudaEventSynchronize(ctx->stage_done);  // the previous copy has left the buffer
    ctx->stage_pending = false;
    if (e == cudaSuccess && ctx->stage_bytes < bytes) {
      cudaFreeHost(ctx->stage);
      ctx->stage = nullptr;
      ctx->stage_bytes = 0;
      e = cudaMallocHost(&ctx->stage, bytes);
      if (e == cudaSuccess) ctx->stage_bytes = bytes;
    }
    if (e == cudaSuccess && !ctx->stage_done) e = cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_trace_image: %s", cudaGetErrorString(e));
    char* h = static_cast<char*>(ctx->stage);
    const ViewDev vd = make_view(*v);
    std::memcpy(h, &vd, sizeof vd);
    std::memcpy(h + off_maps, maps.data(), sizeof(MapDev) * maps.size());
    for (size_t i = 0; i < cands.size(); ++i) std::memcpy(h + off_chunks + i * sizeof(ChunkDev), &cands[i].c, sizeof(ChunkDev));
    e = cudaMallocAsync(&d_tables, bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tables, h, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->stage_done, s);
    if (e != cudaSuccess) {
      if (d_tables) cudaFreeAsync(d_tables, s);
      return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_trace_image: %s",
                  cudaGetErrorString(e));
    }
    ctx->stage_pending = true;
    char* d = static_cast<char*>(d_tables);
    P.views = reinterpret_cast<const ViewDev*>(d);
    P.maps = reinterpret_cast<const MapDev*>(d + off_maps);
    P.chunks = reinterpret_cast<const ChunkDev*>(d + off_chunks);
    P.total = (unsigned int)(cands.size() * kChunk);
  }
  cudaError_t e = cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_stats, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = dispatch_trace(nb, o->precision == RT_MIXED, P, ctx->sm_count, s, is_tube(o));
  if (d_tables) {
    const cudaError_t e2 = cudaFreeAsync(d_tables, s);  // stream-ordered: after the kernel
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_trace_image: %s", cudaGetErrorString(e));
  return RT_OK;
}

rt_status rt_batch_plan_destroy(rt_batch_plan* p) {
  if (!p) return fail(RT_ERR_ARG, "rt_batch_plan_destroy: NULL plan");
  if (p->ctx) cudaSetDevice(p->ctx->device);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaFree(p->chunks);
  cudaFree(p->maps);
  cudaFree(p->views);
  cudaFree(p->counter);
  cudaFree(p->stats);
  delete p;
  return RT_OK;
}

rt_status rt_shard_assign(const double* cost, long n, int world_size, int* rank_of) {
  if (n < 0 || (n > 0 && (!cost || !rank_of))) return fail(RT_ERR_ARG, "rt_shard_assign: bad arguments");
  if (world_size < 1) return fail(RT_ERR_ARG, "rt_shard_assign: world_size = %d", world_size);
  std::vector<long> order((size_t)n);
  for (long i = 0; i < n; ++i) {
    if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return fail(RT_ERR_ARG, "rt_shard_assign: cost %ld", i);
    order[(size_t)i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](long a, long b) { return cost[a] > cost[b]; });
  std::vector<double> load((size_t)world_size, 0.0);
  for (long i : order) {
    int best = 0;
    for (int r = 1; r < world_size; ++r)
      if (load[(size_t)r] < load[(size_t)best]) best = r;
    rank_of[i] = best;
    load[(size_t)best] += cost[i];
  }
  return RT_OK;
}

static rt_status plan_create(rt_ctx* ctx, const rt_grid* g, const rt_request* reqs, int nreq, const rt_options* o,
                             int rank, int world_size, rt_batch_plan** out) {
  if (!ctx || !g || !reqs || !out) return fail(RT_ERR_ARG, "rt_batch_plan_create: NULL argument");
  *out = nullptr;
  if (nreq < 1) return fail(RT_ERR_ARG, "rt_batch_plan_create: nreq = %d", nreq);
  if (world_size < 1 || rank < 0 || rank >= world_size)
    return fail(RT_ERR_ARG, "rt_batch_plan_create: rank %d of %d", rank, world_size);
  int nb = 0;
  rt_status st = check_options(o, &nb);
  if (st != RT_OK) return st;
  std::vector<ViewDev> views;
  std::vector<MapDev> maps;
  std::vector<ChunkCand> cands;
  for (int q = 0; q < nreq; ++q) {
    const rt_request& R = reqs[q];
    if (!R.view || !R.freqs_hz || !R.tb_out || R.nf < 1) return fail(RT_ERR_ARG, "request %d: NULL field or nf < 1", q);
    st = check_view(R.view);
    if (st != RT_OK) return st;
    for (int fi = 0; fi < R.nf; ++fi)
      if (bad_freq(R.freqs_hz[fi])) return fail(RT_ERR_ARG, "request %d frequency %d is not > 0", q, fi);
    views.push_back(make_view(*R.view));
    request_chunks(g, *R.view, R.freqs_hz, R.nf, q, R.tb_out, R.diag, maps, cands);
  }
  if ((double)cands.size() * kChunk >= 4.0e9) return fail(RT_ERR_ARG, "rt_batch_plan_create: too many rays");
  sort_longest_first(cands);
  std::vector<ChunkDev> chunks;
  if (world_size == 1) {
    chunks.resize(cands.size());
    for (size_t i = 0; i < cands.size(); ++i) chunks[i] = cands[i].c;
  } else {  // this rank's share of the longest-first greedy partition (same on every rank)
    std::vector<double> cost(cands.size());
    std::vector<int> owner(cands.size());
    for (size_t i = 0; i < cands.size(); ++i) cost[i] = cands[i].cost;
    st = rt_shard_assign(cost.data(), (long)cands.size(), world_size, owner.data());
    if (st != RT_OK) return st;
    for (size_t i = 0; i < cands.size(); ++i)
      if (owner[i] == rank) chunks.push_back(cands[i].c);
  }
  const size_t n_alloc = std::max<size_t>(chunks.size(), 1);

  RT_CUDA(cudaSetDevice(ctx->device));
  rt_batch_plan* p = new rt_batch_plan;
  p->ctx = ctx;
  cudaError_t e = cudaMalloc(&p->chunks, sizeof(ChunkDev) * n_alloc);
  if (e == cudaSuccess) e = cudaMalloc(&p->maps, sizeof(MapDev) * maps.size());
  if (e == cudaSuccess) e = cudaMalloc(&p->views, sizeof(ViewDev) * views.size());
  if (e == cudaSuccess) e = cudaMalloc(&p->counter, 64);
  if (e == cudaSuccess) e = cudaMalloc(&p->stats, 64);
  if (e == cudaSuccess) e = cudaMemcpy(p->chunks, chunks.data(), sizeof(ChunkDev) * chunks.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->maps, maps.data(), sizeof(MapDev) * maps.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->views, views.data(), sizeof(ViewDev) * views.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  fill_common(P, g, o);
  P.chunks = p->chunks;
  P.maps = p->maps;
  P.views = p->views;
  P.counter = p->counter;
  P.stats = p->stats;
  P.total = (unsigned int)(chunks.size() * kChunk);
  // capture {reset ticket and counters, persistent kernel} once; replay per launch
  if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(p->counter, 0, sizeof(unsigned int), p->cap);
    cudaError_t e2 = cudaMemsetAsync(p->stats, 0, 2 * sizeof(unsigned long long), p->cap);
    cudaError_t e3 = dispatch_trace(nb, o->precision == RT_MIXED, P, ctx->sm_count, p->cap, is_tube(o));
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (e == cudaSuccess) e = (e1 != cudaSuccess) ? e1 : (e2 != cudaSuccess) ? e2 : e3;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (e != cudaSuccess) {
    rt_batch_plan_destroy(p);
    return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_batch_plan_create: %s",
                cudaGetErrorString(e));
  }
  *out = p;
  return RT_OK;
}

rt_status rt_batch_plan_create(rt_ctx* ctx, const rt_grid* g, const rt_request* reqs, int nreq,
                               const rt_options* o, rt_batch_plan** out) {
  return plan_create(ctx, g, reqs, nreq, o, 0, 1, out);
}

rt_status rt_batch_plan_create_shard(rt_ctx* ctx, const rt_grid* g, const rt_request* reqs, int nreq,
                                     const rt_options* o, int rank, int world_size, rt_batch_plan** out) {
  return plan_create(ctx, g, reqs, nreq, o, rank, world_size, out);
}

rt_status rt_batch_plan_launch(rt_batch_plan* p, void* stream) {
  if (!p) return fail(RT_ERR_ARG, "rt_batch_plan_launch: NULL plan");
  RT_CUDA(cudaSetDevice(p->ctx->device));
  RT_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  return RT_OK;
}

rt_status rt_batch_plan_stats(rt_batch_plan* p, void* stream, rt_stats* out) {
  if (!p || !out) return fail(RT_ERR_ARG, "rt_batch_plan_stats: NULL argument");
  RT_CUDA(cudaSetDevice(p->ctx->device));
  unsigned long long h[2] = {0, 0};
  RT_CUDA(cudaMemcpyAsync(h, p->stats, sizeof h, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  RT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  out->ray_steps = h[0];
  out->rays = h[1];
  return RT_OK;
}

rt_status rt_trace_batch(rt_ctx* ctx, const rt_grid* g, const rt_request* reqs, int nreq, const rt_options* o,
                         void* stream) {
  rt_batch_plan* p = nullptr;
  rt_status st = rt_batch_plan_create(ctx, g, reqs, nreq, o, &p);
  if (st != RT_OK) return st;
  st = rt_batch_plan_launch(p, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  rt_batch_plan_destroy(p);
  if (st != RT_OK) return st;
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_trace_batch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // extern "C"

namespace {

// Checks shared by the adjoint's entry points; nb_out: the neighbour count.
rt_status check_backward(const rt_view* v, const double* freqs, int nf, const rt_options* o, int* nb_out,
                         const char* who) {
  rt_status st = check_view(v);
  if (st != RT_OK) return st;
  st = check_options(o, nb_out);
  if (st != RT_OK) return st;
  if (o->straight || o->s_mode == RT_TUBE || !(*nb_out == 0 || *nb_out == 4))
    return fail(RT_ERR_UNSUPPORTED, "%s: supports step-wise magnification with 4 neighbours or none", who);
  if (nf < 1 || nf > kMaxFreq) return fail(RT_ERR_ARG, "%s: nf = %d (1..%d)", who, nf, kMaxFreq);
  for (int i = 0; i < nf; ++i)
    if (bad_freq(freqs[i])) return fail(RT_ERR_ARG, "frequency %d is not > 0", i);
  if ((long)nf * v->nx * v->ny >= (1L << 31)) return fail(RT_ERR_ARG, "%s: too many rays", who);
  return RT_OK;
}

// The forward parameters of the adjoint's passes: image mode without a tile
// walk (ticket t = frequency in ascending order, then pixel).
void backward_params(rt_ctx* ctx, const rt_grid* g, const rt_view* v, const double* freqs, int nf,
                     const rt_options* o, float* tb, RayDiag* diag, TraceParams& P, std::vector<int>& order) {
  std::memset(&P, 0, sizeof P);
  fill_common(P, g, o);
  P.view = make_view(*v);
  P.nf = nf;
  order.resize(nf);
  for (int i = 0; i < nf; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return freqs[a] < freqs[b]; });
  for (int i = 0; i < nf; ++i) P.freq[i] = make_freq(freqs[order[i]], order[i]);
  P.tb_out = tb;
  P.diag = diag;
  P.counter = ctx->d_counter;
  P.stats = ctx->d_stats;
  P.total = (unsigned int)((long)nf * v->nx * v->ny);
}

// Zeroes the gradients and launches the reverse sweep over the checkpoints
// (ck_off, or a tape's ck_prev / ck_last chains).
cudaError_t launch_adjoint(rt_ctx* ctx, const rt_grid* g, const TraceParams& P, int nb, bool mixed,
                           const RayDiag* diag, const float* dL_dTb, float* dL_dne, float* dL_dte, const Ckpt* ckpt,
                           const unsigned long long* ck_off, const int* ck_prev, const int* ck_last,
                           unsigned long long* mismatch, cudaStream_t s) {
  const size_t nodes = (size_t)g->n_r * g->n_t * g->n_p;
  cudaError_t e = cudaMemsetAsync(dL_dne, 0, sizeof(float) * nodes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dL_dte, 0, sizeof(float) * nodes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(mismatch, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  AdjParams A;
  std::memset(&A, 0, sizeof A);
  A.G = g->dev;
  A.h = P.h; A.h2_6 = P.h2_6; A.h_6 = P.h_6; A.h2_12 = P.h2_12; A.hrsun = P.hrsun;
  A.eta = P.eta; A.eps_fixed = P.eps_fixed; A.tbc_K = P.tbc_K; A.tbc_mode = P.tbc_mode; A.emission = P.emission;
  A.view = P.view;
  A.nf = P.nf;
  for (int i = 0; i < P.nf; ++i) A.freq[i] = P.freq[i];
  A.diag = diag;
  A.dL_dTb = dL_dTb;
  A.ckpt = ckpt;
  A.ck_off = ck_off;
  A.ck_prev = ck_prev;
  A.ck_last = ck_last;
  A.dne = dL_dne;
  A.dte = dL_dte;
  A.counter = ctx->d_counter;
  A.total = P.total;
  A.mismatch = mismatch;
  const int per_sm = (nb == 0) ? (mixed ? adj_blocks_per_sm<0, true>() : adj_blocks_per_sm<0, false>())
                               : (mixed ? adj_blocks_per_sm<4, true>() : adj_blocks_per_sm<4, false>());
  const int grid_blocks = ctx->sm_count * per_sm;
  if (nb == 0) {
    if (mixed) adjoint_rays<0, true><<<grid_blocks, kThreads, 0, s>>>(A);
    else adjoint_rays<0, false><<<grid_blocks, kThreads, 0, s>>>(A);
  } else {
    if (mixed) adjoint_rays<4, true><<<grid_blocks, kThreads, 0, s>>>(A);
    else adjoint_rays<4, false><<<grid_blocks, kThreads, 0, s>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

rt_status rt_backward(rt_ctx* ctx, const rt_grid* g, const rt_view* v, const double* freqs, int nf, const rt_options* o,
                      const float* dL_dTb, float* dL_dne, float* dL_dte, float* tb_out, const rt_ray_diag* fwd_diag,
                      void* stream) {
  if (!ctx || !g || !freqs || !dL_dTb || !dL_dne || !dL_dte) return fail(RT_ERR_ARG, "rt_backward: NULL argument");
  int nb = 0;
  rt_status st = check_backward(v, freqs, nf, o, &nb, "rt_backward");
  if (st != RT_OK) return st;
  const long npix = (long)v->nx * v->ny;
  const long total = (long)nf * npix;
  const bool mixed = o->precision == RT_MIXED;
  RT_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;

  // scratch
  float* tb = nullptr;
  RayDiag* diag = nullptr;
  unsigned long long* ck_off = nullptr;
  Ckpt* ckpt = nullptr;
  auto release = [&]() {
    cudaFree(diag);
    cudaFree(ck_off);
    cudaFree(ckpt);
    if (!tb_out) cudaFree(tb);
  };
  cudaError_t e = cudaMalloc(&diag, sizeof(RayDiag) * total);
  if (e == cudaSuccess && !tb_out) e = cudaMalloc(&tb, sizeof(float) * total);
  // checkpoint offsets [total + 1] and, behind them, the adjoint's mismatch flag
  if (e == cudaSuccess) e = cudaMalloc(&ck_off, sizeof(unsigned long long) * (total + 2));
  if (e != cudaSuccess) {
    release();
    return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_backward: %s", cudaGetErrorString(e));
  }
  if (tb_out) tb = tb_out;

  // phase 0: forward with per-ray step counts
  TraceParams P;
  std::vector<int> order;
  backward_params(ctx, g, v, freqs, nf, o, tb, diag, P, order);
  P.skip_zero = dL_dTb;
  auto run_forward = [&]() -> cudaError_t {
    cudaError_t r = cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int), s);
    if (r == cudaSuccess) r = cudaMemsetAsync(ctx->d_stats, 0, 2 * sizeof(unsigned long long), s);
    if (r == cudaSuccess) r = dispatch_trace(nb, mixed, P, ctx->sm_count, s);
    return r;
  };
  std::vector<RayDiag> hd(total);
  if (fwd_diag) {  // the caller's forward already counted the steps
    static_assert(sizeof(RayDiag) == sizeof(rt_ray_diag), "rt_ray_diag layout");
    e = cudaMemcpyAsync(hd.data(), fwd_diag, sizeof(RayDiag) * total, cudaMemcpyDeviceToHost, s);
  } else {
    e = run_forward();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), diag, sizeof(RayDiag) * total, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return fail(RT_ERR_CUDA, "rt_backward (forward): %s", cudaGetErrorString(e));
  }
  // checkpoint offsets, indexed by ticket (frequency in processing order,
  // pixel); a ray with dL/dT_b = 0 is not traced again and holds none
  std::vector<float> hw(total);
  e = cudaMemcpyAsync(hw.data(), dL_dTb, sizeof(float) * total, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return fail(RT_ERR_CUDA, "rt_backward (weights): %s", cudaGetErrorString(e));
  }
  std::vector<unsigned long long> off(total + 1, 0);
  for (long t = 0; t < total; ++t) {
    const long fi = t / npix, pix = t - fi * npix;
    const size_t o = (size_t)order[fi] * npix + pix;
    const RayDiag& d = hd[o];
    const unsigned long long cnt =
        (d.steps > 0 && hw[o] != 0.f) ? (unsigned long long)((d.steps - 1) / kCkptEvery + 1) : 0ull;
    off[t + 1] = off[t] + cnt;
  }
  e = cudaMalloc(&ckpt, sizeof(Ckpt) * std::max<unsigned long long>(off[total], 1ull));
  if (e == cudaSuccess) e = cudaMemcpyAsync(ck_off, off.data(), sizeof(unsigned long long) * (total + 1),
                                            cudaMemcpyHostToDevice, s);
  // phase 1: the same forward again, storing checkpoints
  P.ckpt = ckpt;
  P.ck_off = ck_off;
  if (e == cudaSuccess) e = run_forward();
  // phase 2: reverse sweep
  if (e == cudaSuccess)
    e = launch_adjoint(ctx, g, P, nb, mixed, diag, dL_dTb, dL_dne, dL_dte, ckpt, ck_off, nullptr, nullptr,
                       ck_off + total + 1, s);
  unsigned long long mismatch = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&mismatch, ck_off + total + 1, sizeof mismatch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_backward: %s", cudaGetErrorString(e));
  if (mismatch)
    return fail(RT_ERR_ARG, "rt_backward: fwd_diag does not match this forward (%llu rays with other step counts)",
                mismatch);
  return RT_OK;
}

rt_status rt_tape_free(rt_tape* t) {
  if (!t) return fail(RT_ERR_ARG, "rt_tape_free: NULL tape");
  if (t->ctx) cudaSetDevice(t->ctx->device);
  cudaFree(t->pool);
  cudaFree(t->prev);
  cudaFree(t->last);
  cudaFree(t->counter);
  if (t->own_diag) cudaFree(t->diag);
  delete t;
  return RT_OK;
}

rt_status rt_trace_image_tape(rt_ctx* ctx, const rt_grid* g, const rt_view* v, const double* freqs, int nf,
                              const rt_options* o, size_t pool_bytes, float* tb_out, rt_ray_diag* diag, rt_tape** out,
                              void* stream) {
  if (!ctx || !g || !freqs || !tb_out || !out) return fail(RT_ERR_ARG, "rt_trace_image_tape: NULL argument");
  *out = nullptr;
  int nb = 0;
  rt_status st = check_backward(v, freqs, nf, o, &nb, "rt_trace_image_tape");
  if (st != RT_OK) return st;
  const long npix = (long)v->nx * v->ny;
  const long total = (long)nf * npix;
  // pool: the given bytes, or 1.5 x the estimated checkpoints (the entry chord
  // cut at the turning radius, in steps of h, one checkpoint per kCkptEvery)
  unsigned long long cap = pool_bytes / (sizeof(Ckpt) + sizeof(int));
  if (pool_bytes == 0) {
    const double rmin = g->r.front(), rmax = g->r.back(), h = o->dtau;
    const double du = (v->x1 - v->x0) / v->nx, dv = (v->y1 - v->y0) / v->ny;
    double est = 0.0;
    for (int fi = 0; fi < nf; ++fi) {
      const double rc = turning_radius(g, freqs[fi]);
      for (int iy = 0; iy < v->ny; ++iy)
        for (int ix = 0; ix < v->nx; ++ix) {
          const double u = v->x0 + (ix + 0.5) * du, w = v->y0 + (iy + 0.5) * dv;
          est += path_estimate(std::sqrt(u * u + w * w), rc, rmin, rmax) / h / kCkptEvery + 1.0;
        }
    }
    cap = (unsigned long long)(1.5 * est) + 1024;
  }
  cap = std::min<unsigned long long>(std::max<unsigned long long>(cap, 1), (unsigned long long)std::numeric_limits<int>::max());
  RT_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  rt_tape* t = new rt_tape;
  t->ctx = ctx;
  t->g = g;
  t->view = *v;
  t->freqs.assign(freqs, freqs + nf);
  t->opt = *o;
  t->nb = nb;
  t->mixed = o->precision == RT_MIXED;
  t->cap = cap;
  t->total = total;
  cudaError_t e = cudaMalloc(&t->pool, sizeof(Ckpt) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&t->prev, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&t->last, sizeof(int) * total);
  if (e == cudaSuccess) e = cudaMalloc(&t->counter, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && !diag) {
    e = cudaMalloc(&t->diag, sizeof(RayDiag) * total);
    t->own_diag = true;
  } else if (diag) {
    t->diag = reinterpret_cast<RayDiag*>(diag);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(t->last, 0xff, sizeof(int) * total, s);  // -1: no checkpoint
  if (e == cudaSuccess) e = cudaMemsetAsync(t->counter, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) {
    rt_tape_free(t);
    return fail(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_trace_image_tape: %s",
                cudaGetErrorString(e));
  }
  std::vector<int> order;
  backward_params(ctx, g, v, freqs, nf, o, tb_out, t->diag, t->P, order);
  t->P.ckpt = t->pool;
  t->P.ck_prev = t->prev;
  t->P.ck_last = t->last;
  t->P.pool_counter = t->counter;
  t->P.pool_cap = cap;
  e = cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_stats, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = dispatch_trace(nb, t->mixed, t->P, ctx->sm_count, s);
  if (e != cudaSuccess) {
    rt_tape_free(t);
    return fail(RT_ERR_CUDA, "rt_trace_image_tape: %s", cudaGetErrorString(e));
  }
  *out = t;
  return RT_OK;
}

rt_status rt_tape_info(rt_tape* t, void* stream, unsigned long long* slots_used, unsigned long long* slots_cap) {
  if (!t || !slots_used || !slots_cap) return fail(RT_ERR_ARG, "rt_tape_info: NULL argument");
  RT_CUDA(cudaSetDevice(t->ctx->device));
  unsigned long long used = 0;
  RT_CUDA(cudaMemcpyAsync(&used, t->counter, sizeof used, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  RT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  *slots_used = used;
  *slots_cap = t->cap;
  return RT_OK;
}

rt_status rt_backward_tape(rt_tape* t, const float* dL_dTb, float* dL_dne, float* dL_dte, void* stream) {
  if (!t || !dL_dTb || !dL_dne || !dL_dte) return fail(RT_ERR_ARG, "rt_backward_tape: NULL argument");
  unsigned long long used = 0, cap = 0;
  rt_status st = rt_tape_info(t, stream, &used, &cap);
  if (st != RT_OK) return st;
  if (used > cap)  // the pool overflowed: trace again, as rt_backward does
    return rt_backward(t->ctx, t->g, &t->view, t->freqs.data(), (int)t->freqs.size(), &t->opt, dL_dTb, dL_dne,
                       dL_dte, nullptr, reinterpret_cast<const rt_ray_diag*>(t->diag), stream);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_adjoint(t->ctx, t->g, t->P, t->nb, t->mixed, t->diag, dL_dTb, dL_dne, dL_dte, t->pool,
                                 nullptr, t->prev, t->last, t->counter + 1, s);
  unsigned long long mismatch = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mismatch, t->counter + 1, sizeof mismatch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, "rt_backward_tape: %s", cudaGetErrorString(e));
  if (mismatch) return fail(RT_ERR_ARG, "rt_backward_tape: %llu rays without their checkpoints", mismatch);
  return RT_OK;
}

rt_status rt_trace_paths(rt_ctx* ctx, const rt_grid* g, const rt_view* v, double freq_hz, const int* pixels, int n,
                         const rt_options* o, int cap, rt_path_node* nodes, int* n_nodes, float* tb_out,
                         rt_ray_diag* diag, void* stream) {
  if (!ctx || !g || !pixels || !nodes || !n_nodes || !tb_out) return fail(RT_ERR_ARG, "rt_trace_paths: NULL argument");
  rt_status st = check_view(v);
  if (st != RT_OK) return st;
  int nb = 0;
  st = check_options(o, &nb);
  if (st != RT_OK) return st;
  if (is_tube(o)) return fail(RT_ERR_UNSUPPORTED, "rt_trace_paths: step-wise magnification or none");
  if (n < 1 || n > (1 << 20)) return fail(RT_ERR_ARG, "rt_trace_paths: n = %d (1..2^20)", n);
  if (cap < 1) return fail(RT_ERR_ARG, "rt_trace_paths: cap = %d", cap);
  if (bad_freq(freq_hz)) return fail(RT_ERR_ARG, "rt_trace_paths: frequency is not > 0");
  const long npix = (long)v->nx * v->ny;
  for (int i = 0; i < n; ++i)
    if (pixels[i] < 0 || pixels[i] >= npix) return fail(RT_ERR_ARG, "rt_trace_paths: pixel %d out of range", pixels[i]);
  static_assert(sizeof(PathNode) == sizeof(rt_path_node), "rt_path_node layout");
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  fill_common(P, g, o);
  P.view = make_view(*v);
  P.nf = 1;
  P.freq[0] = make_freq(freq_hz, 0);
  RT_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  int* d_pix = nullptr;
  RT_CUDA(cudaMallocAsync(&d_pix, sizeof(int) * n, s));
  cudaError_t e = cudaMemcpyAsync(d_pix, pixels, sizeof(int) * n, cudaMemcpyHostToDevice, s);
  PathNode* pn = reinterpret_cast<PathNode*>(nodes);
  RayDiag* dg = reinterpret_cast<RayDiag*>(diag);
  const int blocks = (n + 63) / 64;
  const bool mixed = o->precision == RT_MIXED;
  if (e == cudaSuccess) {
#define RT_PATHS(NB)                                                                          \
    (mixed ? trace_paths<NB, true><<<blocks, 64, 0, s>>>(P, d_pix, n, cap, pn, n_nodes, tb_out, dg) \
           : trace_paths<NB, false><<<blocks, 64, 0, s>>>(P, d_pix, n, cap, pn, n_nodes, tb_out, dg))
    switch (nb) {
      case 0: RT_PATHS(0); break;
      case 2: RT_PATHS(2); break;
      case 4: RT_PATHS(4); break;
      default: RT_PATHS(8); break;
    }
#undef RT_PATHS
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(d_pix, s);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(RT_ERR_CUDA, "rt_trace_paths: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  return RT_OK;
}

rt_status rt_beam_convolve(const rt_view* v, const float* tb, const double* freqs_hz, int nf, double baseline_m,
                           float* scratch, float* tb_out, void* stream) {
  if (!tb || !freqs_hz || !scratch || !tb_out) return fail(RT_ERR_ARG, "rt_beam_convolve: NULL argument");
  rt_status st = check_view(v);
  if (st != RT_OK) return st;
  if (nf < 1 || nf > kMaxFreq) return fail(RT_ERR_ARG, "rt_beam_convolve: nf = %d (1..%d)", nf, kMaxFreq);
  if (!(baseline_m > 0.0) || !std::isfinite(baseline_m)) return fail(RT_ERR_ARG, "rt_beam_convolve: baseline must be > 0");
  const double dx = std::fabs(v->x1 - v->x0) / v->nx, dy = std::fabs(v->y1 - v->y0) / v->ny;
  if (!(dx > 0.0) || std::fabs(dx - dy) > 1e-9 * dx)
    return fail(RT_ERR_ARG, "rt_beam_convolve: pixels must be square (dx = %g, dy = %g)", dx, dy);
  BeamParams B;
  std::memset(&B, 0, sizeof B);
  B.nx = v->nx;
  B.ny = v->ny;
  for (int i = 0; i < nf; ++i) {
    if (bad_freq(freqs_hz[i])) return fail(RT_ERR_ARG, "frequency %d is not > 0", i);
    const double fwhm = kSpeedOfLightCmS / freqs_hz[i] / (baseline_m * 100.0) * kAuRsun;  // R_sun
    const double sigma = fwhm / std::sqrt(8.0 * std::log(2.0)) / dx;                    // pixels
    const double hw = std::ceil(4.0 * sigma);
    if (hw > 1 << 20) return fail(RT_ERR_ARG, "rt_beam_convolve: beam of %g pixels is too wide", 2 * hw + 1);
    const float a = (float)(0.5 / (sigma * sigma));
    double sum = 0.0;
    for (int d = -(int)hw; d <= (int)hw; ++d) sum += std::exp(-(double)((float)(d * d) * a));
    B.half[i] = (int)hw;
    B.inv2s2[i] = a;
    B.norm[i] = (float)(1.0 / sum);
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = v->nx * v->ny;
  const dim3 grid((n + kBeamThreads - 1) / kBeamThreads, nf);
  beam_pass<<<grid, kBeamThreads, 0, s>>>(tb, scratch, B, 0);
  beam_pass<<<grid, kBeamThreads, 0, s>>>(scratch, tb_out, B, 1);
  RT_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_disk_mean_tb(const rt_view* v, const float* tb, int nf, double radius, double* mean_out, void* stream) {
  if (!tb || !mean_out) return fail(RT_ERR_ARG, "rt_disk_mean_tb: NULL argument");
  rt_status st = check_view(v);
  if (st != RT_OK) return st;
  if (nf < 1) return fail(RT_ERR_ARG, "rt_disk_mean_tb: nf = %d", nf);
  if (!(radius > 0.0) || !std::isfinite(radius)) return fail(RT_ERR_ARG, "rt_disk_mean_tb: radius must be > 0");
  disk_mean<<<nf, kDiskThreads, 0, (cudaStream_t)stream>>>(tb, v->nx, v->ny, v->x0, (v->x1 - v->x0) / v->nx, v->y0,
                                                          (v->y1 - v->y0) / v->ny, radius * radius, mean_out);
  RT_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_probe_field(rt_ctx* ctx, const rt_grid* g, const float* xyz, int n, float* out, void* stream) {
  if (!ctx || !g || (n > 0 && (!xyz || !out))) return fail(RT_ERR_ARG, "rt_probe_field: NULL argument");
  if (n < 0) return fail(RT_ERR_ARG, "rt_probe_field: n = %d", n);
  if (n == 0) return RT_OK;
  RT_CUDA(cudaSetDevice(ctx->device));
  probe_field<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(g->dev, xyz, n, out);
  RT_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_sync(rt_ctx* ctx, void* stream) {
  if (!ctx) return fail(RT_ERR_ARG, "rt_sync: ctx is NULL");
  RT_CUDA(cudaSetDevice(ctx->device));
  RT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  RT_CUDA(cudaGetLastError());
  return RT_OK;
}

rt_status rt_get_stats(rt_ctx* ctx, void* stream, rt_stats* out) {
  if (!ctx || !out) return fail(RT_ERR_ARG, "rt_get_stats: NULL argument");
  RT_CUDA(cudaSetDevice(ctx->device));
  unsigned long long h[2] = {0, 0};
  RT_CUDA(cudaMemcpyAsync(h, ctx->d_stats, sizeof h, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  RT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  out->ray_steps = h[0];
  out->rays = h[1];
  return RT_OK;
}

}  // extern "C"

// ------------------------------------------------------- allocation-free batch
// Scratch of rt_trace_batch_noalloc: [0, 256) ticket (u32 at 0) and ray
// counters (2 x u64 at 8), then the view, map and chunk tables (16-byte
// aligned).  Host code only ever uses the address returned by
// cudaGetSymbolAddress for the current device, never the symbol itself.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
struct NoAllocDevice {
  std::once_flag once;
  unsigned char* scratch = nullptr;
  int sm_count = 0;
  cudaError_t err = cudaSuccess;
};
NoAllocDevice g_noalloc_devices[kMaxDevices];

size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

// Host staging of the tables, also static: the call allocates no host memory
// either.  One image of the device scratch, and the chunk candidates with
// their length estimates for the longest-first order.  The mutex serialises
// callers on different threads while they fill and copy it (a pageable
// cudaMemcpyAsync has read its source when it returns).
constexpr size_t kNoAllocMaxChunks = RT_NOALLOC_SCRATCH_BYTES / sizeof(ChunkDev);
struct NoAllocCand {
  double cost;
  unsigned int order;  // position in the request order: ties keep it
  ChunkDev c;
};
alignas(256) unsigned char g_noalloc_image[RT_NOALLOC_SCRATCH_BYTES];
NoAllocCand g_noalloc_cands[kNoAllocMaxChunks];
std::mutex g_noalloc_host_mutex;

}  // namespace

extern "C" rt_status rt_trace_batch_noalloc(const rt_grid* g, const rt_request* reqs, int nreq, const rt_options* o,
                                            void* stream) {
  if (!g || !reqs) return fail(RT_ERR_ARG, "rt_trace_batch_noalloc: NULL argument");
  if (nreq < 1) return fail(RT_ERR_ARG, "rt_trace_batch_noalloc: nreq = %d", nreq);
  int nb = 0;
  rt_status st = check_options(o, &nb);
  if (st != RT_OK) return st;
  int dev = 0;
  RT_CUDA(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(RT_ERR_ARG, "rt_trace_batch_noalloc: the current device is %d, the grid lives on device %d", dev,
                g->device);
  if (dev < 0 || dev >= kMaxDevices) return fail(RT_ERR_ARG, "rt_trace_batch_noalloc: device %d", dev);
  NoAllocDevice& D = g_noalloc_devices[dev];
  std::call_once(D.once, [&D, dev]() {
    void* p = nullptr;
    D.err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (D.err == cudaSuccess) D.err = cudaDeviceGetAttribute(&D.sm_count, cudaDevAttrMultiProcessorCount, dev);
    D.scratch = static_cast<unsigned char*>(p);
  });
  if (D.err != cudaSuccess || !D.scratch)
    return fail(RT_ERR_CUDA, "rt_trace_batch_noalloc: scratch set-up failed: %s", cudaGetErrorString(D.err));

  // sizes first: one view per request, one map per (request, frequency),
  // chunks of up to kChunk pixels
  size_t n_maps = 0, n_chunks = 0;
  for (int q = 0; q < nreq; ++q) {
    const rt_request& R = reqs[q];
    if (!R.view || !R.freqs_hz || !R.tb_out || R.nf < 1) return fail(RT_ERR_ARG, "request %d: NULL field or nf < 1", q);
    st = check_view(R.view);
    if (st != RT_OK) return st;
    for (int fi = 0; fi < R.nf; ++fi)
      if (bad_freq(R.freqs_hz[fi])) return fail(RT_ERR_ARG, "request %d frequency %d is not > 0", q, fi);
    n_maps += (size_t)R.nf;
    n_chunks += (size_t)R.nf * (((size_t)R.view->nx * R.view->ny + kChunk - 1) / kChunk);
  }
  const size_t off_views = 256;
  const size_t off_maps = align16(off_views + sizeof(ViewDev) * (size_t)nreq);
  const size_t off_chunks = align16(off_maps + sizeof(MapDev) * n_maps);
  const size_t bytes = off_chunks + sizeof(ChunkDev) * n_chunks;
  if (bytes > RT_NOALLOC_SCRATCH_BYTES || n_chunks > kNoAllocMaxChunks)
    return fail(RT_ERR_ARG, "rt_trace_batch_noalloc: the batch needs %zu bytes of scratch, the static scratch holds %u",
                bytes, (unsigned)RT_NOALLOC_SCRATCH_BYTES);

  std::lock_guard<std::mutex> lock(g_noalloc_host_mutex);
  unsigned char* img = g_noalloc_image;
  std::memset(img, 0, off_views);  // the zero control block clears the ticket and counters
  ViewDev* views = reinterpret_cast<ViewDev*>(img + off_views);
  MapDev* maps = reinterpret_cast<MapDev*>(img + off_maps);
  const double rmin = g->r.front(), rmax = g->r.back();
  size_t m = 0, c = 0;
  for (int q = 0; q < nreq; ++q) {
    const rt_request& R = reqs[q];
    views[q] = make_view(*R.view);
    const int npix = R.view->nx * R.view->ny;
    const double du = (R.view->x1 - R.view->x0) / R.view->nx, dv = (R.view->y1 - R.view->y0) / R.view->ny;
    for (int fi = 0; fi < R.nf; ++fi, ++m) {
      MapDev M;
      M.f = make_freq(R.freqs_hz[fi], fi);
      M.view = q;
      M.out = R.tb_out + (size_t)fi * npix;
      M.diag = R.diag ? reinterpret_cast<RayDiag*>(R.diag) + (size_t)fi * npix : nullptr;
      maps[m] = M;
      const double rc = turning_radius(g, R.freqs_hz[fi]);
      for (int p0 = 0; p0 < npix; p0 += kChunk, ++c) {
        const int pix = p0 + std::min(kChunk, npix - p0) / 2, ix = pix % R.view->nx, iy = pix / R.view->nx;
        const double u = R.view->x0 + (ix + 0.5) * du, v = R.view->y0 + (iy + 0.5) * dv;
        g_noalloc_cands[c] = {path_estimate(std::sqrt(u * u + v * v), rc, rmin, rmax), (unsigned int)c,
                              ChunkDev{(int)m, p0, std::min(kChunk, npix - p0), 0}};
      }
    }
  }
  // longest first; std::sort works in place (no temporary buffer), the
  // request order breaks ties
  std::sort(g_noalloc_cands, g_noalloc_cands + n_chunks, [](const NoAllocCand& a, const NoAllocCand& b) {
    return a.cost > b.cost || (a.cost == b.cost && a.order < b.order);
  });
  ChunkDev* chunks = reinterpret_cast<ChunkDev*>(img + off_chunks);
  for (size_t i = 0; i < n_chunks; ++i) chunks[i] = g_noalloc_cands[i].c;

  cudaStream_t s = (cudaStream_t)stream;
  RT_CUDA(cudaMemcpyAsync(D.scratch, img, bytes, cudaMemcpyHostToDevice, s));
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  fill_common(P, g, o);
  P.views = reinterpret_cast<const ViewDev*>(D.scratch + off_views);
  P.maps = reinterpret_cast<const MapDev*>(D.scratch + off_maps);
  P.chunks = reinterpret_cast<const ChunkDev*>(D.scratch + off_chunks);
  P.counter = reinterpret_cast<unsigned int*>(D.scratch);
  P.stats = reinterpret_cast<unsigned long long*>(D.scratch + 8);
  P.total = (unsigned int)(n_chunks * kChunk);
  RT_CUDA(dispatch_trace(nb, o->precision == RT_MIXED, P, D.sm_count, s, is_tube(o)));
  return RT_OK;
}
