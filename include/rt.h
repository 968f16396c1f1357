/*
 * librt — GB300 (sm_103a) refractive radio ray tracing with ray-tube
 * magnification and thermal free-free transfer.
 *
 * The library computes the method of "Modeling the Thermal Low-Frequency
 * Radio Sun with Ray Tracing" (arXiv 2606.02413):
 *   - rays from the observer through a spherical (r, theta, phi) grid of
 *     electron density n_e and temperature T_e (Sec. 3.1-3.2), one ray per
 *     image pixel and frequency;
 *   - unmagnetised Hamiltonian ray equations dr/dtau = k, dk/dtau =
 *     grad(n^2)/2 with n^2 = 1 - f_pe^2/f^2, advanced by RK4 with a fixed
 *     step (Sec. 2.1, Eq. 4);
 *   - the ray-tube area S(s) from step-wise perturbation retracing of
 *     neighbour rays (Sec. 2.1, Eqs. 5-11);
 *   - the transfer equation dI/ds = j - kappa I - I dlnS/ds (Eqs. 2-3,
 *     12) with thermal free-free j and kappa, integrated along each ray.
 *
 * Units: lengths in solar radii (R_sun = 6.957e10 cm), frequencies in Hz,
 * n_e in cm^-3, temperatures in K, brightness temperature T_b in K.
 *
 * Conventions for every entry point:
 *   - Every call returns rt_status: RT_OK (0) or a negative error code.
 *     Nothing throws across the ABI.  rt_last_error() returns a message for
 *     the calling thread's most recent failure.
 *   - Argument errors are reported synchronously, before any work is queued.
 *   - Work is queued on the caller's CUDA stream (passed as void*, a
 *     cudaStream_t; NULL = the legacy default stream) and runs
 *     asynchronously; device-side errors surface in rt_sync().
 *   - Pointers documented "device" must be device (or managed) memory of the
 *     context's device; "host" pointers are read before the call returns.
 *   - Physically odd inputs are not errors: a frequency below the local
 *     plasma frequency only makes rays turn earlier.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int rt_status;
enum {
  RT_OK = 0,
  RT_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad option) */
  RT_ERR_GRID = -2,     /* grid descriptor or grid values rejected               */
  RT_ERR_CUDA = -3,     /* a CUDA runtime call failed                            */
  RT_ERR_OOM = -4,      /* device allocation failed                              */
  RT_ERR_TIMEOUT = -5,  /* a bounded device wait expired                         */
  RT_ERR_CHECKED = -6,  /* a device-side bounds check recorded a violation       */
  RT_ERR_UNSUPPORTED = -7 /* a valid request the library does not implement    */
};

enum { RT_F32 = 0, RT_F64 = 1 };                       /* grid value types        */
enum { RT_STEPWISE = 0, RT_TUBE = 1, RT_MAG_OFF = 2 }; /* ray-tube area mode      */
enum { RT_PLAIN_F32 = 0, RT_MIXED = 1 };               /* arithmetic form         */

/* Per-ray status (rt_ray_diag.status). */
enum {
  RT_RAY_EXIT_OUTER = 1, /* left the outer sphere moving outward              */
  RT_RAY_HIT_INNER = 2,  /* reached the inner sphere r = r_min                */
  RT_RAY_TAU_STOP = 3,   /* optical depth reached tau_stop                    */
  RT_RAY_STEP_LIMIT = 4, /* max_steps central steps taken                     */
  RT_RAY_MISS = 5,       /* line misses the outer sphere or cannot enter      */
  RT_RAY_NAN = 6         /* state became non-finite                           */
};

typedef struct rt_ctx rt_ctx;
typedef struct rt_grid rt_grid;

/* Spherical grid (Sec. 3.1: n_e, T_e on an r x theta x phi mesh).
 * r nodes: strictly increasing, r[0] > 0; r[0] and r[n_r-1] are the inner
 *   and outer termination spheres.  Any spacing.
 * theta nodes (colatitude, rad): strictly increasing in [0, pi], uniformly
 *   spaced.  Outside [theta[0], theta[n_t-1]] the field is clamped.
 * phi nodes (rad): uniformly spaced with n_p * dphi = 2 pi (periodic).
 * Values ne, te: [n_r][n_t][n_p], phi fastest; ne >= 0, te > 0, finite. */
typedef struct {
  int n_r, n_theta, n_phi;
  const double* r_nodes;      /* host, n_r entries      */
  const double* theta_nodes;  /* host, n_theta entries  */
  const double* phi_nodes;    /* host, n_phi entries    */
  int dtype;                  /* RT_F32 or RT_F64 for ne and te            */
  int on_device;              /* 1: ne/te are device pointers, 0: host     */
} rt_grid_desc;

/* Observer view (Sec. 3.2).  The observer direction is
 * o = (cos lat cos lon, cos lat sin lon, sin lat); rays travel along -o.
 * Image axes e_u = (-sin lon, cos lon, 0), e_v = o x e_u; pixel (ix, iy)
 * sits at u = x0 + (ix + 1/2)(x1 - x0)/nx, v = y0 + (iy + 1/2)(y1 - y0)/ny. */
typedef struct {
  double lon_rad, lat_rad;
  int nx, ny;
  double x0, x1, y0, y1;
} rt_view;

typedef struct {
  double dtau;      /* fixed RK4 step of the Hamiltonian parameter [R_sun] (> 0)   */
  int s_mode;       /* RT_STEPWISE (paper), RT_TUBE, RT_MAG_OFF                     */
  int n_nb;         /* neighbour rays: 2 (paper, one-sided), 4 or 8                 */
  int eps_mode;     /* 0: eps = eta |dr| (Eq. 8); 1: eps = delta                    */
  double eta;       /* perturbation ratio (Eq. 8)                                   */
  double delta;     /* fixed offset [R_sun]                                         */
  double tau_stop;  /* stop a ray once its optical depth reaches this (<= 0: never) */
  int max_steps;    /* central steps per ray; <= 0: ceil(40 r_max / dtau)           */
  int tbc_mode;     /* 0: inner boundary T_bc = T_e at the crossing; 1: tbc_K        */
  double tbc_K;
  int emission;     /* 1: free-free j and kappa; 0: j = kappa = 0 (I S = const)     */
  int straight;     /* 1: straight lines of sight, n = 1, no magnification           */
  int precision;    /* RT_PLAIN_F32 or RT_MIXED (compensated state and accumulators) */
  int tile;         /* launch: rt_trace_image takes pixels in tile x tile blocks (2..32); */
                    /* 0 = 64-pixel chunks, longest first.  Results do not depend on it. */
  int blocks_per_sm;/* launch: persistent blocks per SM; 0 = as many as fit              */
} rt_options;

/* Optional per-ray diagnostics (28 bytes). */
typedef struct {
  float exit_pos[3]; /* last path node: crossing point for EXIT/HIT, else last node */
  float tau;         /* optical depth along the path                               */
  float ln_s;        /* ln(S_N / S_0)                                              */
  int32_t steps;     /* central RK4 steps                                           */
  int32_t status;    /* RT_RAY_*                                                    */
} rt_ray_diag;

/* Counters of the most recent trace call on a context. */
typedef struct {
  unsigned long long ray_steps;  /* central RK4 steps summed over rays               */
  unsigned long long rays;       /* rays traced (MISS included)                      */
} rt_stats;

/* Fills *o with the defaults: dtau 2e-3, step-wise, 4 neighbours, eta 0.5,
 * delta 1e-3, tau_stop 30, max_steps auto, T_bc = T_e, emission on, plain FP32. */
void rt_default_options(rt_options* o);

const char* rt_status_string(rt_status s);
/* Message of the calling thread's last failed call ("" if none). */
const char* rt_last_error(void);

/* Creates a context on CUDA device `device`; *out owns a few KB of device
 * scratch (queue counter, statistics).  Errors: RT_ERR_ARG, RT_ERR_CUDA. */
rt_status rt_create(rt_ctx** out, int device);
/* Releases the context and its scratch.  Grids must be freed first. */
rt_status rt_destroy(rt_ctx* ctx);

/* Copies the grid into library-owned device memory, converted to FP32 and
 * repacked cell by cell (the 8 corner values of each cell contiguous, for
 * n_e and T_e; 64 B per cell, plus one all-zero shell of cells that the
 * lookup selects beyond r_max (1 + 1e-6), the vacuum), and builds the radial
 * lookup table.  Synchronous: returns
 * after the copy and a device-side value check; the caller may free ne/te
 * afterwards.  Errors: RT_ERR_ARG (null pointers), RT_ERR_GRID (node
 * arrays not monotone / not uniform where required, non-finite or negative
 * n_e, non-positive T_e), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_load_grid(rt_ctx* ctx, const rt_grid_desc* desc, const void* ne, const void* te,
                       void* stream, rt_grid** out);
rt_status rt_free_grid(rt_ctx* ctx, rt_grid* grid);

/* Traces one image at nf frequencies (Sec. 3.2-3.3): for every pixel and
 * frequency one ray bundle (the central ray and its n_nb neighbours: one
 * thread per bundle in the step-wise forms and with magnification off,
 * adjacent lanes of a warp in tube mode), stepped with RK4, with the tube
 * magnification and the free-free transfer accumulated along the way.
 * freqs_hz: host, nf entries (1 <= nf <= 64), each > 0.
 * tb_out:   device, [nf][ny][nx] float, caller-owned, fully overwritten.
 * diag:     device, [nf][ny][nx] rt_ray_diag, or NULL.
 * Work order: with opt->tile = 0 the rays are taken in 64-pixel chunks of
 * all frequencies, longest estimated paths first (as a batch plan orders
 * them), from a work table that the call stages in the context's pinned
 * host buffer and copies into a stream-ordered device allocation freed
 * after the launch; a call may wait for the previous call's table copy to
 * leave that buffer.  opt->tile > 0: tiles of each frequency in turn,
 * lowest frequency first, no table.  Results do not depend on the order.
 * Asynchronous on `stream`.  Errors: RT_ERR_ARG, RT_ERR_UNSUPPORTED,
 * RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_trace_image(rt_ctx* ctx, const rt_grid* grid, const rt_view* view,
                         const double* freqs_hz, int nf, const rt_options* opt,
                         float* tb_out, rt_ray_diag* diag, void* stream);

/* One image request of a batch: a view and its frequencies. */
typedef struct {
  const rt_view* view;     /* host                                                */
  const double* freqs_hz;  /* host, nf entries, each > 0                          */
  int nf;                  /* >= 1                                                */
  float* tb_out;           /* device [nf][ny][nx] float, caller-owned             */
  rt_ray_diag* diag;       /* device [nf][ny][nx] or NULL                         */
} rt_request;

typedef struct rt_batch_plan rt_batch_plan;

/* Plans one launch over heterogeneous requests (many images, frequencies
 * and observer longitudes at once; the per-ray work is that of
 * rt_trace_image, Sec. 3.2).  The rays are cut into chunks of up to 64
 * pixels of one (request, frequency) map and ordered longest-first by a
 * path-length estimate (entry chord, and the turning radius where the
 * shell-mean plasma frequency equals f); one persistent kernel takes them
 * from a device ticket queue, so rays of very uneven length keep every warp
 * busy.  The plan owns its device tables and a few bytes of scratch (the
 * queue ticket and counters) and captures {reset scratch, kernel} in a CUDA
 * graph.  Synchronous (uploads the tables).  The requests' output buffers
 * must stay valid while the plan is launched.  Errors: RT_ERR_ARG,
 * RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_batch_plan_create(rt_ctx* ctx, const rt_grid* grid, const rt_request* reqs, int nreq,
                               const rt_options* opt, rt_batch_plan** out);
/* Multi-GPU partition of one job (the (request, frequency, pixel-chunk)
 * items of the rays, which are independent, Sec. 3.2): the plan of rank
 * `rank` of `world_size` holds only the chunks that the longest-first greedy
 * partition (rt_shard_assign over the plan's path-length estimates) gives
 * that rank.  Every rank computes the same partition from the same
 * requests, so the ranks' plans cover every ray exactly once; each rank
 * writes only its own rays' pixels of the output maps (zero the maps and sum
 * them over the ranks to gather them).  Per-ray arithmetic is that of
 * rt_batch_plan_create.  Errors: as rt_batch_plan_create, and RT_ERR_ARG for
 * rank outside [0, world_size). */
rt_status rt_batch_plan_create_shard(rt_ctx* ctx, const rt_grid* grid, const rt_request* reqs, int nreq,
                                     const rt_options* opt, int rank, int world_size, rt_batch_plan** out);
/* The partition above, on the host (needs no GPU): items are taken in order
 * of decreasing cost (stable), each given to the rank with the least total
 * cost so far (the lowest rank on ties).  cost: host [n], finite, >= 0;
 * rank_of: host [n], written.  Errors: RT_ERR_ARG. */
rt_status rt_shard_assign(const double* cost, long n, int world_size, int* rank_of);
/* Replays the plan's graph on `stream` (asynchronous). */
rt_status rt_batch_plan_launch(rt_batch_plan* plan, void* stream);
/* Counters of the plan's most recent launch (waits for `stream`). */
rt_status rt_batch_plan_stats(rt_batch_plan* plan, void* stream, rt_stats* out);
rt_status rt_batch_plan_destroy(rt_batch_plan* plan);

/* One-shot batch: plan, launch on `stream`, wait for it, release the plan. */
rt_status rt_trace_batch(rt_ctx* ctx, const rt_grid* grid, const rt_request* reqs, int nreq,
                         const rt_options* opt, void* stream);

/* Gradient of a map misfit with respect to the grid (adjoint of
 * rt_trace_image; the paper's forward method differentiated, Sec. 2.1
 * Eqs. 4-12 and Sec. 3.2).  For L = sum over pixels and frequencies of
 * dL_dTb * T_b, returns dL/dn_e and dL/dT_e at every grid node, exact for
 * the discrete forward computation with its discrete events held fixed
 * (cell indices, the basis axis branch, the step count, the termination
 * step).  Internally: the forward pass (skipped when fwd_diag is given), a
 * second forward pass that stores the ray state every 32 central steps, then
 * a reverse sweep that recomputes each 32-step segment and runs the
 * transfer, tube-area, neighbour-retrace and RK4 adjoints back through it,
 * scattering node gradients with atomics.
 * view, freqs_hz, nf, opt: as for rt_trace_image; supported forms: s_mode
 * RT_STEPWISE with n_nb = 4, or RT_MAG_OFF; not straight lines of sight.
 * dL_dTb:  device [nf][ny][nx] float.  A ray whose weight is exactly 0 cannot
 *          contribute and is not traced by any pass of the call (so a
 *          caller that splits the rays between GPUs by zeroing the others'
 *          weights does only its own share of the work).
 * dL_dne, dL_dte: device [n_r][n_theta][n_phi] float, caller-owned,
 *          overwritten (zeroed by the call first).
 * tb_out:  device [nf][ny][nx] float for the forward T_b (0 for rays with a
 *          zero weight), or NULL.
 * fwd_diag: optional device [nf][ny][nx] rt_ray_diag that rt_trace_image
 *          returned for the same grid, view, frequencies and options.  The
 *          checkpoints are sized from its
 *          step counts and the first forward pass is skipped.  NULL: the
 *          call traces the rays once more to count their steps.  A diag
 *          whose step counts differ from this forward's gives RT_ERR_ARG
 *          (no ray reads another ray's checkpoints).
 * Synchronous: returns when the gradients are complete.  Allocates and
 * frees its own device scratch (checkpoints ~ total ray steps / 32 x 68 B).
 * Errors: RT_ERR_ARG, RT_ERR_UNSUPPORTED, RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_backward(rt_ctx* ctx, const rt_grid* grid, const rt_view* view, const double* freqs_hz, int nf,
                      const rt_options* opt, const float* dL_dTb, float* dL_dne, float* dL_dte, float* tb_out,
                      const rt_ray_diag* fwd_diag, void* stream);

/* An adjoint tape: the forward of rt_trace_image, run once with the ray
 * state stored every 32 central steps, so that rt_backward_tape reverses it
 * without tracing the rays again (rt_backward traces them twice more).  The
 * forward is the arithmetic of rt_trace_image: T_b and the diagnostics are
 * identical (no tile walk: opt->tile is ignored).
 * view, freqs_hz, nf, opt: as for rt_backward (its supported forms).
 * pool_bytes: device memory for the stored states, 72 B per started
 *          32-step segment of every ray; 0 sizes the pool at 1.5 times an
 *          estimate from the entry chords cut at each frequency's turning
 *          radius.  A pool that overflows leaves the tape usable:
 *          rt_backward_tape then traces twice more, as rt_backward does.
 * tb_out:  device [nf][ny][nx] float, caller-owned.
 * diag:    device [nf][ny][nx] rt_ray_diag, caller-owned, kept by the tape
 *          until rt_backward_tape; or NULL (the tape holds its own).
 * out:     the tape; it refers to grid, which must outlive it.  Release it
 *          with rt_tape_free.
 * Asynchronous on stream.  Errors: RT_ERR_ARG, RT_ERR_UNSUPPORTED,
 * RT_ERR_OOM, RT_ERR_CUDA. */
typedef struct rt_tape rt_tape;
rt_status rt_trace_image_tape(rt_ctx* ctx, const rt_grid* grid, const rt_view* view, const double* freqs_hz,
                              int nf, const rt_options* opt, size_t pool_bytes, float* tb_out, rt_ray_diag* diag,
                              rt_tape** out, void* stream);
/* The gradient of sum dL_dTb * T_b (as rt_backward) from a tape: only the
 * reverse sweep runs.  dL_dTb, dL_dne, dL_dte as for rt_backward.  A tape may
 * be reversed more than once (for several weight maps).  Synchronous.
 * Errors: RT_ERR_ARG (NULL argument, or checkpoints missing for a ray),
 * RT_ERR_CUDA. */
rt_status rt_backward_tape(rt_tape* tape, const float* dL_dTb, float* dL_dne, float* dL_dte, void* stream);
/* Pool slots the tape's forward took and the pool's capacity (used > cap:
 * it overflowed).  Waits for stream. */
rt_status rt_tape_info(rt_tape* tape, void* stream, unsigned long long* slots_used, unsigned long long* slots_cap);
rt_status rt_tape_free(rt_tape* tape);

/* Allocation-free batch.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they trace:
 * real-time loops that must not stall (cudaMalloc and cudaFree synchronise
 * the device and can take milliseconds) or that run on a memory budget fixed
 * at start-up, and hosts whose device memory is all owned by another
 * allocator (a framework's caching pool), where a cudaMalloc of the library
 * can fail or fragment that pool.  It computes what rt_trace_batch computes,
 * but its scratch (the work-queue ticket, the ray counters and the
 * request/map/chunk tables) lives in one file-scope device array of
 * RT_NOALLOC_SCRATCH_BYTES (2 MiB) that every GPU loading the library holds
 * until the process exits; it calls no cudaMalloc, cudaFree or allocating
 * library routine, and stages its tables in static host memory.
 *   - Runs on the calling thread's current device, which must be the device
 *     that holds `grid` (loaded earlier with rt_load_grid; otherwise
 *     RT_ERR_ARG).  The caller passes inputs and outputs as for
 *     rt_trace_batch; no context is needed.
 *   - The first call on a device looks up the array's device address (and
 *     loads the library's kernels there).
 *   - All calls share the array, which keeps the last call's contents (the
 *     call clears the ticket and counters itself).  Calls whose work
 *     overlaps on the GPU race and give wrong results: issue them on one
 *     stream, or order them with events.
 *   - Asynchronous on `stream`; the host tables have been copied when the
 *     call returns.
 * Errors: RT_ERR_ARG (bad request, wrong device, or the tables of this batch
 * need more than RT_NOALLOC_SCRATCH_BYTES: about 100k chunks of 64 pixels),
 * RT_ERR_CUDA. */
#define RT_NOALLOC_SCRATCH_BYTES (2u << 20)
rt_status rt_trace_batch_noalloc(const rt_grid* grid, const rt_request* reqs, int nreq,
                                 const rt_options* opt, void* stream);

/* Disk-mean brightness temperature spectrum (Sec. 3.4, Fig. 10: the mean
 * T_b within 0.5 R_sun of disk centre at each frequency).  For each of the nf
 * maps of tb, the mean over the pixels whose centre (u, v) (the pixel
 * mapping of rt_view) satisfies u^2 + v^2 < radius^2; 0 where no pixel
 * centre lies inside.  Sums in FP64, in a fixed order.
 * view:     host; the view the maps were traced with (its nx, ny and extent).
 * tb:       device [nf][ny][nx] float (as written by rt_trace_image).
 * radius:   > 0, in R_sun.
 * mean_out: device double [nf], caller-owned.
 * Asynchronous on `stream`.  Errors: RT_ERR_ARG, RT_ERR_CUDA. */
rt_status rt_disk_mean_tb(const rt_view* view, const float* tb, int nf, double radius, double* mean_out,
                          void* stream);

/* One node of a recorded ray path (32 bytes). */
typedef struct {
  float r[3];     /* position [R_sun]                                                  */
  float ln_s;     /* ln(S / S_0) at the node                                           */
  float dlns_ds;  /* ln M of the step arriving at the node / its chord length [1/R_sun] */
  float tau;      /* optical depth from the entry to the node                          */
  float ne, te;   /* interpolated n_e [cm^-3] and T_e [K] at the node                  */
} rt_path_node;

/* Ray-fan diagnostics (Sec. 3.2, Figs. 4 and 6): the whole path of the rays
 * of selected pixels at one frequency, node by node (entry node first; the
 * crossing point last on a ray that ends on a sphere), with the local
 * magnification rate d ln S/ds = ln M / ds of each step.  The rays are
 * stepped with the same code and in the same order as rt_trace_image, so
 * their T_b and diagnostics equal its values for those pixels.
 * pixels:  host [n], flat indices iy * nx + ix of `view` (1 <= n <= 2^20).
 * opt:     step-wise magnification or none (tube mode: RT_ERR_UNSUPPORTED).
 * nodes:   device [n][cap] rt_path_node, caller-owned: ray i's first cap
 *          nodes (a longer path is cut, its n_nodes still counts them all).
 * n_nodes: device [n] int, the node count of each path.
 * tb_out:  device [n] float, the rays' T_b.
 * diag:    device [n] rt_ray_diag, or NULL.
 * Asynchronous on `stream` (a small stream-ordered allocation holds the
 * pixel list).  Errors: RT_ERR_ARG, RT_ERR_UNSUPPORTED, RT_ERR_CUDA. */
rt_status rt_trace_paths(rt_ctx* ctx, const rt_grid* grid, const rt_view* view, double freq_hz, const int* pixels,
                         int n, const rt_options* opt, int cap, rt_path_node* nodes, int* n_nodes, float* tb_out,
                         rt_ray_diag* diag, void* stream);

/* Beam-convolved maps (Sec. 3.3, Figs. 7-8: the maps as an interferometer
 * of maximum baseline B would see them).  Each map f is convolved with a
 * circular Gaussian beam of FWHM lambda_f / B radians, placed on the image
 * plane at 1 AU (FWHM in R_sun = lambda_f / B x 215.03), separably (rows,
 * then columns) with zero outside the image.  The weights are the samples of
 * exp(-d^2 / 2 sigma^2) at the integer pixel offsets |d| <= ceil(4 sigma),
 * normalised to sum to 1 per pass.  Sums in FP64.
 * view:      host; the view the maps were traced with (square pixels).
 * tb:        device [nf][ny][nx] float.
 * freqs_hz:  host [nf], > 0 (1 <= nf <= 64); baseline_m > 0.
 * scratch:   device [nf][ny][nx] float, caller-owned work space.
 * tb_out:    device [nf][ny][nx] float, caller-owned (may not alias tb or scratch).
 * Asynchronous on `stream`.  Errors: RT_ERR_ARG, RT_ERR_CUDA. */
rt_status rt_beam_convolve(const rt_view* view, const float* tb, const double* freqs_hz, int nf, double baseline_m,
                           float* scratch, float* tb_out, void* stream);

/* Samples the interpolated corona at n points: the field evaluation of
 * every RK4 stage (trilinear n_e, T_e in (r, theta, phi) and the exact
 * Cartesian gradient of the n_e interpolant; Sec. 3.1-3.2, Eq. 4).
 * xyz: device float [n][3] (R_sun).  out: device float [n][5] =
 * (n_e, T_e, dn_e/dx, dn_e/dy, dn_e/dz), caller-owned.  n >= 0.
 * Asynchronous on `stream`.  Errors: RT_ERR_ARG, RT_ERR_CUDA. */
rt_status rt_probe_field(rt_ctx* ctx, const rt_grid* grid, const float* xyz, int n, float* out,
                         void* stream);

/* Waits for `stream` and reports device-side errors of earlier calls. */
rt_status rt_sync(rt_ctx* ctx, void* stream);

/* Reads the counters of the context's most recent trace call (waits for
 * `stream`). */
rt_status rt_get_stats(rt_ctx* ctx, void* stream, rt_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* RT_H */
