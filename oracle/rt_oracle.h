/* Oracle test infrastructure: a plain, slow FP64 CPU implementation of the
 * refractive ray-tracing + ray-tube magnification + free-free transfer method
 * ("Modeling the Thermal Low-Frequency Radio Sun with Ray Tracing",
 * Sec. 2-3, Eqs. 1-12).  Only tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load or run it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * All lengths are in solar radii (R_sun = 6.957e10 cm), frequencies in Hz,
 * densities in cm^-3, temperatures in K.  Every call is synchronous and
 * returns 0 on success, a negative number on a bad argument.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_GRID = 0, ORC_UNIFORM = 1, ORC_VACUUM = 2, ORC_SLAB = 3, ORC_NEWKIRK = 4 };
enum { ORC_STEPWISE = 0, ORC_TUBE = 1, ORC_MAG_OFF = 2 };
enum { ORC_RUNNING = 0, ORC_EXIT_OUTER = 1, ORC_HIT_INNER = 2, ORC_TAU_STOP = 3,
       ORC_STEP_LIMIT = 4, ORC_MISS = 5, ORC_NAN = 6 };

typedef struct {
  int kind;                  /* ORC_GRID or an analytic field                   */
  double r_min, r_max;       /* termination spheres (grid: first / last r node) */
  int n_r, n_t, n_p;         /* grid node counts                                */
  const double *r, *theta, *phi;   /* node coordinates (monotone; phi periodic)  */
  const double *ne, *te;     /* node values [n_r][n_t][n_p], phi fastest        */
  double ne0, te0;           /* analytic: uniform n_e (slab: dn_e/dq), T_e      */
  double q[3], c;            /* slab: n_e = ne0 * max(q.x - c, 0)               */
} orc_field;

typedef struct { double lon, lat; int nx, ny; double x0, x1, y0, y1; } orc_view;

typedef struct {
  double dtau;      /* RK4 step in the Hamiltonian parameter [R_sun]          */
  int s_mode;       /* ORC_STEPWISE (paper), ORC_TUBE, ORC_MAG_OFF            */
  int n_nb;         /* 2 (paper, one-sided), 4 or 8 neighbour rays            */
  int eps_mode;     /* 0: eps = eta * |dr| (Eq. 8); 1: eps = delta           */
  double eta;       /* perturbation ratio                                     */
  double delta;     /* fixed offset [R_sun] (eps_mode 1, tube mode)           */
  double tau_stop;  /* stop once the optical depth reaches it (<= 0: never)   */
  int max_steps;    /* <= 0: ceil(40 r_max / dtau)                            */
  int tbc_mode;     /* 0: inner boundary T_bc = T_e at the crossing; 1: tbc_K */
  double tbc_K;
  int emission;     /* 1: free-free j, kappa; 0: j = kappa = 0                */
  int straight;     /* 1: straight line of sight (no refraction, n = 1)       */
  double jitter;    /* conditioning probe (orc_trace only): relative noise    */
                    /* of this size on r, theta, phi of every grid lookup;    */
                    /* 0 = off (the method itself)                            */
  unsigned long long jitter_seed;
} orc_options;

typedef struct {
  double tb;        /* brightness temperature [K]                             */
  double tau;       /* optical depth along the path                           */
  double ln_s;      /* ln(S_N / S_0)                                          */
  double exit[3];   /* last path node (crossing point for EXIT/HIT)           */
  double alpha;     /* fraction of the last step kept (1 unless clipped)      */
  int status;       /* ORC_* ray status                                       */
  int steps;        /* central RK4 steps taken                                */
} orc_ray;

/* C_pe = e^2 / (pi m_e) [Hz^2 cm^3] and R_sun [cm] as the oracle uses them. */
double orc_c_pe(void);
double orc_r_sun_cm(void);

/* n_e, grad n_e and T_e of the field at p (Sec. 3.2 trilinear reading). */
int orc_field_eval(const orc_field* F, const double p[3], double* ne, double grad[3], double* te);

/* One RK4 step of dr/dtau = k, dk/dtau = 1/2 grad n^2 (Eq. 4) in place. */
int orc_rk4_step(const orc_field* F, double f_hz, double h, int straight, double r[3], double k[3]);

/* Step-wise magnification M^{i+1} of one central step from (r, k) (Eqs. 5-11). */
int orc_stepwise_m(const orc_field* F, double f_hz, const orc_options* o,
                   const double r[3], const double k[3], double* m_out);

/* Free-free absorption coefficient kappa_vac [cm^-1] (Dulk 1985). */
double orc_kappa_vac(double ne, double te, double f_hz);

/* Trace the listed pixels (iy*nx + ix; NULL = all) at every frequency.
 * out has nf*npix entries, frequency-major. */
int orc_trace(const orc_field* F, const orc_view* V, const double* freqs, int nf,
              const orc_options* o, const int* pixels, int npix, orc_ray* out, int nthreads);

/* One ray with its whole path: node positions r[3*cap], wave vectors k[3*cap],
 * node n_e, T_e, ln S (cap entries each).  *n_nodes receives the node count
 * (which may exceed cap: then only the first cap nodes are written). */
int orc_trace_path(const orc_field* F, const orc_view* V, double f_hz, const orc_options* o,
                   int pixel, int cap, double* r, double* k, double* ne, double* te,
                   double* ln_s, int* n_nodes, orc_ray* out);

/* Gradient of L = sum dL_dTb * T_b over the listed rays with respect to the
 * grid node values (tape reverse mode, discrete events held fixed).
 * dL_dne, dL_dte: [n_r*n_t*n_p], overwritten.  tb_out (optional): [nf*npix]. */
int orc_backward(const orc_field* F, const orc_view* V, const double* freqs, int nf,
                 const orc_options* o, const int* pixels, int npix, const double* dL_dTb,
                 double* dL_dne, double* dL_dte, double* tb_out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
