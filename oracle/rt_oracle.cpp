// Oracle test infrastructure: plain FP64 CPU restatement of the paper's method.
// Only tests, the package smoke check and the benchmark's CPU-baseline leg may
// load or run it; it shares nothing with the CUDA library.
//
// The code follows the paper's two-stage order (Sec. 3.2): each ray is first
// traced from the observer toward the Sun with RK4 (Eq. 4), the ray-tube area
// being re-estimated at every step by step-wise perturbation retracing
// (Eqs. 5-11); the whole path is stored; only then is the transfer equation
// with the magnification term (Eqs. 2, 3, 12) integrated from the far end of
// the path back to the observer.  Everything is templated on the scalar type
// so that the same code runs on doubles and on the tape AD scalar for the
// oracle's adjoint.
#include "rt_oracle.h"
#include "ad_tape.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace oracle {

using std::atan2;
using std::exp;
using std::expm1;
using std::fabs;
using std::log;
using std::log1p;
using std::sqrt;

constexpr double kPi = 3.14159265358979323846;
// CODATA 2018 in CGS units.
constexpr double kElectronCharge = 4.803204712570263e-10;  // statC
constexpr double kElectronMass = 9.1093837015e-28;         // g
// f_pe^2 = n_e e^2 / (pi m_e)
const double kCpe = kElectronCharge * kElectronCharge / (kPi * kElectronMass);
constexpr double kRsunCm = 6.957e10;  // IAU nominal solar radius
// Points farther than r_max (1 + kOuterBand) are vacuum; the band absorbs the
// rounding of points constructed on the outer sphere.
constexpr double kOuterBand = 1e-6;

template <class T>
struct Vec3 {
  T x, y, z;
};
template <class T> Vec3<T> operator+(const Vec3<T>& a, const Vec3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> Vec3<T> operator-(const Vec3<T>& a, const Vec3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S> Vec3<T> scale(const S& s, const Vec3<T>& a) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> T dot(const Vec3<T>& a, const Vec3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> Vec3<T> cross(const Vec3<T>& a, const Vec3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> T norm(const Vec3<T>& a) { return sqrt(dot(a, a)); }
template <class T> Vec3<T> cvt(const Vec3<double>& a) { return {T(a.x), T(a.y), T(a.z)}; }

// ----------------------------------------------------------------- node values
// Plain doubles for the forward oracle; tape leaves for the adjoint.
struct PlainNodes {
  const orc_field* F;
  double ne(long i) const { return F->ne[i]; }
  double te(long i) const { return F->te[i]; }
};

struct TapeNodes {
  const orc_field* F;
  std::unordered_map<long, AD>* ne_leaf;
  std::unordered_map<long, AD>* te_leaf;
  AD ne(long i) const {
    auto it = ne_leaf->find(i);
    if (it != ne_leaf->end()) return it->second;
    AD v = AD::leaf(F->ne[i]);
    (*ne_leaf)[i] = v;
    return v;
  }
  AD te(long i) const {
    auto it = te_leaf->find(i);
    if (it != te_leaf->end()) return it->second;
    AD v = AD::leaf(F->te[i]);
    (*te_leaf)[i] = v;
    return v;
  }
};

// Conditioning probe (test instrument, off by default; not part of the
// method): perturbs r, theta and phi of every field evaluation by a relative
// amount of order `amp` from a counter-free xorshift stream, mimicking the
// rounding of single-precision geometry.  Rays whose result moves a lot
// under it are ill-conditioned at that precision.
struct Jitter {
  double amp = 0.0;
  unsigned long long state = 0;
  double next() {
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return ((state >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
  }
};

template <class T>
struct Sample {
  T ne, te;
  Vec3<T> grad;  // grad n_e
};

// Index i of the cell [a[i], a[i+1]) containing x, restricted to [0, n-2].
static int cell_index(const double* a, int n, double x) {
  int i = int(std::upper_bound(a, a + n, x) - a) - 1;
  return std::min(std::max(i, 0), n - 2);
}

// --------------------------------------------------------------------- field
// Electron density, its gradient and the temperature at p.
//
// Grid fields (reading of Sec. 3.1-3.2): n_e and T_e are trilinear in
// (r, theta, phi) within a cell, linear in physical r; grad n_e is the exact
// gradient of that interpolant, taken to Cartesian by the chain rule
//   grad f = f_r r_hat + f_theta theta_hat / r + f_phi phi_hat / (r sin theta).
// Radially the first / last cell extends linearly below r_min and up to the
// vacuum band; theta is clamped to the outermost nodes (no theta derivative
// there); phi is periodic.
template <class T, class Nodes>
Sample<T> eval_field(const orc_field& F, const Nodes& nodes, const Vec3<T>& p, Jitter* J = nullptr) {
  Sample<T> s{T(0.0), T(0.0), {T(0.0), T(0.0), T(0.0)}};
  T r = norm(p);
  const bool jit = J && J->amp > 0.0 && F.kind == ORC_GRID;
  if (jit) r = r * (1.0 + J->amp * J->next());
  if (val(r) > F.r_max * (1.0 + kOuterBand)) return s;  // vacuum
  switch (F.kind) {
    case ORC_VACUUM:
      s.te = T(F.te0);
      return s;
    case ORC_UNIFORM:
      s.ne = T(F.ne0);
      s.te = T(F.te0);
      return s;
    case ORC_SLAB: {
      Vec3<double> q{F.q[0], F.q[1], F.q[2]};
      T depth = dot(cvt<T>(q), p) - F.c;
      s.te = T(F.te0);
      if (val(depth) > 0.0) {
        s.ne = F.ne0 * depth;
        s.grad = cvt<T>(scale(F.ne0, q));
      }
      return s;
    }
    case ORC_NEWKIRK: {
      // n_e = 4.2e4 * 10^(4.32 / r): d n_e / d r = -n_e ln(10) 4.32 / r^2
      T ne = 4.2e4 * exp(std::log(10.0) * 4.32 / r);
      T dndr = -(ne * (std::log(10.0) * 4.32)) / (r * r);
      s.ne = ne;
      s.te = T(F.te0);
      s.grad = scale(dndr / r, p);
      return s;
    }
    default:
      break;
  }

  const int nr = F.n_r, nt = F.n_t, np = F.n_p;
  T rho = sqrt(p.x * p.x + p.y * p.y);
  T th = atan2(rho, p.z);
  T ph = atan2(p.y, p.x) - F.phi[0];
  if (jit) {
    th = th + 3.0 * J->amp * J->next();
    ph = ph + 3.0 * J->amp * J->next();
  }
  const double two_pi = 2.0 * kPi;
  if (val(ph) < 0.0) ph = ph + two_pi;
  if (val(ph) >= two_pi) ph = ph - two_pi;

  const int i = cell_index(F.r, nr, val(r));
  const double dr = F.r[i + 1] - F.r[i];
  T u = (r - F.r[i]) / dr;

  int j;
  T v;
  bool theta_inside;
  if (val(th) <= F.theta[0]) {
    j = 0; v = T(0.0); theta_inside = false;
  } else if (val(th) >= F.theta[nt - 1]) {
    j = nt - 2; v = T(1.0); theta_inside = false;
  } else {
    j = cell_index(F.theta, nt, val(th));
    v = (th - F.theta[j]) / (F.theta[j + 1] - F.theta[j]);
    theta_inside = true;
  }
  const double dth = F.theta[j + 1] - F.theta[j];

  // phi cell k spans [phi_k, phi_{k+1}); the last one wraps to phi_0 + 2 pi.
  int k = 0;
  while (k + 1 < np && F.phi[k + 1] - F.phi[0] <= val(ph)) ++k;
  const double lo = F.phi[k] - F.phi[0];
  const double hi = (k + 1 < np) ? F.phi[k + 1] - F.phi[0] : two_pi;
  const double dph = hi - lo;
  T w = (ph - lo) / dph;
  const int k1 = (k + 1) % np;

  auto idx = [&](int a, int b, int c) { return (long(i + a) * nt + (j + b)) * np + c; };
  T one(1.0);
  T wu[2] = {one - u, u}, wv[2] = {one - v, v}, ww[2] = {one - w, w};
  const double sg[2] = {-1.0, 1.0};
  T f(0.0), fu(0.0), fv(0.0), fw(0.0), te(0.0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        long id = idx(a, b, c ? k1 : k);
        T ne_c = nodes.ne(id);
        T te_c = nodes.te(id);
        f = f + wu[a] * wv[b] * ww[c] * ne_c;
        te = te + wu[a] * wv[b] * ww[c] * te_c;
        fu = fu + sg[a] * wv[b] * ww[c] * ne_c;
        fv = fv + wu[a] * sg[b] * ww[c] * ne_c;
        fw = fw + wu[a] * wv[b] * sg[c] * ne_c;
      }
  T f_r = fu / dr;
  T f_th = theta_inside ? fv / dth : T(0.0);
  T f_ph = fw / dph;

  Vec3<T> g = scale(f_r / r, p);
  if (val(rho) > 0.0) {
    T r2 = r * r;
    Vec3<T> dth_dx{p.z * p.x / (r2 * rho), p.z * p.y / (r2 * rho), -rho / r2};
    T rho2 = rho * rho;
    Vec3<T> dph_dx{-p.y / rho2, p.x / rho2, T(0.0)};
    g = g + scale(f_th, dth_dx) + scale(f_ph, dph_dx);
  }
  s.ne = f;
  s.te = te;
  s.grad = g;
  return s;
}

// ------------------------------------------------------------------ physics
// Free-free absorption in vacuum units (Dulk 1985, pure hydrogen, n_i = n_e):
//   kappa_vac = 9.78e-3 n_e^2 / (f^2 T^1.5) * G,
//   G = 24.5 + ln T - ln f (T > 2e5 K), 18.2 + ln T^1.5 - ln f otherwise.
// The plasma absorption coefficient is kappa_vac / n; ds = n dtau cancels n.
template <class T>
T kappa_vac(const T& ne, const T& te, double f) {
  if (!(val(ne) > 0.0) || !(val(te) > 0.0)) return T(0.0);
  T lnT = log(te);
  T G = (val(te) > 2e5) ? (24.5 + lnT - std::log(f)) : (18.2 + 1.5 * lnT - std::log(f));
  return 9.78e-3 * ne * ne * G / (f * f * te * sqrt(te));
}

struct RayCtx {
  const orc_field* F;
  const orc_options* o;
  double f;
  double h;
  Jitter* J = nullptr;
};

// dk/dtau = 1/2 grad n^2 = -(C_pe / 2 f^2) grad n_e  (Eq. 4 in the
// normalisation k_tilde = k / omega, tau = c t; see the Hamiltonian below).
template <class T, class Nodes>
Vec3<T> force(const RayCtx& C, const Nodes& nodes, const Vec3<T>& p) {
  if (C.o->straight) return {T(0.0), T(0.0), T(0.0)};
  Sample<T> s = eval_field<T>(*C.F, nodes, p, C.J);
  return scale(-kCpe / (2.0 * C.f * C.f), s.grad);
}

// Classical RK4 on x = (r, k) with fixed step h (Sec. 2.1):
// H = (k^2 - n^2) / 2 = 0, dr/dtau = dH/dk = k, dk/dtau = -dH/dr = grad(n^2)/2.
template <class T, class Nodes>
void rk4(const RayCtx& C, const Nodes& nodes, Vec3<T>& r, Vec3<T>& k) {
  const double h = C.h;
  Vec3<T> a1 = force<T>(C, nodes, r);
  Vec3<T> r2 = r + scale(h / 2, k), k2 = k + scale(h / 2, a1);
  Vec3<T> a2 = force<T>(C, nodes, r2);
  Vec3<T> r3 = r + scale(h / 2, k2), k3 = k + scale(h / 2, a2);
  Vec3<T> a3 = force<T>(C, nodes, r3);
  Vec3<T> r4 = r + scale(h, k3), k4 = k + scale(h, a3);
  Vec3<T> a4 = force<T>(C, nodes, r4);
  r = r + scale(h / 6, k + scale(2.0, k2) + scale(2.0, k3) + k4);
  k = k + scale(h / 6, a1 + scale(2.0, a2) + scale(2.0, a3) + a4);
}

// Transverse basis of Eq. 6: a = z unless |t_z| is near 1 (> 0.9), then y.
template <class T>
void transverse_basis(const Vec3<T>& t, Vec3<T>& e1, Vec3<T>& e2) {
  Vec3<T> a = (fabs(val(t.z)) <= 0.9) ? Vec3<T>{T(0.0), T(0.0), T(1.0)} : Vec3<T>{T(0.0), T(1.0), T(0.0)};
  Vec3<T> c = cross(a, t);
  e1 = scale(T(1.0) / norm(c), c);
  e2 = cross(t, e1);
}

template <class T>
T abs_det(const Vec3<T>& d1, const Vec3<T>& d2, const Vec3<T>& t) {
  return fabs(dot(cross(d1, d2), t));
}

// Step-wise magnification (Eqs. 5-11) of the central step r0 -> r0n, taken
// from (r0, k0).  Neighbours start at r0 + sigma eps e_j with the central
// wave vector k0 and are advanced one RK4 step.
//   2 neighbours (paper): d_j = r_j' - r0n.
//   4 neighbours: +-e_j pairs, d_j = (r_{+j}' - r_{-j}') / 2.
//   8 neighbours: the 4-neighbour estimate averaged with the same estimate in
//   the basis rotated by 45 degrees, g1 = (e1 + e2)/sqrt2, g2 = (e2 - e1)/sqrt2.
// M = |(d1 x d2) . t| / eps^2 (Eq. 10 without its 1/2 so that M = 1 marks an
// unchanged tube, as Eq. 11 states).
template <class T, class Nodes>
T stepwise_m(const RayCtx& C, const Nodes& nodes, const Vec3<T>& r0, const Vec3<T>& k0,
             const Vec3<T>& r0n) {
  Vec3<T> dr = r0n - r0;
  T ds = norm(dr);
  Vec3<T> t = scale(T(1.0) / ds, dr);
  Vec3<T> e1, e2;
  transverse_basis(t, e1, e2);
  T eps = (C.o->eps_mode == 1) ? T(C.o->delta) : C.o->eta * ds;
  auto advance = [&](const Vec3<T>& dir, double sigma) {
    Vec3<T> r = r0 + scale(sigma * eps, dir);
    Vec3<T> k = k0;
    rk4<T>(C, nodes, r, k);
    return r;
  };
  if (C.o->n_nb == 2) {
    Vec3<T> d1 = advance(e1, 1.0) - r0n;
    Vec3<T> d2 = advance(e2, 1.0) - r0n;
    return abs_det(d1, d2, t) / (eps * eps);
  }
  auto pair_m = [&](const Vec3<T>& a, const Vec3<T>& b) {
    Vec3<T> d1 = scale(0.5, advance(a, 1.0) - advance(a, -1.0));
    Vec3<T> d2 = scale(0.5, advance(b, 1.0) - advance(b, -1.0));
    return abs_det(d1, d2, t) / (eps * eps);
  };
  T m = pair_m(e1, e2);
  if (C.o->n_nb == 8) {
    const double s = 1.0 / std::sqrt(2.0);
    Vec3<T> g1 = scale(s, e1 + e2), g2 = scale(s, e2 - e1);
    m = 0.5 * (m + pair_m(g1, g2));
  }
  return m;
}

// ------------------------------------------------------------------- launch
struct Frame {
  Vec3<double> o, eu, ev, d;  // observer direction, image axes, ray direction
};

static Frame view_frame(const orc_view& V) {
  const double cl = std::cos(V.lon), sl = std::sin(V.lon), cb = std::cos(V.lat), sb = std::sin(V.lat);
  Frame fr;
  fr.o = {cb * cl, cb * sl, sb};
  fr.eu = {-sl, cl, 0.0};
  fr.ev = {-sb * cl, -sb * sl, cb};
  fr.d = {-fr.o.x, -fr.o.y, -fr.o.z};
  return fr;
}

// Entry point on the outer sphere of the line through the image-plane point
// (u, v) along -o, and k0 = n(r0) d so that H = 0.  False: the line misses
// the sphere, or the wave cannot propagate at the entry point.
template <class T, class Nodes>
bool launch(const RayCtx& C, const Nodes& nodes, const Frame& fr, double u, double v,
            Vec3<T>& r0, Vec3<T>& k0) {
  const double R = C.F->r_max;
  const double b2 = u * u + v * v;
  if (b2 >= R * R) return false;
  Vec3<double> p = scale(u, fr.eu) + scale(v, fr.ev) + scale(std::sqrt(R * R - b2), fr.o);
  r0 = cvt<T>(p);
  if (C.o->straight) {
    k0 = cvt<T>(fr.d);
    return true;
  }
  Sample<T> s = eval_field<T>(*C.F, nodes, r0, C.J);
  T n2 = 1.0 - kCpe * s.ne / (C.f * C.f);
  if (!(val(n2) > 0.0)) return false;
  k0 = scale(sqrt(n2), cvt<T>(fr.d));
  return true;
}

// Root alpha in [0, 1] of |r + alpha dr| = R on the chord, taking the
// entering (inner) or leaving (outer) crossing.
template <class T>
T chord_crossing(const Vec3<T>& r, const Vec3<T>& dr, double R, bool leaving) {
  T A = dot(dr, dr), B = 2.0 * dot(r, dr), Cc = dot(r, r) - R * R;
  T disc = B * B - 4.0 * A * Cc;
  if (val(disc) < 0.0) disc = T(0.0);
  T a = leaving ? (-B + sqrt(disc)) / (2.0 * A) : (-B - sqrt(disc)) / (2.0 * A);
  if (val(a) < 0.0) a = T(0.0);
  if (val(a) > 1.0) a = T(1.0);
  return a;
}

// ---------------------------------------------------------------- one ray
template <class T>
struct Path {
  std::vector<Vec3<T>> r, k;
  std::vector<T> ne, te, ln_s;
  T alpha{1.0};
  T tbc{0.0};
  int status = ORC_RUNNING;
};

template <class T>
struct RayResult {
  T tb{0.0}, tau{0.0}, ln_s{0.0};
  Vec3<T> exit{T(0.0), T(0.0), T(0.0)};
  T alpha{1.0};
  int status = ORC_MISS, steps = 0;
};

// Stage 1 (Sec. 3.2): trace from the observer toward the Sun, storing the path
// and the accumulated ln(S/S_0) at each node.
template <class T, class Nodes>
Path<T> trace_path(const RayCtx& C, const Nodes& nodes, const Frame& fr, double u, double v) {
  Path<T> P;
  const orc_options& o = *C.o;
  const double rmin = C.F->r_min, rmax = C.F->r_max;
  const int max_steps = (o.max_steps > 0) ? o.max_steps : int(std::ceil(40.0 * rmax / o.dtau));
  Vec3<T> r, k;
  if (!launch<T>(C, nodes, fr, u, v, r, k)) {
    P.status = ORC_MISS;
    return P;
  }
  const int mag_mode = o.straight ? ORC_MAG_OFF : o.s_mode;

  // Tube mode: neighbours launched at image-plane offsets +-delta along the
  // image axes (and the 45-degree diagonals with 8 neighbours) and integrated
  // in lock-step with the central ray; S_0 = delta^2.
  std::vector<Vec3<T>> nb_r, nb_k;
  bool tube_ok = (mag_mode == ORC_TUBE);
  if (mag_mode == ORC_TUBE) {
    const double s = 1.0 / std::sqrt(2.0);
    std::vector<std::pair<double, double>> offs;
    if (o.n_nb == 2) offs = {{1, 0}, {0, 1}};
    else offs = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    if (o.n_nb == 8) offs.insert(offs.end(), {{s, s}, {-s, -s}, {-s, s}, {s, -s}});
    for (auto& of : offs) {
      Vec3<T> rn, kn;
      if (!launch<T>(C, nodes, fr, u + o.delta * of.first, v + o.delta * of.second, rn, kn)) tube_ok = false;
      nb_r.push_back(rn);
      nb_k.push_back(kn);
    }
  }

  auto sample = [&](const Vec3<T>& p) {
    Sample<T> s = eval_field<T>(*C.F, nodes, p, C.J);
    P.ne.push_back(s.ne);
    P.te.push_back(s.te);
  };
  P.r.push_back(r);
  P.k.push_back(k);
  sample(r);
  P.ln_s.push_back(T(0.0));
  T tau(0.0);
  const double seg = o.dtau * kRsunCm;

  for (int i = 0;; ++i) {
    Vec3<T> rn = r, kn = k;
    rk4<T>(C, nodes, rn, kn);
    Vec3<T> dr = rn - r;

    T ln_s_next = P.ln_s.back();
    if (mag_mode == ORC_STEPWISE) {
      ln_s_next = ln_s_next + log(stepwise_m<T>(C, nodes, r, k, rn));
    } else if (mag_mode == ORC_TUBE) {
      for (size_t j = 0; j < nb_r.size(); ++j) rk4<T>(C, nodes, nb_r[j], nb_k[j]);
      if (tube_ok) {
        Vec3<T> t = scale(T(1.0) / norm(dr), dr);
        auto sep = [&](int j) {
          return (o.n_nb == 2) ? nb_r[j] - rn : scale(0.5, nb_r[j] - nb_r[j + 1]);
        };
        T S;
        if (o.n_nb == 2) S = abs_det(sep(0), sep(1), t);
        else S = abs_det(sep(0), sep(2), t);
        if (o.n_nb == 8) S = 0.5 * (S + abs_det(sep(4), sep(6), t));
        ln_s_next = log(S / (o.delta * o.delta));
      }
    }

    // geometric termination on the chord r -> rn
    int status = ORC_RUNNING;
    T alpha(1.0);
    if (val(norm(rn)) < rmin) {
      status = ORC_HIT_INNER;
      alpha = chord_crossing(r, dr, rmin, false);
    } else if (val(norm(rn)) > rmax && val(dot(rn, kn)) > 0.0) {
      status = ORC_EXIT_OUTER;
      alpha = chord_crossing(r, dr, rmax, true);
    }
    if (status != ORC_RUNNING) {
      Vec3<T> pc = r + scale(alpha, dr);
      P.r.push_back(pc);
      P.k.push_back(kn);
      sample(pc);
      P.ln_s.push_back(ln_s_next);
      P.alpha = alpha;
      P.status = status;
      if (status == ORC_HIT_INNER) P.tbc = (o.tbc_mode == 1) ? T(o.tbc_K) : P.te.back();
      return P;
    }

    r = rn;
    k = kn;
    P.r.push_back(r);
    P.k.push_back(k);
    sample(r);
    P.ln_s.push_back(ln_s_next);
    if (!std::isfinite(val(r.x) + val(r.y) + val(r.z) + val(k.x) + val(k.y) + val(k.z))) {
      P.status = ORC_NAN;
      return P;
    }
    if (o.emission) {
      size_t n = P.ne.size();
      tau = tau + 0.5 * (kappa_vac(P.ne[n - 2], P.te[n - 2], C.f) + kappa_vac(P.ne[n - 1], P.te[n - 1], C.f)) * seg;
    }
    if (o.tau_stop > 0.0 && val(tau) >= o.tau_stop) {
      P.status = ORC_TAU_STOP;
      return P;
    }
    if (i + 1 >= max_steps) {
      P.status = ORC_STEP_LIMIT;
      return P;
    }
  }
}

// Stage 2 (Sec. 3.2, Eq. 2 with Eq. 12): transfer from the far end of the
// path back to the observer,
//   I_N = T_bc,
//   I_i = [I_{i+1} e^{-dtau_i} + Tbar_i (1 - e^{-dtau_i})] S_{i+1} / S_i,
// with dtau_i = (kappa_i + kappa_{i+1})/2 * dtau * R_sun (times the kept
// fraction on a clipped last step) and Tbar_i the segment-mean T_e
// (Rayleigh-Jeans source function T_e).
template <class T>
RayResult<T> transfer(const RayCtx& C, const Path<T>& P) {
  RayResult<T> R;
  R.status = P.status;
  if (P.status == ORC_MISS) return R;
  const int N = int(P.r.size()) - 1;
  R.steps = N;
  R.exit = P.r.back();
  R.alpha = P.alpha;
  R.ln_s = P.ln_s.back();
  const bool clipped = (P.status == ORC_HIT_INNER || P.status == ORC_EXIT_OUTER);
  const double seg = C.o->dtau * kRsunCm;
  T I = P.tbc;
  T tau(0.0);
  for (int i = N - 1; i >= 0; --i) {
    T frac = (clipped && i == N - 1) ? P.alpha : T(1.0);
    T dt(0.0);
    if (C.o->emission)
      dt = 0.5 * (kappa_vac(P.ne[i], P.te[i], C.f) + kappa_vac(P.ne[i + 1], P.te[i + 1], C.f)) * seg * frac;
    T tbar = 0.5 * (P.te[i] + P.te[i + 1]);
    T att = exp(-dt);
    I = (I * att + tbar * (-expm1(-dt))) * exp(P.ln_s[i + 1] - P.ln_s[i]);
    tau = tau + dt;
  }
  R.tb = I;
  R.tau = tau;
  return R;
}

struct PixelGeom {
  double u, v;
};
static PixelGeom pixel_centre(const orc_view& V, int pixel) {
  const int ix = pixel % V.nx, iy = pixel / V.nx;
  return {V.x0 + (ix + 0.5) * (V.x1 - V.x0) / V.nx, V.y0 + (iy + 0.5) * (V.y1 - V.y0) / V.ny};
}

static bool field_ok(const orc_field* F) {
  if (!F || !(F->r_max > F->r_min) || F->r_min < 0) return false;
  if (F->kind == ORC_GRID) {
    if (F->n_r < 2 || F->n_t < 2 || F->n_p < 2 || !F->r || !F->theta || !F->phi || !F->ne || !F->te) return false;
  }
  return true;
}

static void fill_ray(const RayResult<double>& R, orc_ray* out) {
  out->tb = R.tb;
  out->tau = R.tau;
  out->ln_s = R.ln_s;
  out->exit[0] = R.exit.x;
  out->exit[1] = R.exit.y;
  out->exit[2] = R.exit.z;
  out->alpha = R.alpha;
  out->status = R.status;
  out->steps = R.steps;
}

}  // namespace oracle

using namespace oracle;

extern "C" {

double orc_c_pe(void) { return kCpe; }
double orc_r_sun_cm(void) { return kRsunCm; }

int orc_field_eval(const orc_field* F, const double p[3], double* ne, double grad[3], double* te) {
  if (!field_ok(F) || !p) return -1;
  PlainNodes nodes{F};
  Sample<double> s = eval_field<double>(*F, nodes, Vec3<double>{p[0], p[1], p[2]});
  if (ne) *ne = s.ne;
  if (te) *te = s.te;
  if (grad) { grad[0] = s.grad.x; grad[1] = s.grad.y; grad[2] = s.grad.z; }
  return 0;
}

int orc_rk4_step(const orc_field* F, double f_hz, double h, int straight, double r[3], double k[3]) {
  if (!field_ok(F) || !(f_hz > 0)) return -1;
  orc_options o{};
  o.dtau = h;
  o.straight = straight;
  RayCtx C{F, &o, f_hz, h};
  PlainNodes nodes{F};
  Vec3<double> rv{r[0], r[1], r[2]}, kv{k[0], k[1], k[2]};
  rk4<double>(C, nodes, rv, kv);
  r[0] = rv.x; r[1] = rv.y; r[2] = rv.z;
  k[0] = kv.x; k[1] = kv.y; k[2] = kv.z;
  return 0;
}

int orc_stepwise_m(const orc_field* F, double f_hz, const orc_options* o, const double r[3],
                   const double k[3], double* m_out) {
  if (!field_ok(F) || !o || !(o->dtau > 0)) return -1;
  RayCtx C{F, o, f_hz, o->dtau};
  PlainNodes nodes{F};
  Vec3<double> r0{r[0], r[1], r[2]}, k0{k[0], k[1], k[2]};
  Vec3<double> rn = r0, kn = k0;
  rk4<double>(C, nodes, rn, kn);
  *m_out = stepwise_m<double>(C, nodes, r0, k0, rn);
  return 0;
}

double orc_kappa_vac(double ne, double te, double f_hz) { return kappa_vac<double>(ne, te, f_hz); }

int orc_trace(const orc_field* F, const orc_view* V, const double* freqs, int nf, const orc_options* o,
              const int* pixels, int npix, orc_ray* out, int nthreads) {
  if (!field_ok(F) || !V || !freqs || nf <= 0 || !o || !out || !(o->dtau > 0)) return -1;
  if (!pixels) npix = V->nx * V->ny;
  const Frame fr = view_frame(*V);
  const long total = long(nf) * npix;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (long t = 0; t < total; ++t) {
    const int fi = int(t / npix);
    const int px = pixels ? pixels[t % npix] : int(t % npix);
    Jitter J;
    J.amp = o->jitter;
    // the seed is spread over all bits first, so that seeds differing only in
    // bit 0 still give different streams after the final | 1
    J.state = ((o->jitter_seed * 0xBF58476D1CE4E5B9ull) ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(t + 1))) | 1ull;
    RayCtx C{F, o, freqs[fi], o->dtau, &J};
    PlainNodes nodes{F};
    PixelGeom g = pixel_centre(*V, px);
    Path<double> P = trace_path<double>(C, nodes, fr, g.u, g.v);
    fill_ray(transfer<double>(C, P), &out[t]);
  }
  return 0;
}

int orc_trace_path(const orc_field* F, const orc_view* V, double f_hz, const orc_options* o, int pixel,
                   int cap, double* r, double* k, double* ne, double* te, double* ln_s, int* n_nodes,
                   orc_ray* out) {
  if (!field_ok(F) || !V || !o || !(o->dtau > 0)) return -1;
  const Frame fr = view_frame(*V);
  RayCtx C{F, o, f_hz, o->dtau};
  PlainNodes nodes{F};
  PixelGeom g = pixel_centre(*V, pixel);
  Path<double> P = trace_path<double>(C, nodes, fr, g.u, g.v);
  const int n = int(P.r.size());
  if (n_nodes) *n_nodes = n;
  for (int i = 0; i < std::min(n, cap); ++i) {
    if (r) { r[3 * i] = P.r[i].x; r[3 * i + 1] = P.r[i].y; r[3 * i + 2] = P.r[i].z; }
    if (k) { k[3 * i] = P.k[i].x; k[3 * i + 1] = P.k[i].y; k[3 * i + 2] = P.k[i].z; }
    if (ne) ne[i] = P.ne[i];
    if (te) te[i] = P.te[i];
    if (ln_s) ln_s[i] = P.ln_s[i];
  }
  if (out) fill_ray(transfer<double>(C, P), out);
  return 0;
}

int orc_backward(const orc_field* F, const orc_view* V, const double* freqs, int nf, const orc_options* o,
                 const int* pixels, int npix, const double* dL_dTb, double* dL_dne, double* dL_dte,
                 double* tb_out, int nthreads) {
  if (!field_ok(F) || F->kind != ORC_GRID || !V || !freqs || nf <= 0 || !o || !dL_dTb || !dL_dne || !dL_dte)
    return -1;
  if (!pixels) npix = V->nx * V->ny;
  const long nn = long(F->n_r) * F->n_t * F->n_p;
  std::fill(dL_dne, dL_dne + nn, 0.0);
  std::fill(dL_dte, dL_dte + nn, 0.0);
  const Frame fr = view_frame(*V);
  const long total = long(nf) * npix;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    std::vector<double> gne(nn, 0.0), gte(nn, 0.0);
    Tape tape;
    active_tape() = &tape;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (long t = 0; t < total; ++t) {
      const int fi = int(t / npix);
      const int px = pixels ? pixels[t % npix] : int(t % npix);
      RayCtx C{F, o, freqs[fi], o->dtau};
      std::unordered_map<long, AD> ne_leaf, te_leaf;
      TapeNodes nodes{F, &ne_leaf, &te_leaf};
      tape.clear();
      PixelGeom g = pixel_centre(*V, px);
      Path<AD> P = trace_path<AD>(C, nodes, fr, g.u, g.v);
      RayResult<AD> R = transfer<AD>(C, P);
      if (tb_out) tb_out[t] = R.tb.v;
      if (R.tb.id < 0 || dL_dTb[t] == 0.0) continue;
      std::vector<double> adj(tape.size(), 0.0);
      adj[R.tb.id] = dL_dTb[t];
      tape.reverse(adj);
      for (auto& kv : ne_leaf) gne[kv.first] += adj[kv.second.id];
      for (auto& kv : te_leaf) gte[kv.first] += adj[kv.second.id];
    }
    active_tape() = nullptr;
#ifdef _OPENMP
#pragma omp critical
#endif
    {
      for (long i = 0; i < nn; ++i) {
        dL_dne[i] += gne[i];
        dL_dte[i] += gte[i];
      }
    }
  }
  return 0;
}

}  // extern "C"
