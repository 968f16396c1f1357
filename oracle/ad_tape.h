// Oracle test infrastructure (FP64 CPU oracle of the ray-tracing method).
// Only tests, the package smoke check and the benchmark's CPU-baseline leg
// may load or run anything under oracle/.
//
// A minimal reverse-mode automatic-differentiation scalar on a thread-local
// tape.  Every arithmetic result records at most two parents with their local
// partial derivatives; a reverse sweep over the tape accumulates adjoints.
// Discrete decisions (comparisons, floor) read the value and are therefore
// held fixed, which is the convention the oracle's adjoint uses.
#pragma once
#include <cmath>
#include <vector>

namespace oracle {

struct Tape {
  std::vector<int> pa, pb;
  std::vector<double> da, db;
  void clear() { pa.clear(); pb.clear(); da.clear(); db.clear(); }
  int push(int a, double ga, int b, double gb) {
    pa.push_back(a); da.push_back(ga); pb.push_back(b); db.push_back(gb);
    return (int)pa.size() - 1;
  }
  int size() const { return (int)pa.size(); }
  // adj must have size() entries, seeded by the caller.
  void reverse(std::vector<double>& adj) const {
    for (int i = size() - 1; i >= 0; --i) {
      double g = adj[i];
      if (g == 0.0) continue;
      if (pa[i] >= 0) adj[pa[i]] += g * da[i];
      if (pb[i] >= 0) adj[pb[i]] += g * db[i];
    }
  }
};

inline Tape*& active_tape() { static thread_local Tape* t = nullptr; return t; }

struct AD {
  double v;
  int id;  // -1: constant (not on the tape)
  AD() : v(0.0), id(-1) {}
  AD(double x) : v(x), id(-1) {}
  static AD leaf(double x) { AD r(x); r.id = active_tape()->push(-1, 0.0, -1, 0.0); return r; }
};

inline AD mk1(double v, const AD& a, double ga) {
  AD r(v);
  if (a.id >= 0) r.id = active_tape()->push(a.id, ga, -1, 0.0);
  return r;
}
inline AD mk2(double v, const AD& a, double ga, const AD& b, double gb) {
  AD r(v);
  if (a.id >= 0 || b.id >= 0) r.id = active_tape()->push(a.id, ga, b.id, gb);
  return r;
}

inline AD operator+(const AD& a, const AD& b) { return mk2(a.v + b.v, a, 1.0, b, 1.0); }
inline AD operator-(const AD& a, const AD& b) { return mk2(a.v - b.v, a, 1.0, b, -1.0); }
inline AD operator*(const AD& a, const AD& b) { return mk2(a.v * b.v, a, b.v, b, a.v); }
inline AD operator/(const AD& a, const AD& b) {
  double q = a.v / b.v;
  return mk2(q, a, 1.0 / b.v, b, -q / b.v);
}
inline AD operator-(const AD& a) { return mk1(-a.v, a, -1.0); }
inline AD operator+(const AD& a, double b) { return mk1(a.v + b, a, 1.0); }
inline AD operator+(double a, const AD& b) { return mk1(a + b.v, b, 1.0); }
inline AD operator-(const AD& a, double b) { return mk1(a.v - b, a, 1.0); }
inline AD operator-(double a, const AD& b) { return mk1(a - b.v, b, -1.0); }
inline AD operator*(const AD& a, double b) { return mk1(a.v * b, a, b); }
inline AD operator*(double a, const AD& b) { return mk1(a * b.v, b, a); }
inline AD operator/(const AD& a, double b) { return mk1(a.v / b, a, 1.0 / b); }
inline AD operator/(double a, const AD& b) { double q = a / b.v; return mk1(q, b, -q / b.v); }
inline AD& operator+=(AD& a, const AD& b) { a = a + b; return a; }
inline AD& operator-=(AD& a, const AD& b) { a = a - b; return a; }
inline AD& operator*=(AD& a, const AD& b) { a = a * b; return a; }

inline bool operator<(const AD& a, const AD& b) { return a.v < b.v; }
inline bool operator>(const AD& a, const AD& b) { return a.v > b.v; }
inline bool operator<=(const AD& a, const AD& b) { return a.v <= b.v; }
inline bool operator>=(const AD& a, const AD& b) { return a.v >= b.v; }

inline AD sqrt(const AD& a) { double s = std::sqrt(a.v); return mk1(s, a, s > 0 ? 0.5 / s : 0.0); }
inline AD exp(const AD& a) { double e = std::exp(a.v); return mk1(e, a, e); }
inline AD expm1(const AD& a) { return mk1(std::expm1(a.v), a, std::exp(a.v)); }
inline AD log(const AD& a) { return mk1(std::log(a.v), a, 1.0 / a.v); }
inline AD log1p(const AD& a) { return mk1(std::log1p(a.v), a, 1.0 / (1.0 + a.v)); }
inline AD fabs(const AD& a) { return mk1(std::fabs(a.v), a, a.v < 0 ? -1.0 : 1.0); }
inline AD pow(const AD& a, double p) { double y = std::pow(a.v, p); return mk1(y, a, p * std::pow(a.v, p - 1.0)); }
inline AD atan2(const AD& y, const AD& x) {
  double d = x.v * x.v + y.v * y.v;
  return mk2(std::atan2(y.v, x.v), y, x.v / d, x, -y.v / d);
}

inline double val(double x) { return x; }
inline double val(const AD& x) { return x.v; }

}  // namespace oracle
