// Forward-mode dual numbers over FP64: test instrumentation for the
// hand-written reverse passes of csrc/fdcgks_reverse.cuh.
//
// Dual<N> carries a value and N directional derivatives.  Instantiating the
// device arithmetic of fdcgks_math.cuh (reconstruction, kinetic solves,
// nodal flux) on Dual<N> evaluates, besides the value, the derivatives of
// every output with respect to N seeded inputs: the Jacobian columns the CPU
// tests contract with output adjoints to check the reverse passes.  Branches
// (GENO saturation, the positivity safeguard) follow the values, so the
// derivative is that of the branch the forward step took.
#pragma once

#include "fdcgks_math.cuh"

namespace fdk {

template <int N>
struct Dual {
  double v;
  double d[N];
  FD_HD Dual() : v(0.0) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.0;
  }
  FD_HD Dual(double x) : v(x) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.0;
  }
  FD_HD Dual(int x) : Dual((double)x) {}
  FD_HD Dual(float x) : Dual((double)x) {}

  friend FD_HD Dual operator+(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
  }
  friend FD_HD Dual operator-(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
  }
  friend FD_HD Dual operator-(const Dual& a) {
    Dual r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
  }
  // A zero tangent times an infinite partial derivative is taken as 0 (a
  // structural zero), not NaN: the kinetic time coefficients at a vanishing
  // collision time divide by tau, but are exponentially flat there.
  friend FD_HD Dual operator*(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; ++k)
      r.d[k] = (a.d[k] == 0.0 ? 0.0 : a.d[k] * b.v) + (b.d[k] == 0.0 ? 0.0 : a.v * b.d[k]);
    return r;
  }
  friend FD_HD Dual operator/(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double num = a.d[k] - (b.d[k] == 0.0 ? 0.0 : r.v * b.d[k]);
      r.d[k] = num == 0.0 ? 0.0 : num * ib;
    }
    return r;
  }
  friend FD_HD Dual& operator+=(Dual& a, const Dual& b) { return a = a + b; }
  friend FD_HD Dual& operator-=(Dual& a, const Dual& b) { return a = a - b; }
  friend FD_HD Dual& operator*=(Dual& a, const Dual& b) { return a = a * b; }
  friend FD_HD Dual& operator/=(Dual& a, const Dual& b) { return a = a / b; }
  friend FD_HD bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
  friend FD_HD bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
  friend FD_HD bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
  friend FD_HD bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
  friend FD_HD bool operator==(const Dual& a, const Dual& b) { return a.v == b.v; }
  friend FD_HD bool operator!=(const Dual& a, const Dual& b) { return a.v != b.v; }
};

// f(a) with value fv and derivative df/da = dv (a zero factor wins, as above)
template <int N>
FD_HD Dual<N> dual_chain(const Dual<N>& a, double fv, double dv) {
  Dual<N> r;
  r.v = fv;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] == 0.0 || dv == 0.0) ? 0.0 : a.d[k] * dv;
  return r;
}

template <int N> FD_HD Dual<N> s_sqrt(const Dual<N>& a) {
  const double v = sqrt(a.v);
  return dual_chain(a, v, 0.5 / v);
}
template <int N> FD_HD Dual<N> s_exp(const Dual<N>& a) {
  const double v = exp(a.v);
  return dual_chain(a, v, v);
}
// d/dx erfc(x) = -(2/sqrt(pi)) exp(-x^2)
template <int N> FD_HD Dual<N> s_erfc(const Dual<N>& a) {
  return dual_chain(a, erfc(a.v), -1.1283791670955126 * exp(-a.v * a.v));
}
template <int N> FD_HD Dual<N> s_erfc_e(const Dual<N>& x, const Dual<N>& ex2) {
  return dual_chain(x, erfc(x.v), -1.1283791670955126 * ex2.v);
}
template <int N> FD_HD Dual<N> s_tanh(const Dual<N>& a) {
  const double v = tanh(a.v);
  return dual_chain(a, v, 1.0 - v * v);
}
template <int N> FD_HD Dual<N> s_expm1(const Dual<N>& a) {
  const double v = expm1(a.v);
  return dual_chain(a, v, v + 1.0);
}
// |a| at a = 0: derivative 0, the symmetric choice (what a central difference sees)
template <int N> FD_HD Dual<N> s_abs(const Dual<N>& a) { return a.v < 0.0 ? -a : a.v > 0.0 ? a : Dual<N>(0.0); }
// min/max at a tie: the mean of the two derivatives, again what a central
// difference sees (ties are exact on symmetric data, e.g. mirror-image
// GENO sub-stencils about a symmetry line of the flow)
template <int N> FD_HD Dual<N> dual_mean(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = 0.5 * (a.d[k] + b.d[k]);
  return r;
}
template <int N> FD_HD Dual<N> s_min(const Dual<N>& a, const Dual<N>& b) {
  return b.v < a.v ? b : a.v < b.v ? a : dual_mean(a, b);
}
template <int N> FD_HD Dual<N> s_max(const Dual<N>& a, const Dual<N>& b) {
  return b.v > a.v ? b : a.v > b.v ? a : dual_mean(a, b);
}
template <int N> FD_HD Dual<N> s_div(const Dual<N>& a, const Dual<N>& b) { return a / b; }

template <int N> struct TanhSat<Dual<N>> { static constexpr double z = 19.5; };
template <int N> struct Wide<Dual<N>> { typedef Dual<N> T; };

// run constants of the FP64 path as constants (zero derivatives) of Dual<N>
template <int N>
FD_HD GenoK<Dual<N>> dual_geno(const GenoK<double>& g) {
  GenoK<Dual<N>> r;
  r.linear = g.linear;
  r.r = g.r;
  r.eps_a = g.eps_a;
  r.eps_w = g.eps_w;
  r.C = g.C;
  r.tanhC = g.tanhC;
  r.inv_tanhC = g.inv_tanhC;
  for (int k = 0; k < 3; ++k) {
    r.d_iface[k] = g.d_iface[k];
    r.d_node[k] = g.d_node[k];
  }
  return r;
}

template <int N>
FD_HD GasK<Dual<N>> dual_gas(const GasK<double>& g) {
  GasK<Dual<N>> r;
  r.K = g.K;
  r.gm1 = g.gm1;
  r.c4K = g.c4K;
  r.prfix = g.prfix;
  r.mu = g.mu;
  r.c1 = g.c1;
  r.c2 = g.c2;
  r.dt = g.dt;
  r.inv_dt = g.inv_dt;
  r.mu_r = g.mu_r;
  r.c1_r = g.c1_r;
  r.c2_r = g.c2_r;
  r.dt_r = g.dt_r;
  r.inv_dt_r = g.inv_dt_r;
  return r;
}

}  // namespace fdk
