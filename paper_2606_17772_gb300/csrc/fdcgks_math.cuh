// Device arithmetic of the FD-CGKS hot path, templated on the compute type R
// (double for the FP64 path, float for the mixed path).  Everything here is
// __host__ __device__ so that the same source can be instantiated on the host
// with an operation-counting scalar to obtain exact algorithmic flop counts.
//
// Paper: "Finite Difference Implementation of a High-order Space-Time Coupled
// Compact Gas-Kinetic Scheme" (Zhao, Chen, Xu).
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define FD_HD __host__ __device__ __forceinline__
#else
#define FD_HD inline
#endif

namespace fdk {

// ---------------------------------------------------------------------------
// scalar helpers (overload points for other scalar types)
// ---------------------------------------------------------------------------
FD_HD double s_sqrt(double x) { return sqrt(x); }
FD_HD float s_sqrt(float x) { return sqrtf(x); }
FD_HD double s_exp(double x) { return exp(x); }
FD_HD float s_exp(float x) { return expf(x); }
FD_HD double s_erfc(double x) { return erfc(x); }
FD_HD float s_erfc(float x) { return erfcf(x); }
FD_HD double s_tanh(double x) { return tanh(x); }
FD_HD float s_tanh(float x) { return tanhf(x); }
FD_HD double s_abs(double x) { return fabs(x); }
FD_HD float s_abs(float x) { return fabsf(x); }
FD_HD double s_min(double a, double b) { return fmin(a, b); }
FD_HD float s_min(float a, float b) { return fminf(a, b); }
FD_HD double s_max(double a, double b) { return fmax(a, b); }
FD_HD float s_max(float a, float b) { return fmaxf(a, b); }
FD_HD double s_expm1(double x) { return expm1(x); }
FD_HD float s_expm1(float x) { return expm1f(x); }

// The FP64 part of the arithmetic (collision time and time coefficients) runs
// in Wide<R>::T: double for both compute types; an instrumented scalar type
// maps to its own wide counterpart.
template <class R> struct Wide { typedef double T; };
template <class R> FD_HD typename Wide<R>::T to_w(R x) { return (typename Wide<R>::T)x; }
template <class R> FD_HD R from_w(typename Wide<R>::T x) { return (R)x; }

// Division in the compute type: IEEE in FP64; in FP32 on the device the
// fast division x * (1/y) with an approximate reciprocal (2 ulp), which is
// below the FP32 path's own error.  Denominators here are bounded away from
// 0 and from 2^126.
FD_HD double s_div(double a, double b) { return a / b; }
FD_HD float s_div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdividef(a, b);
#else
  return a / b;
#endif
}

// erfc(x) given ex2 = exp(-x^2), which the caller has already computed.
// FP64: erfc(|x|) = exp(-x^2) erfcx(|x|) with the library's scaled function
// erfcx, and erfc(x) = 2 - erfc(-x) for x < 0, so the exponential is not
// evaluated twice (1.7 % of the FP64 point kernel's time on the 1024^2
// vortex).  FP32: the library erfcf, which keeps a few ulp of relative
// accuracy where erfc is small, while an absolute-error approximation (e.g.
// Abramowitz & Stegun 7.1.26, |error| <= 1.5e-7, written as a polynomial times
// exp(-x^2)) is off by up to 1e-3 relative there; that inconsistency between
// the half-space moments of the two sides seeded a grid-scale mode across the
// strong shock of the 1000 x 500 viscous shock tube in the mixed path.
FD_HD double s_erfc_e(double x, double ex2) {
#if defined(__CUDA_ARCH__)
  const double r = ex2 * erfcx(fabs(x));
  return x >= 0.0 ? r : 2.0 - r;
#else
  (void)ex2;   // host builds (tests, the flop counter): the C library has no erfcx
  return erfc(x);
#endif
}
FD_HD float s_erfc_e(float x, float ex2) { (void)ex2; return erfcf(x); }

// value at which tanh(z) rounds to exactly 1 in the compute type
template <class R> struct TanhSat;
template <> struct TanhSat<double> { static constexpr double z = 19.5; };
template <> struct TanhSat<float> { static constexpr float z = 9.5f; };

// ---------------------------------------------------------------------------
// constants of one run, in compute precision
// ---------------------------------------------------------------------------
template <class R>
struct GenoK {
  int linear;        // 1: chi = 1 everywhere (linear scheme)
  int r;             // exponent of GENO-IS-linear
  R eps_a, eps_w, C, tanhC, inv_tanhC;
  R d_iface[3];      // ideal weights of the interface sub-stencils (App. C1/C2 order)
  R d_node[3];       // ideal weights of the node sub-stencils (Sec. 3.2 order, central first)
};

template <class R>
struct GasK {
  R K;               // internal degrees of freedom, (4 - 2 gamma)/(gamma - 1)
  R gm1;             // gamma - 1 = 2/(K + 2)
  R c4K;             // 4/(K + 2)
  R prfix;           // 1/Pr - 1 (heat-flux correction)
  double mu, c1, c2, dt, inv_dt;
  R mu_r, c1_r, c2_r, dt_r, inv_dt_r;   // the same in the compute type
};

// dt/tau above which the time coefficients show no cancellation and the FP32
// path evaluates them in FP32 (e^{-dt/tau} < 0.02); at or below it they are
// computed in FP64 with expm1
const double TIME_COEF_FP32_RATIO = 4.0;

template <class R> FD_HD R rpow(R x, int r) { return r == 3 ? x * x * x : x * x; }

// ---------------------------------------------------------------------------
// GENO blend (Sec. 3.2, Eqs. GENO-nonlinear, GENO-IS-linear, GENO-1d-IS-HL)
// of a high-order value/derivative with ENO-weighted sub-stencil values and
// derivatives (the same weights serve both).
// ---------------------------------------------------------------------------
template <class R> struct IsF32 { static constexpr bool v = false; };
template <> struct IsF32<float> { static constexpr bool v = true; };

// FP32 rounding floor of the smoothness indicators: the indicators are
// squares of differences of O(|Q|) values, which FP32 resolves only to about
// u |Q| (u = 2^-24); below (64 u |Q|)^2 they measure rounding, not the data.
// The FP32 path adds it to eps_a, so that data varying by less than about
// 4e-6 of their magnitude count as smooth (FP64: no floor).
template <class R>
FD_HD R geno_floor(R qmax) {
  if (IsF32<R>::v) {
    const R e = R(64.0 * 5.9604644775390625e-8) * qmax;
    return e * e;
  }
  return R(0);
}

template <class R>
FD_HD R geno_chi(const GenoK<R>& g, R IS0, R IS1, R IS2, R floor = R(0)) {
  if (g.linear) return R(1);
  R ISL = s_min(IS0, s_min(IS1, IS2));
  R ISH = s_max(IS0, s_max(IS1, IS2));
  R tau = s_abs(R(0.5) * (IS1 + IS2) - IS0);
  R alpha;
  if (IsF32<R>::v) {
    // FP32: quotient form (the product form could overflow for large IS)
    const R ea = g.eps_a + floor;
    R aH = R(1) + rpow(s_div(tau, ISH + ea), g.r);
    R aL = R(1) + rpow(s_div(tau, ISL + ea), g.r);
    alpha = s_div(R(2) * aH, aH + aL);
  } else {
    // alpha = 2 aH/(aH + aL), aH = 1 + (tau/h)^r, aL = 1 + (tau/l)^r, written
    // over the common denominator h^r l^r; tanh(C alpha) rounds to 1 when
    // C alpha > z_sat, which is tested before dividing.  A floor is added to
    // eps_a only when one is given (the FP64 linearisation of a mixed run)
    R ea = g.eps_a;
    if (floor != R(0)) ea = ea + floor;
    R hr = rpow(ISH + ea, g.r), lr = rpow(ISL + ea, g.r), tr = rpow(tau, g.r);
    R num = R(2) * (hr + tr) * lr;
    R den = (hr + tr) * lr + (lr + tr) * hr;
    if (g.C * num > R(TanhSat<R>::z) * den) return g.inv_tanhC;
    alpha = num / den;
  }
  R z = g.C * alpha;
  // tanh(z) is exactly 1 in this precision above the saturation point
  if (z > R(TanhSat<R>::z)) return g.inv_tanhC;
  return s_tanh(z) * g.inv_tanhC;
}

template <class R>
FD_HD void geno_weights(const GenoK<R>& g, const R d[3], R IS0, R IS1, R IS2, R w[3]) {
  R e0 = IS0 + g.eps_w, e1 = IS1 + g.eps_w, e2 = IS2 + g.eps_w;
  R s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
  if (IsF32<R>::v) {
    R t0 = s_div(d[0], s0), t1 = s_div(d[1], s1), t2 = s_div(d[2], s2);
    R inv = s_div(R(1), t0 + t1 + t2);
    w[0] = t0 * inv;
    w[1] = t1 * inv;
    w[2] = t2 * inv;
  } else {
    // d_k/s_k normalised = d_k P_k / sum_m d_m P_m with P_k the product of the other two s
    R t0 = d[0] * s1 * s2, t1 = d[1] * s0 * s2, t2 = d[2] * s0 * s1;
    R inv = R(1) / (t0 + t1 + t2);
    w[0] = t0 * inv;
    w[1] = t1 * inv;
    w[2] = t2 * inv;
  }
}

// The floor of an FP64 evaluation: (fscale max|Q|)^2 when fscale is given
// (fscale = 64 u reproduces the FP32 path's floor in FP64, for the reverse
// pass of a mixed run), else none; the FP32 path always takes its own.
template <class R>
FD_HD R geno_floor_of(R qmax, R fscale) {
  if (IsF32<R>::v) return geno_floor(qmax);
  if (fscale != R(0)) {
    const R e = fscale * qmax;
    return e * e;
  }
  return R(0);
}

// left and right states at the interface between Q[1] and Q[2] of a 4-point
// line, with averaged gradients Qx[0..3] of the same 4 nodes (Sec. 3.1 Eq.
// 7th-compact-recons; App. C1 and C2).  h: spacing, ih = 1/h; fscale: see
// geno_floor_of.
template <class R>
FD_HD void recon_interface(const GenoK<R>& g, const R Q[4], const R Qx[4], R h, R ih,
                           R& vl, R& dl, R& chil, R& vr, R& dr, R& chir, R fscale = R(0)) {
  const R c64 = R(1.0 / 64.0), c30 = R(1.0 / 30.0);
  // shared high-order derivative (identical for left and right)
  R PHx = -((Q[0] + R(45) * Q[1] - R(45) * Q[2] - Q[3]) * ih + R(9) * (Qx[1] + Qx[2])) * c30;
  R dq12 = (Q[2] - Q[1]) * ih;    // q2x = q3x (left), q2x = q3x (right)
  const R fl = geno_floor_of(s_max(s_max(s_abs(Q[0]), s_abs(Q[1])), s_max(s_abs(Q[2]), s_abs(Q[3]))), fscale);
  // ---- left state (App. C1) ----
  {
    R PH = ((R(7) * Q[0] + R(35) * Q[1] + R(21) * Q[2] + Q[3]) + (Qx[0] + R(22) * Qx[1] - R(7) * Qx[2]) * h) * c64;
    R q0 = (R(-5) * Q[0] + R(9) * Q[1] - R(3) * Qx[0] * h) * R(0.25);
    R q1 = (-Q[0] + R(6) * Q[1] + R(3) * Q[2]) * R(0.125);
    R q2 = (R(3) * Q[1] + R(6) * Q[2] - Q[3]) * R(0.125);
    R qx0 = (R(-3) * Q[0] + R(3) * Q[1]) * ih - R(2) * Qx[0];
    R t = Q[1] - Q[0] - Qx[0] * h;
    R u = R(2) * (Q[1] - Q[0]) - Qx[0] * h;
    R IS0 = R(13.0 / 3.0) * t * t + u * u;
    t = Q[0] - R(2) * Q[1] + Q[2];
    u = Q[2] - Q[0];
    R IS1 = R(13.0 / 12.0) * t * t + R(0.25) * u * u;
    t = Q[1] - R(2) * Q[2] + Q[3];
    u = R(3) * Q[1] - R(4) * Q[2] + Q[3];
    R IS2 = R(13.0 / 12.0) * t * t + R(0.25) * u * u;
    R chi = geno_chi(g, IS0, IS1, IS2, fl);
    chil = chi;
    if (chi == R(1)) {
      vl = PH;
      dl = PHx;
    } else {
      R w[3];
      geno_weights(g, g.d_iface, IS0, IS1, IS2, w);
      R PL = w[0] * q0 + w[1] * q1 + w[2] * q2;
      R PLx = w[0] * qx0 + (w[1] + w[2]) * dq12;
      vl = chi * PH + (R(1) - chi) * PL;
      dl = chi * PHx + (R(1) - chi) * PLx;
    }
  }
  // ---- right state (App. C2, formulas for interface j+1/2) ----
  {
    R PH = ((Q[0] + R(21) * Q[1] + R(35) * Q[2] + R(7) * Q[3]) + (R(7) * Qx[1] - R(22) * Qx[2] - Qx[3]) * h) * c64;
    R q0 = (R(-5) * Q[3] + R(9) * Q[2] + R(3) * Qx[3] * h) * R(0.25);
    R q1 = (-Q[3] + R(6) * Q[2] + R(3) * Q[1]) * R(0.125);
    R q2 = (-Q[0] + R(6) * Q[1] + R(3) * Q[2]) * R(0.125);
    R qx0 = (R(-3) * Q[2] + R(3) * Q[3]) * ih - R(2) * Qx[3];
    R t = Q[2] - Q[3] + Qx[3] * h;
    R u = R(2) * (Q[3] - Q[2]) - Qx[3] * h;
    R IS0 = R(13.0 / 3.0) * t * t + u * u;
    t = Q[1] - R(2) * Q[2] + Q[3];
    u = Q[3] - Q[1];
    R IS1 = R(13.0 / 12.0) * t * t + R(0.25) * u * u;
    t = Q[0] - R(2) * Q[1] + Q[2];
    u = R(3) * Q[2] - R(4) * Q[1] + Q[0];
    R IS2 = R(13.0 / 12.0) * t * t + R(0.25) * u * u;
    R chi = geno_chi(g, IS0, IS1, IS2, fl);
    chir = chi;
    if (chi == R(1)) {
      vr = PH;
      dr = PHx;
    } else {
      R w[3];
      geno_weights(g, g.d_iface, IS0, IS1, IS2, w);
      R PL = w[0] * q0 + w[1] * q1 + w[2] * q2;
      R PLx = w[0] * qx0 + (w[1] + w[2]) * dq12;
      vr = chi * PH + (R(1) - chi) * PL;
      dr = chi * PHx + (R(1) - chi) * PLx;
    }
  }
}

// rho > 0 and 2 E rho > m_x^2 + m_y^2 (positive pressure), both finite: the
// test of the positivity safeguard of the interface states
template <class R>
FD_HD bool physical_state(const R W[4]) {
  return W[0] > R(0) && R(2) * W[3] * W[0] > W[1] * W[1] + W[2] * W[2] && W[0] < R(INFINITY) &&
         W[3] < R(INFINITY);
}

// derivative at the middle node of a 3-point line (Sec. 3.1 Eq.
// 6th-compact-recons; App. C3 with the Sec. 3.2 sub-stencil order)
template <class R>
FD_HD R recon_node(const GenoK<R>& g, const R Q[3], const R Qx[3], R h, R ih, R fscale = R(0)) {
  R PHx = (R(9) * (Q[0] - Q[2]) * ih + (Qx[0] + R(46) * Qx[1] + Qx[2])) * R(1.0 / 30.0);
  R qx0 = (Q[2] - Q[0]) * R(0.5) * ih;                         // central
  R qx1 = R(2) * (Q[1] - Q[0]) * ih - Qx[0];                     // {Q_{j-1}, Q_j, Q_{x,j-1}}
  R qx2 = R(2) * (Q[2] - Q[1]) * ih - Qx[2];                     // {Q_j, Q_{j+1}, Q_{x,j+1}}
  R t = Q[0] - R(2) * Q[1] + Q[2];
  R u = Q[2] - Q[0];
  R IS0 = R(13.0 / 12.0) * t * t + R(0.25) * u * u;
  t = Q[1] - Q[0] - Qx[0] * h;
  u = R(2) * (Q[1] - Q[0]) - Qx[0] * h;
  R IS1 = R(13.0 / 3.0) * t * t + u * u;
  t = Q[2] - Q[1] - Qx[2] * h;
  u = R(2) * (Q[2] - Q[1]) - Qx[2] * h;
  R IS2 = R(13.0 / 3.0) * t * t + u * u;
  R chi = geno_chi(g, IS0, IS1, IS2, geno_floor_of(s_max(s_abs(Q[1]), s_max(s_abs(Q[0]), s_abs(Q[2]))), fscale));
  if (chi == R(1)) return PHx;
  R w[3];
  geno_weights(g, g.d_node, IS0, IS1, IS2, w);
  R PLx = w[0] * qx0 + w[1] * qx1 + w[2] * qx2;
  return chi * PHx + (R(1) - chi) * PLx;
}

// ---------------------------------------------------------------------------
// Maxwellian moments (App. A1).  Tables hold normalized moments <u^n>, <v^n>,
// <xi^{2c}> of g / rho; half-space tables restrict u to one sign.
// ---------------------------------------------------------------------------
template <class R>
struct Maxw {
  R rho, U, V, lam;
  R ir;    // 1/rho
  R p;     // pressure rho/(2 lam)
  R i2l;   // 1/(2 lam) = p/rho
};

// conservative W -> Maxwellian; rho E = rho (U^2 + V^2 + (K+2)/(2 lam))/2,
// so p = (gamma - 1)(rho E - rho (U^2+V^2)/2) and lam = rho/(2 p)
template <class R>
FD_HD Maxw<R> maxw_from_W(const R W[4], R gm1) {
  Maxw<R> g;
  g.rho = W[0];
  g.ir = s_div(R(1), W[0]);
  g.U = W[1] * g.ir;
  g.V = W[2] * g.ir;
  g.p = gm1 * (W[3] - R(0.5) * W[0] * (g.U * g.U + g.V * g.V));
  g.i2l = g.p * g.ir;
  g.lam = s_div(R(0.5), g.i2l);
  return g;
}

const int NT = 7;   // moment orders 0..6

template <class R>
struct Tab {
  R u[NT], v[NT], xi[3];
};

template <class R>
FD_HD void recur(R m, R i2l, R* t) {
  // <c^{n+2}> = m <c^{n+1}> + (n+1)/(2 lam) <c^n>
#pragma unroll
  for (int n = 0; n + 2 < NT; ++n) t[n + 2] = m * t[n + 1] + R(n + 1) * i2l * t[n];
}

// full-space tables of g
template <class R>
FD_HD void tab_full(const Maxw<R>& g, R K, Tab<R>& T) {
  R i2l = g.i2l;
  T.u[0] = R(1); T.u[1] = g.U;
  T.v[0] = R(1); T.v[1] = g.V;
  recur(g.U, i2l, T.u);
  recur(g.V, i2l, T.v);
  T.xi[0] = R(1);
  T.xi[1] = K * i2l;
  T.xi[2] = K * (K + R(2)) * i2l * i2l;
}

// u-half-space tables (sign +1: u > 0, -1: u < 0), sharing v and xi with T
template <class R>
FD_HD void tab_half(const Maxw<R>& g, int sign, const Tab<R>& full, Tab<R>& H) {
  R i2l = g.i2l;
  R sl = s_sqrt(g.lam);
  R isl = sl * (R(2) * i2l);                   // 1/sqrt(lam)
  R e = s_exp(-g.lam * g.U * g.U);
  const R isqpi = R(0.56418958354775628695);   // 1/sqrt(pi)
  H.u[0] = R(0.5) * s_erfc_e(-R(sign) * sl * g.U, e);
  H.u[1] = g.U * H.u[0] + R(sign) * R(0.5) * e * isqpi * isl;
  recur(g.U, i2l, H.u);
#pragma unroll
  for (int n = 0; n < NT; ++n) H.v[n] = full.v[n];
  H.xi[0] = full.xi[0]; H.xi[1] = full.xi[1]; H.xi[2] = full.xi[2];
}

template <int a, int b, int c, class R>
FD_HD R mm(const Tab<R>& T) { return T.u[a] * T.v[b] * T.xi[c]; }

// <u^a v^b xi^{2c} psi>, psi = (1, u, v, (u^2+v^2+xi^2)/2)
template <int a, int b, int c, class R>
FD_HD void mpsi(const Tab<R>& T, R o[4]) {
  o[0] = mm<a, b, c>(T);
  o[1] = mm<a + 1, b, c>(T);
  o[2] = mm<a, b + 1, c>(T);
  o[3] = R(0.5) * (mm<a + 2, b, c>(T) + mm<a, b + 2, c>(T) + mm<a, b, c + 1>(T));
}

// <s u^a v^b psi> for a slope polynomial s = s0 + s1 u + s2 v + s3 psi_4,
// psi_4 = (u^2 + v^2 + xi^2)/2.  The moments factor, <u^p v^q xi^2m> =
// u[p] v[q] xi[m], so with h = s3/2 the slope-weighted moment is
//   <s u^p v^q> = v[q] U(p) + u[p] V(q),
//   U(p) = (s0 + h xi[1]) u[p] + s1 u[p+1] + h u[p+2],  V(q) = s2 v[q+1] + h v[q+2],
//   <s u^p v^q xi^2> = xi[1] (v[q] U'(p) + u[p] V(q)) + h xi[2] u[p] v[q],
//   U'(p) = s0 u[p] + s1 u[p+1] + h u[p+2],
// and the psi components are <s u^a v^b (1, u, v)> and half the sum of
// <s u^(a+2) v^b>, <s u^a v^(b+2)> and <s u^a v^b xi^2>.
template <int p, class R>
FD_HD R slope_u(const Tab<R>& T, R c0, R s1, R h) { return c0 * T.u[p] + s1 * T.u[p + 1] + h * T.u[p + 2]; }
template <int q, class R>
FD_HD R slope_v(const Tab<R>& T, R s2, R h) { return s2 * T.v[q + 1] + h * T.v[q + 2]; }
template <int p, int q, class R>
FD_HD R slope_uv(const Tab<R>& T, R c0, const R s[4], R h) {
  return T.v[q] * slope_u<p>(T, c0, s[1], h) + T.u[p] * slope_v<q>(T, s[2], h);
}

template <int a, int b, class R>
FD_HD void mslope(const Tab<R>& T, const R s[4], R o[4]) {
  const R h = R(0.5) * s[3];
  const R c0 = s[0] + h * T.xi[1];
  const R sx = T.xi[1] * (T.v[b] * slope_u<a>(T, s[0], s[1], h) + T.u[a] * slope_v<b>(T, s[2], h)) +
               h * T.xi[2] * T.u[a] * T.v[b];
  o[0] = slope_uv<a, b>(T, c0, s, h);
  o[1] = slope_uv<a + 1, b>(T, c0, s, h);
  o[2] = slope_uv<a, b + 1>(T, c0, s, h);
  o[3] = R(0.5) * (slope_uv<a + 2, b>(T, c0, s, h) + slope_uv<a, b + 2>(T, c0, s, h) + sx);
}

// slope s with <s psi> = r (r = dW / rho), closed form of the 4x4 moment system
template <class R>
FD_HD void slope_solve(const Maxw<R>& g, R K, R c4K, const R r[4], R s[4]) {
  R q = g.U * g.U + g.V * g.V + (K + R(2)) * g.i2l;
  R Ah = r[1] - g.U * r[0];
  R Ch = r[2] - g.V * r[0];
  R B = R(2) * r[3] - q * r[0];
  s[3] = c4K * g.lam * g.lam * (B - R(2) * g.U * Ah - R(2) * g.V * Ch);
  s[2] = R(2) * g.lam * Ch - g.V * s[3];
  s[1] = R(2) * g.lam * Ah - g.U * s[3];
  s[0] = r[0] - g.U * s[1] - g.V * s[2] - R(0.5) * s[3] * q;
}

// heat flux of the energy equation relative to (U0, V0) from the moments
// F = int u psi f and W = int psi f of one distribution (x-normal)
template <class R>
FD_HD R heat_flux_x(const R F[4], const R W[4], R U0, R V0) {
  return F[3] - U0 * W[3] - U0 * F[1] - V0 * F[2] + (R(1.5) * U0 * U0 + R(0.5) * V0 * V0) * W[1] +
         U0 * V0 * W[2] - R(0.5) * U0 * (U0 * U0 + V0 * V0) * W[0];
}
// same for the y-normal flux G = int v psi f
template <class R>
FD_HD R heat_flux_y(const R G[4], const R W[4], R U0, R V0) {
  return G[3] - V0 * W[3] - V0 * G[2] - U0 * G[1] + (R(1.5) * V0 * V0 + R(0.5) * U0 * U0) * W[2] +
         U0 * V0 * W[1] - R(0.5) * V0 * (U0 * U0 + V0 * V0) * W[0];
}

// ---------------------------------------------------------------------------
// Time coefficients of the interface distribution, integrated over
// [0, delta] for delta = dt/2 and dt and fitted to f^n + t f_t^n (App. A1).
// Always FP64: the coefficients cancel when dt/tau is small.
// ---------------------------------------------------------------------------
template <class TW>
struct TimeCoef {
  TW cn[6], ct[6];
  TW E, e1;   // exp(-dt/tau), 1 - exp(-dt/tau)
};

// integrals over [0, d] of the equilibrium coefficients c1..c3 of f(0,t);
// the initial-data coefficients follow from c1 + c4 = 1, c2 + c5 = -tau,
// c3 + c6 = t - tau
template <class TW>
FD_HD void time_integrals_d(TW tau, TW d, TW E, TW e1, TW C[3]) {
  C[0] = d - tau * e1;
  C[1] = -tau * d * (TW(1) + E) + TW(2) * tau * tau * e1;
  C[2] = TW(0.5) * d * d - tau * d + tau * tau * e1;
}

template <class TW>
FD_HD TimeCoef<TW> time_coef(TW tau, TW dt, TW inv_dt) {
  TimeCoef<TW> t;
  // one transcendental: em = exp(-dt/(2 tau)) - 1, then
  // exp(-dt/tau) - 1 = em (em + 2) without cancellation
  TW em = s_expm1(-TW(0.5) * dt / tau);
  TW Eh = TW(1) + em, e1h = -em;
  t.E = Eh * Eh;
  t.e1 = -em * (em + TW(2));
  TW Ch[3], Cf[3];
  time_integrals_d(tau, TW(0.5) * dt, Eh, e1h, Ch);
  time_integrals_d(tau, dt, t.E, t.e1, Cf);
  for (int k = 0; k < 3; ++k) {
    // linear-in-time fit of App. A1: f^n = (4 fbar(dt/2) - fbar(dt))/dt,
    // f_t^n = 4 (fbar(dt) - 2 fbar(dt/2))/dt^2
    t.cn[k] = (TW(4) * Ch[k] - Cf[k]) * inv_dt;
    t.ct[k] = TW(4) * (Cf[k] - TW(2) * Ch[k]) * inv_dt * inv_dt;
  }
  // fits of c4..c6: the fit of (c1 + c4) = 1 is 1 (value) and 0 (slope),
  // of (c2 + c5) = -tau is -tau and 0, of (c3 + c6) = t - tau is -tau and 1
  t.cn[3] = TW(1) - t.cn[0];
  t.ct[3] = -t.ct[0];
  t.cn[4] = -tau - t.cn[1];
  t.ct[4] = -t.ct[1];
  t.cn[5] = -tau - t.cn[2];
  t.ct[5] = TW(1) - t.ct[2];
  return t;
}

// ---------------------------------------------------------------------------
// Interface solve with x as the normal (App. A1-A2, Eq. eq:W-model).
// Inputs: left/right reconstructed states, their normal (x) derivatives and
// the shared tangential (y) derivative.  want_n = false skips the outputs
// that the second S2O4 stage does not use (F^, W^ values).
// ---------------------------------------------------------------------------
template <class R>
struct IfaceOut {
  R F[4], Ft[4], Wl[4], Wr[4], Wlt[4], Wrt[4];
};

template <class R>
FD_HD void iface_solve_x(const GasK<R>& gas, const R Wl[4], const R Wr[4], const R Wln[4], const R Wrn[4],
                         const R Wt[4], bool want_n, IfaceOut<R>& o) {
  const R K = gas.K;
  Maxw<R> gl = maxw_from_W(Wl, gas.gm1), gr = maxw_from_W(Wr, gas.gm1);
  Tab<R> Tl, Tr, Tlp, Trn;
  tab_full(gl, K, Tl);
  tab_full(gr, K, Tr);
  tab_half(gl, +1, Tl, Tlp);
  tab_half(gr, -1, Tr, Trn);

  // equilibrium state from the particles crossing the interface
  R W0[4], t4[4];
  mpsi<0, 0, 0>(Tlp, W0);
  mpsi<0, 0, 0>(Trn, t4);
#pragma unroll
  for (int k = 0; k < 4; ++k) W0[k] = gl.rho * W0[k] + gr.rho * t4[k];
  Maxw<R> g0 = maxw_from_W(W0, gas.gm1);
  Tab<R> T0;
  tab_full(g0, K, T0);

  // slopes (x: normal, y: tangential)
  R al[4], bl[4], ar[4], br[4], a0[4], b0[4], r[4];
  R irl = gl.ir, irr = gr.ir, ir0 = g0.ir;
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wln[k] * irl;
  slope_solve(gl, K, gas.c4K, r, al);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wt[k] * irl;
  slope_solve(gl, K, gas.c4K, r, bl);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wrn[k] * irr;
  slope_solve(gr, K, gas.c4K, r, ar);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wt[k] * irr;
  slope_solve(gr, K, gas.c4K, r, br);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = R(0.5) * (Wln[k] + Wrn[k]) * ir0;
  slope_solve(g0, K, gas.c4K, r, a0);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wt[k] * ir0;
  slope_solve(g0, K, gas.c4K, r, b0);

  // time slopes from compatibility <(a u + b v + A) psi> = 0
  R Al[4], Ar[4], A0[4], rl[4], rr[4], r0[4], x1[4], x2[4];
  mslope<1, 0>(Tl, al, x1);
  mslope<0, 1>(Tl, bl, x2);
#pragma unroll
  for (int k = 0; k < 4; ++k) rl[k] = -(x1[k] + x2[k]);
  slope_solve(gl, K, gas.c4K, rl, Al);
  mslope<1, 0>(Tr, ar, x1);
  mslope<0, 1>(Tr, br, x2);
#pragma unroll
  for (int k = 0; k < 4; ++k) rr[k] = -(x1[k] + x2[k]);
  slope_solve(gr, K, gas.c4K, rr, Ar);
  mslope<1, 0>(T0, a0, x1);
  mslope<0, 1>(T0, b0, x2);
#pragma unroll
  for (int k = 0; k < 4; ++k) r0[k] = -(x1[k] + x2[k]);
  slope_solve(g0, K, gas.c4K, r0, A0);

  // collision time and time coefficients: FP64 with expm1 where they cancel
  // (dt/tau small); in the FP32 path, FP32 where dt/tau > 4
  typedef typename Wide<R>::T TW;
  R cn[6], ct[6], E, e1;
  R ip0r = R(2) * g0.lam * g0.ir;              // 1/p0
  R taur = gas.c1_r * gas.dt_r + gas.mu_r * ip0r + gas.c2_r * gas.dt_r * s_div(s_abs(gl.p - gr.p), gl.p + gr.p);
  if (IsF32<R>::v && gas.dt_r > R(TIME_COEF_FP32_RATIO) * taur) {
    TimeCoef<R> tc = time_coef(taur, gas.dt_r, gas.inv_dt_r);
#pragma unroll
    for (int k = 0; k < 6; ++k) { cn[k] = tc.cn[k]; ct[k] = tc.ct[k]; }
    E = tc.E;
    e1 = tc.e1;
  } else {
    TW pl = to_w(gl.p), pr = to_w(gr.p);
    TW ip0 = to_w(ip0r);
    TW dtw = TW(gas.dt);
    TW tau = TW(gas.c1) * dtw + TW(gas.mu) * ip0 + TW(gas.c2) * dtw * s_abs(pl - pr) / (pl + pr);
    TimeCoef<TW> tc = time_coef(tau, dtw, TW(gas.inv_dt));
#pragma unroll
    for (int k = 0; k < 6; ++k) { cn[k] = from_w<R>(tc.cn[k]); ct[k] = from_w<R>(tc.ct[k]); }
    E = from_w<R>(tc.E);
    e1 = from_w<R>(tc.e1);
  }

  // moment vectors of the six basis terms, flux (u psi) and W (psi)
  R F[4], Ftt[4], We[4], Wet[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { F[k] = R(0); Ftt[k] = R(0); We[k] = R(0); Wet[k] = R(0); }
  auto acc = [&](int kk, const R mf[4], const R mw[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      F[k] += cn[kk] * mf[k];
      Ftt[k] += ct[kk] * mf[k];
      We[k] += cn[kk] * mw[k];
      Wet[k] += ct[kk] * mw[k];
    }
  };
  R mf[4], mw[4], y1[4], y2[4];
  // 1: g0
  mpsi<1, 0, 0>(T0, mf);
  mpsi<0, 0, 0>(T0, mw);
#pragma unroll
  for (int k = 0; k < 4; ++k) { mf[k] *= g0.rho; mw[k] *= g0.rho; }
  acc(0, mf, mw);
  // 2: (a0 u + b0 v) g0
  mslope<2, 0>(T0, a0, x1);
  mslope<1, 1>(T0, b0, x2);
#pragma unroll
  for (int k = 0; k < 4; ++k) { mf[k] = g0.rho * (x1[k] + x2[k]); mw[k] = -g0.rho * r0[k]; }
  acc(1, mf, mw);
  // 3: A0 g0; int psi A0 g0 = rho0 r0 by construction of A0 (compatibility)
  mslope<1, 0>(T0, A0, x1);
#pragma unroll
  for (int k = 0; k < 4; ++k) { mf[k] = g0.rho * x1[k]; mw[k] = g0.rho * r0[k]; }
  acc(2, mf, mw);
  // 4: gl H(u) + gr (1 - H(u))
  mpsi<1, 0, 0>(Tlp, x1);
  mpsi<1, 0, 0>(Trn, x2);
#pragma unroll
  for (int k = 0; k < 4; ++k) { mf[k] = gl.rho * x1[k] + gr.rho * x2[k]; mw[k] = W0[k]; }
  acc(3, mf, mw);
  // 5: (a u + b v) g on each side
  mslope<2, 0>(Tlp, al, x1);
  mslope<1, 1>(Tlp, bl, x2);
  mslope<2, 0>(Trn, ar, y1);
  mslope<1, 1>(Trn, br, y2);
#pragma unroll
  for (int k = 0; k < 4; ++k) mf[k] = gl.rho * (x1[k] + x2[k]) + gr.rho * (y1[k] + y2[k]);
  mslope<1, 0>(Tlp, al, x1);
  mslope<0, 1>(Tlp, bl, x2);
  mslope<1, 0>(Trn, ar, y1);
  mslope<0, 1>(Trn, br, y2);
#pragma unroll
  for (int k = 0; k < 4; ++k) mw[k] = gl.rho * (x1[k] + x2[k]) + gr.rho * (y1[k] + y2[k]);
  acc(4, mf, mw);
  // 6: A g on each side
  mslope<1, 0>(Tlp, Al, x1);
  mslope<1, 0>(Trn, Ar, y1);
  mslope<0, 0>(Tlp, Al, x2);
  mslope<0, 0>(Trn, Ar, y2);
#pragma unroll
  for (int k = 0; k < 4; ++k) { mf[k] = gl.rho * x1[k] + gr.rho * y1[k]; mw[k] = gl.rho * x2[k] + gr.rho * y2[k]; }
  acc(5, mf, mw);

  // Prandtl-number correction of the energy flux
  F[3] += gas.prfix * heat_flux_x(F, We, g0.U, g0.V);
  Ftt[3] += gas.prfix * heat_flux_x(Ftt, Wet, g0.U, g0.V);

  // interface flow variables, Eq. (eq:W-model) with tau_0 = tau; the one-sided
  // time derivatives are W_t = -rho <(a u + b v) psi> = rho * (compatibility rhs)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    o.Ft[k] = Ftt[k];
    o.Wlt[k] = e1 * Wet[k] + E * gl.rho * rl[k];
    o.Wrt[k] = e1 * Wet[k] + E * gr.rho * rr[k];
    if (want_n) {
      o.F[k] = F[k];
      o.Wl[k] = e1 * We[k] + E * Wl[k];
      o.Wr[k] = e1 * We[k] + E * Wr[k];
    }
  }
}

// y-normal solve through the x <-> y transposition of the equations; the
// transposition is a register select, so one copy of the x-normal solve
// serves both normals
template <class R>
FD_HD void swap_uv(const R a[4], R b[4], bool sw) {
  b[0] = a[0];
  b[1] = sw ? a[2] : a[1];
  b[2] = sw ? a[1] : a[2];
  b[3] = a[3];
}

template <class R>
FD_HD void iface_solve(const GasK<R>& gas, int normal, const R Wl[4], const R Wr[4], const R Wln[4],
                       const R Wrn[4], const R Wt[4], bool want_n, IfaceOut<R>& o) {
  const bool sw = normal != 0;
  R a[4], b[4], c[4], d[4], e[4];
  swap_uv(Wl, a, sw); swap_uv(Wr, b, sw); swap_uv(Wln, c, sw); swap_uv(Wrn, d, sw); swap_uv(Wt, e, sw);
  IfaceOut<R> t;
  iface_solve_x(gas, a, b, c, d, e, want_n, t);
  swap_uv(t.Ft, o.Ft, sw); swap_uv(t.Wlt, o.Wlt, sw); swap_uv(t.Wrt, o.Wrt, sw);
  if (want_n) { swap_uv(t.F, o.F, sw); swap_uv(t.Wl, o.Wl, sw); swap_uv(t.Wr, o.Wr, sw); }
}

// ---------------------------------------------------------------------------
// Nodal flux from smooth local data (Sec. 2.1): f = g(1 - tau(a u + b v + A)),
// f_t = A g.  Outputs x-flux F, y-flux G and their time derivatives;
// want_n = false computes the time derivatives only (F, G are set to 0): the
// second S2O4 stage uses no other nodal output.
// ---------------------------------------------------------------------------
template <class R>
FD_HD void nodal_flux(const GasK<R>& gas, const R W[4], const R Wx[4], const R Wy[4], R F[4], R G[4], R Ft[4],
                      R Gt[4], bool want_n = true) {
  const R K = gas.K;
  Maxw<R> g = maxw_from_W(W, gas.gm1);
  Tab<R> T;
  tab_full(g, K, T);
  R a[4], b[4], A[4], r[4], ir = g.ir;
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wx[k] * ir;
  slope_solve(g, K, gas.c4K, r, a);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = Wy[k] * ir;
  slope_solve(g, K, gas.c4K, r, b);
  R x1[4], x2[4], Wt[4];
  mslope<1, 0>(T, a, x1);
  mslope<0, 1>(T, b, x2);
#pragma unroll
  for (int k = 0; k < 4; ++k) r[k] = -(x1[k] + x2[k]);
  slope_solve(g, K, gas.c4K, r, A);
#pragma unroll
  for (int k = 0; k < 4; ++k) Wt[k] = g.rho * r[k];   // int psi A g
  R tau = gas.c1_r * gas.dt_r + gas.mu_r * (R(2) * g.lam * g.ir);   // c1 dt + mu/p

  R e0[4], ea[4], eb[4], eA[4];
  // time derivatives f_t = A g
  mslope<1, 0>(T, A, eA);
#pragma unroll
  for (int k = 0; k < 4; ++k) Ft[k] = g.rho * eA[k];
  mslope<0, 1>(T, A, eA);
#pragma unroll
  for (int k = 0; k < 4; ++k) Gt[k] = g.rho * eA[k];
  // Prandtl correction; int psi f^n = W (compatibility), int psi f_t = Wt
  Ft[3] += gas.prfix * heat_flux_x(Ft, Wt, g.U, g.V);
  Gt[3] += gas.prfix * heat_flux_y(Gt, Wt, g.U, g.V);
  if (!want_n) {
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = G[k] = R(0);
    return;
  }
  // x-flux
  mpsi<1, 0, 0>(T, e0);
  mslope<2, 0>(T, a, ea);
  mslope<1, 1>(T, b, eb);
  mslope<1, 0>(T, A, eA);
#pragma unroll
  for (int k = 0; k < 4; ++k) F[k] = g.rho * (e0[k] - tau * (ea[k] + eb[k] + eA[k]));
  // y-flux
  mpsi<0, 1, 0>(T, e0);
  mslope<1, 1>(T, a, ea);
  mslope<0, 2>(T, b, eb);
  mslope<0, 1>(T, A, eA);
#pragma unroll
  for (int k = 0; k < 4; ++k) G[k] = g.rho * (e0[k] - tau * (ea[k] + eb[k] + eA[k]));
  F[3] += gas.prfix * heat_flux_x(F, W, g.U, g.V);
  G[3] += gas.prfix * heat_flux_y(G, W, g.U, g.V);
}

// ---------------------------------------------------------------------------
// Compact numerical flux (Eqs. fd-conservative-flux, -flux-1, -flux-2).
// Fi = {F_{j-1/2}, F_{j+1/2}, F_{j+3/2}}, Fn0 = F_j, Fn1 = F_{j+1}
// ---------------------------------------------------------------------------
template <class R>
FD_HD R compact_flux(int variant, R chi, R Fim, R Fi0, R Fip, R Fn0, R Fn1) {
  R Fbar = (Fim + R(46) * Fi0 + Fip - R(9) * (Fn0 + Fn1)) * R(1.0 / 30.0);
  R Flow = variant == 62 ? Fi0 : (R(8) * Fi0 - Fn0 - Fn1) * R(1.0 / 6.0);
  return (R(1) - chi) * Flow + chi * Fbar;
}

}  // namespace fdk
