// Algorithmic operation counts of the FD-CGKS device arithmetic.
//
// Instrumentation: fdcgks_math.cuh is instantiated on the host with a scalar
// type that tallies the floating-point operations it performs, on sampled
// real inputs, so that the throughput benchmark can quote algorithmic flops
// per node update.  Convention: add, sub, mul = 1 flop each (a fused
// multiply-add is 2), div = 1, sqrt = 1, and each call of exp, erfc, tanh or
// expm1 = 1 (tallied separately as well).  Sign flips, abs, min, max and
// comparisons count 0.
//
// Operations are hash-consed: an operation whose opcode and operand values'
// identities were already seen (commutative operands in either order) is a
// common subexpression and is not counted again, and multiplying by the
// constant 1 or adding the constant 0 is free.  The count is thus that of the
// arithmetic after common-subexpression elimination, which is what a
// compiler emits for the fully unrolled source.  The library and its Python
// binding never call this.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <unordered_map>

namespace cnt {
struct Counts {
  long long add, mul, div, sqrt_, exp_, erfc_, tanh_, expm1_;
};
Counts c64, c32;
template <int P> Counts& C() { return P == 64 ? c64 : c32; }

// value identities and the table of operations already performed
uint32_t next_id = 1;
std::unordered_map<uint64_t, uint32_t> const_ids;     // constant bit pattern -> id
std::unordered_map<uint64_t, uint32_t> op_ids;        // (op, a, b) -> result id
std::unordered_map<uint64_t, double> op_vals;
uint32_t one64 = 0, zero64 = 0;
void reset_ids() {
  next_id = 1;
  const_ids.clear();
  op_ids.clear();
  op_vals.clear();
}
uint32_t const_id(double v, int P) {
  uint64_t bits;
  std::memcpy(&bits, &v, sizeof(bits));
  bits ^= (uint64_t)P << 63 >> 1;   // distinct tables per precision
  auto it = const_ids.find(bits);
  if (it != const_ids.end()) return it->second;
  uint32_t id = next_id++;
  const_ids[bits] = id;
  return id;
}
}  // namespace cnt

template <int P>
struct CN {
  typedef typename std::conditional<P == 64, double, float>::type V;
  V v;
  uint32_t id;   // 0: not yet identified (treated as a constant of its value)
  CN() : v(0), id(0) {}
  CN(double x) : v((V)x), id(0) {}
  CN(float x) : v((V)x), id(0) {}
  CN(int x) : v((V)x), id(0) {}
  template <int Q> explicit CN(const CN<Q>& o) : v((V)o.v), id(0) {}
  uint32_t ident() const { return id ? id : cnt::const_id((double)v, P); }
  bool is_const(double c) const { return id == 0 && (double)v == c; }
};
typedef CN<64> CD;
typedef CN<32> CF;

enum { OP_ADD = 1, OP_SUB, OP_MUL, OP_DIV, OP_SQRT, OP_EXP, OP_ERFC, OP_TANH, OP_EXPM1, OP_ABS };

// result of an operation: counted only the first time (op, operands) is seen
template <int P>
CN<P> apply(int op, uint32_t a, uint32_t b, typename CN<P>::V value, long long& counter) {
  if ((op == OP_ADD || op == OP_MUL) && a > b) { uint32_t t = a; a = b; b = t; }
  uint64_t key = ((uint64_t)op << 58) ^ ((uint64_t)(P == 64) << 57) ^ ((uint64_t)a << 28) ^ (uint64_t)b;
  CN<P> r;
  r.v = value;
  auto it = cnt::op_ids.find(key);
  if (it != cnt::op_ids.end()) {
    r.id = it->second;
    return r;
  }
  counter++;
  r.id = cnt::next_id++;
  cnt::op_ids[key] = r.id;
  return r;
}

template <int P> CN<P> operator+(const CN<P>& a, const CN<P>& b) {
  if (a.is_const(0.0)) return b;
  if (b.is_const(0.0)) return a;
  return apply<P>(OP_ADD, a.ident(), b.ident(), a.v + b.v, cnt::C<P>().add);
}
template <int P> CN<P> operator-(const CN<P>& a, const CN<P>& b) {
  if (b.is_const(0.0)) return a;
  return apply<P>(OP_SUB, a.ident(), b.ident(), a.v - b.v, cnt::C<P>().add);
}
template <int P> CN<P> operator*(const CN<P>& a, const CN<P>& b) {
  if (a.is_const(1.0)) return b;
  if (b.is_const(1.0)) return a;
  return apply<P>(OP_MUL, a.ident(), b.ident(), a.v * b.v, cnt::C<P>().mul);
}
template <int P> CN<P> operator/(const CN<P>& a, const CN<P>& b) {
  if (b.is_const(1.0)) return a;
  return apply<P>(OP_DIV, a.ident(), b.ident(), a.v / b.v, cnt::C<P>().div);
}
template <int P> CN<P>& operator+=(CN<P>& a, const CN<P>& b) { a = a + b; return a; }
template <int P> CN<P>& operator*=(CN<P>& a, const CN<P>& b) { a = a * b; return a; }
template <int P> CN<P> operator-(const CN<P>& a) {
  // a sign flip is free; it still is a distinct value for later operations
  long long dummy = 0;
  CN<P> r = apply<P>(OP_SUB, 0, a.ident(), -a.v, dummy);
  return r;
}
template <int P> bool operator>(const CN<P>& a, const CN<P>& b) { return a.v > b.v; }
template <int P> bool operator<(const CN<P>& a, const CN<P>& b) { return a.v < b.v; }
template <int P> bool operator==(const CN<P>& a, const CN<P>& b) { return a.v == b.v; }
template <int P> bool operator!=(const CN<P>& a, const CN<P>& b) { return a.v != b.v; }

namespace fdk {
template <int P> CN<P> s_sqrt(CN<P> x) { return apply<P>(OP_SQRT, x.ident(), 0, std::sqrt(x.v), cnt::C<P>().sqrt_); }
template <int P> CN<P> s_exp(CN<P> x) { return apply<P>(OP_EXP, x.ident(), 0, std::exp(x.v), cnt::C<P>().exp_); }
template <int P> CN<P> s_erfc(CN<P> x) { return apply<P>(OP_ERFC, x.ident(), 0, std::erfc(x.v), cnt::C<P>().erfc_); }
template <int P> CN<P> s_tanh(CN<P> x) { return apply<P>(OP_TANH, x.ident(), 0, std::tanh(x.v), cnt::C<P>().tanh_); }
template <int P> CN<P> s_expm1(CN<P> x) {
  return apply<P>(OP_EXPM1, x.ident(), 0, std::expm1(x.v), cnt::C<P>().expm1_);
}
template <int P> CN<P> s_abs(CN<P> x) {
  long long dummy = 0;
  return apply<P>(OP_ABS, x.ident(), 0, std::fabs(x.v), dummy);
}
template <int P> CN<P> s_min(CN<P> a, CN<P> b) { return a.v < b.v ? a : b; }
template <int P> CN<P> s_max(CN<P> a, CN<P> b) { return a.v > b.v ? a : b; }
template <int P> CN<P> s_div(CN<P> a, CN<P> b) { return a / b; }
// erfc given exp(-x^2): one erfc in either precision (the kernels call the
// library's erfcx or erfcf)
inline CD s_erfc_e(CD x, CD e) { (void)e; return s_erfc(x); }
inline CF s_erfc_e(CF x, CF e) { (void)e; return s_erfc(x); }
}  // namespace fdk

#include "fdcgks_math.cuh"

namespace fdk {
template <> struct TanhSat<CD> { static constexpr double z = 19.5; };
template <> struct IsF32<CF> { static constexpr bool v = true; };
template <> struct TanhSat<CF> { static constexpr float z = 9.5f; };
template <> struct Wide<CD> { typedef CD T; };
template <> struct Wide<CF> { typedef CD T; };
template <> inline CD to_w<CD>(CD x) { return x; }
template <> inline CD to_w<CF>(CF x) {
  long long dummy = 0;
  return apply<64>(OP_ABS + 1, x.ident(), 1, (double)x.v, dummy);
}
template <> inline CD from_w<CD>(CD x) { return x; }
template <> inline CF from_w<CF>(CD x) {
  long long dummy = 0;
  return apply<32>(OP_ABS + 2, x.ident(), 1, (float)x.v, dummy);
}
}  // namespace fdk

using namespace fdk;

namespace {

template <class R>
GenoK<R> geno_of(int variant) {
  GenoK<R> g;
  g.linear = variant == 2;
  g.C = R(20.0);
  g.tanhC = R(std::tanh(20.0));
  g.inv_tanhC = R(1.0 / std::tanh(20.0));
  g.eps_w = R(1e-6);
  if (variant == 1) {
    g.r = 3; g.eps_a = R(1e-15);
    g.d_iface[0] = R(1); g.d_iface[1] = R(8); g.d_iface[2] = R(1);
  } else {
    g.r = 2; g.eps_a = R(1e-12);
    g.d_iface[0] = R(8); g.d_iface[1] = R(1); g.d_iface[2] = R(1);
  }
  g.d_node[0] = R(8); g.d_node[1] = R(1); g.d_node[2] = R(1);
  return g;
}

template <class R>
GasK<R> gas_of(const double* gp) {   // gamma, mu, Pr, c1, c2, dt
  GasK<R> g;
  const double K = (4.0 - 2.0 * gp[0]) / (gp[0] - 1.0);
  g.K = R(K);
  g.gm1 = R(gp[0] - 1.0);
  g.c4K = R(4.0 / (K + 2.0));
  g.prfix = R(1.0 / gp[2] - 1.0);
  g.mu = gp[1]; g.c1 = gp[3]; g.c2 = gp[4]; g.dt = gp[5]; g.inv_dt = 1.0 / gp[5];
  g.mu_r = R(gp[1]); g.c1_r = R(gp[3]); g.c2_r = R(gp[4]); g.dt_r = R(gp[5]); g.inv_dt_r = R(1.0 / gp[5]);
  return g;
}

void reset() { std::memset(&cnt::c64, 0, sizeof(cnt::Counts)); std::memset(&cnt::c32, 0, sizeof(cnt::Counts)); }

void dump(long long* out) {
  const cnt::Counts* cs[2] = {&cnt::c64, &cnt::c32};
  for (int p = 0; p < 2; ++p) {
    const cnt::Counts& c = *cs[p];
    long long v[8] = {c.add, c.mul, c.div, c.sqrt_, c.exp_, c.erfc_, c.tanh_, c.expm1_};
    for (int k = 0; k < 8; ++k) out[8 * p + k] = v[k];
  }
}

template <class R>
void run(int what, int variant, const double* gp, int normal, double h, int n, const double* in) {
  GenoK<R> g = geno_of<R>(variant);
  GasK<R> gas = gas_of<R>(gp);
  R hh = R(h), ih = R(1.0 / h);
  for (int t = 0; t < n; ++t) {
    cnt::reset_ids();
    if (what == 0) {            // interface reconstruction of one line component (both sides)
      R Q[4], Qx[4];
      for (int k = 0; k < 4; ++k) { Q[k] = R(in[t * 8 + k]); Qx[k] = R(in[t * 8 + 4 + k]); }
      R vl, dl, cl, vr, dr, cr;
      recon_interface(g, Q, Qx, hh, ih, vl, dl, cl, vr, dr, cr);
    } else if (what == 1) {     // node derivative of one component
      R Q[3], Qx[3];
      for (int k = 0; k < 3; ++k) { Q[k] = R(in[t * 6 + k]); Qx[k] = R(in[t * 6 + 3 + k]); }
      recon_node(g, Q, Qx, hh, ih);
    } else if (what == 2) {     // interface solve
      R v[20];
      for (int k = 0; k < 20; ++k) v[k] = R(in[t * 20 + k]);
      IfaceOut<R> o;
      iface_solve(gas, normal, v, v + 4, v + 8, v + 12, v + 16, true, o);
    } else if (what == 3 || what == 5) {     // nodal flux (5: time derivatives only)
      R v[12];
      for (int k = 0; k < 12; ++k) v[k] = R(in[t * 12 + k]);
      R F[4], G[4], Ft[4], Gt[4];
      nodal_flux(gas, v, v + 4, v + 8, F, G, Ft, Gt, what == 3);
    } else {                    // compact flux (in: chi, 3 interface, 2 nodal fluxes)
      R x[6];
      for (int k = 0; k < 6; ++k) x[k] = R(in[t * 6 + k]);
      compact_flux(normal, x[0], x[1], x[2], x[3], x[4], x[5]);
    }
  }
}

}  // namespace

extern "C" {

// what: 0 interface reconstruction, 1 node reconstruction, 2 interface solve,
// 3 nodal flux, 4 compact flux (normal = flux variant), 5 nodal flux time
// derivatives only (second stage).  precision 0: FP64
// compute type, 1: FP32 compute type (its FP64 part counted separately).
// out[16] = FP64 (add, mul, div, sqrt, exp, erfc, tanh, expm1), then FP32 (same).
void flop_count(int what, int precision, int variant, const double* gas, int normal, double h, int n,
                const double* in, long long* out) {
  reset();
  if (precision == 1) run<CF>(what, variant, gas, normal, h, n, in);
  else run<CD>(what, variant, gas, normal, h, n, in);
  dump(out);
}

}  // extern "C"
