// Host build of the hand-written reverse mode (csrc/fdcgks_reverse.cuh) next
// to forward-mode dual numbers (tests/fdcgks_dual.cuh) on the same device
// arithmetic, so that the CPU test suite compares the two without a GPU.
//
// Test instrumentation only: each probe returns, for one set of inputs and
// output adjoints ob, the reverse-mode vector-Jacobian product and the same
// product assembled from the dual numbers' Jacobian columns (one seeded
// input per pass).
#include <cmath>

#include "fdcgks_dual.cuh"
#include "fdcgks_reverse.cuh"

using namespace fdk;

namespace {

typedef Dual<1> D1;

GenoK<double> geno_of(int variant) {
  GenoK<double> g;
  g.linear = variant == 2;
  g.C = 20.0;
  g.tanhC = std::tanh(20.0);
  g.inv_tanhC = 1.0 / std::tanh(20.0);
  g.eps_w = 1e-6;
  if (variant == 1) {
    g.r = 3; g.eps_a = 1e-15;
    g.d_iface[0] = 1; g.d_iface[1] = 8; g.d_iface[2] = 1;
  } else {
    g.r = 2; g.eps_a = 1e-12;
    g.d_iface[0] = 8; g.d_iface[1] = 1; g.d_iface[2] = 1;
  }
  g.d_node[0] = 8; g.d_node[1] = 1; g.d_node[2] = 1;
  return g;
}

GasK<double> gas_of(double gamma, double mu, double Pr, double c1, double c2, double dt) {
  GasK<double> g;
  const double K = (4.0 - 2.0 * gamma) / (gamma - 1.0);
  g.K = K;
  g.gm1 = gamma - 1.0;
  g.c4K = 4.0 / (K + 2.0);
  g.prfix = 1.0 / Pr - 1.0;
  g.mu = mu; g.c1 = c1; g.c2 = c2; g.dt = dt; g.inv_dt = 1.0 / dt;
  g.mu_r = mu; g.c1_r = c1; g.c2_r = c2; g.dt_r = dt; g.inv_dt_r = 1.0 / dt;
  return g;
}

}  // namespace

extern "C" {

// in = Wl, Wr, Wln, Wrn, Wt (20); ob = F, Ft, Wl, Wr, Wlt, Wrt adjoints (24)
void probe_solve_vjp(double gamma, double mu, double Pr, double c1, double c2, double dt, int normal, int want_n,
                     const double* in, const double* ob, double* rev, double* dual) {
  const GasK<double> gas = gas_of(gamma, mu, Pr, c1, c2, dt);
  IfaceOut<double> o;
  for (int k = 0; k < 4; ++k) {
    o.F[k] = ob[k]; o.Ft[k] = ob[4 + k]; o.Wl[k] = ob[8 + k];
    o.Wr[k] = ob[12 + k]; o.Wlt[k] = ob[16 + k]; o.Wrt[k] = ob[20 + k];
  }
  for (int k = 0; k < 20; ++k) rev[k] = 0.0;
  rev::iface_solve_adj(gas, normal, in, in + 4, in + 8, in + 12, in + 16, want_n != 0, o, rev, rev + 4, rev + 8,
                       rev + 12, rev + 16);
  const GasK<D1> gd = dual_gas<1>(gas);
  for (int m = 0; m < 20; ++m) {
    D1 x[20];
    for (int k = 0; k < 20; ++k) x[k] = D1(in[k]);
    x[m].d[0] = 1.0;
    IfaceOut<D1> y;
    iface_solve(gd, normal, x, x + 4, x + 8, x + 12, x + 16, want_n != 0, y);
    double acc = 0.0;
    for (int k = 0; k < 4; ++k) {
      acc += y.Ft[k].d[0] * ob[4 + k] + y.Wlt[k].d[0] * ob[16 + k] + y.Wrt[k].d[0] * ob[20 + k];
      if (want_n) acc += y.F[k].d[0] * ob[k] + y.Wl[k].d[0] * ob[8 + k] + y.Wr[k].d[0] * ob[12 + k];
    }
    dual[m] = acc;
  }
}

// in = Q[4], Qx[4]; ob = vl, dl, chil, vr, dr, chir adjoints; fscale: the
// path-function floor (0: none)
void probe_recon_iface_vjp(int variant, double h, double fscale, const double* in, const double* ob, double* rev,
                           double* dual) {
  const GenoK<double> g = geno_of(variant);
  for (int k = 0; k < 8; ++k) rev[k] = 0.0;
  rev::recon_interface_adj(g, in, in + 4, h, 1.0 / h, ob[0], ob[1], ob[2], ob[3], ob[4], ob[5], rev, rev + 4,
                           fscale);
  const GenoK<D1> gd = dual_geno<1>(g);
  for (int m = 0; m < 8; ++m) {
    D1 x[8];
    for (int k = 0; k < 8; ++k) x[k] = D1(in[k]);
    x[m].d[0] = 1.0;
    D1 vl, dl, cl, vr, dr, cr;
    recon_interface(gd, x, x + 4, D1(h), D1(1.0 / h), vl, dl, cl, vr, dr, cr, D1(fscale));
    dual[m] = vl.d[0] * ob[0] + dl.d[0] * ob[1] + cl.d[0] * ob[2] + vr.d[0] * ob[3] + dr.d[0] * ob[4] +
              cr.d[0] * ob[5];
  }
}

// in = Q[3], Qx[3]; ob = adjoint of the node derivative
void probe_recon_node_vjp(int variant, double h, double fscale, const double* in, double ob, double* rev,
                          double* dual) {
  const GenoK<double> g = geno_of(variant);
  for (int k = 0; k < 6; ++k) rev[k] = 0.0;
  rev::recon_node_adj(g, in, in + 3, h, 1.0 / h, ob, rev, rev + 3, fscale);
  const GenoK<D1> gd = dual_geno<1>(g);
  for (int m = 0; m < 6; ++m) {
    D1 x[6];
    for (int k = 0; k < 6; ++k) x[k] = D1(in[k]);
    x[m].d[0] = 1.0;
    dual[m] = recon_node(gd, x, x + 3, D1(h), D1(1.0 / h), D1(fscale)).d[0] * ob;
  }
}

// one 4-point line of the point kernel (recon_line_ld with the positivity
// safeguard): in = x[e * 8 + f] (32); ob = vl[4], dl[4], vr[4], dr[4], chi (17);
// *acted: bit 0 / bit 1 set where the safeguard replaced the left / right state
void probe_recon_line_vjp(int variant, double h, double fscale, const double* in, const double* ob, double* rev,
                          double* dual, int* acted) {
  const GenoK<double> g = geno_of(variant);
  for (int k = 0; k < 32; ++k) rev[k] = 0.0;
  double vb[4][4];
  for (int s = 0; s < 4; ++s)
    for (int c = 0; c < 4; ++c) vb[s][c] = ob[4 * s + c];
  rev::recon_line_adj(g, in, h, 1.0 / h, vb, ob[16], rev,
                      [&](const double* Q, const double* Qx, double vlb, double dlb, double chilb, double vrb,
                          double drb, double chirb, double* Qb, double* Qxb) {
                        rev::recon_interface_adj(g, Q, Qx, h, 1.0 / h, vlb, dlb, chilb, vrb, drb, chirb, Qb, Qxb,
                                                 fscale);
                      },
                      fscale);
  const GenoK<D1> gd = dual_geno<1>(g);
  for (int m = 0; m < 32; ++m) {
    D1 x[32];
    for (int k = 0; k < 32; ++k) x[k] = D1(in[k]);
    x[m].d[0] = 1.0;
    D1 vl[4], dl[4], vr[4], dr[4], chi;
    // the safeguard of recon_line_ld, on this line alone
    for (int c = 0; c < 4; ++c) {
      const D1 Q[4] = {x[c], x[8 + c], x[16 + c], x[24 + c]}, Qx[4] = {x[4 + c], x[12 + c], x[20 + c], x[28 + c]};
      D1 cl, cr;
      recon_interface(gd, Q, Qx, D1(h), D1(1.0 / h), vl[c], dl[c], cl, vr[c], dr[c], cr, D1(fscale));
      if (c == 0) chi = s_min(cl, cr);
    }
    const bool badl = !physical_state(vl), badr = !physical_state(vr);
    *acted = (badl ? 1 : 0) | (badr ? 2 : 0);
    if (badl) {
      for (int c = 0; c < 4; ++c) { vl[c] = x[8 + c]; dl[c] = D1(0.0); }
      chi = D1(0.0);
    }
    if (badr) {
      for (int c = 0; c < 4; ++c) { vr[c] = x[16 + c]; dr[c] = D1(0.0); }
      chi = D1(0.0);
    }
    double acc = chi.d[0] * ob[16];
    for (int c = 0; c < 4; ++c)
      acc += vl[c].d[0] * ob[c] + dl[c].d[0] * ob[4 + c] + vr[c].d[0] * ob[8 + c] + dr[c].d[0] * ob[12 + c];
    dual[m] = acc;
  }
}

// in = W, Wx, Wy (12); ob = F, G, Ft, Gt adjoints (16)
void probe_nodal_vjp(double gamma, double mu, double Pr, double c1, double dt, const double* in, const double* ob,
                     double* rev, double* dual) {
  const GasK<double> gas = gas_of(gamma, mu, Pr, c1, 0.0, dt);
  for (int k = 0; k < 12; ++k) rev[k] = 0.0;
  rev::nodal_flux_adj(gas, in, in + 4, in + 8, ob, ob + 4, ob + 8, ob + 12, rev, rev + 4, rev + 8);
  const GasK<D1> gd = dual_gas<1>(gas);
  for (int m = 0; m < 12; ++m) {
    D1 x[12];
    for (int k = 0; k < 12; ++k) x[k] = D1(in[k]);
    x[m].d[0] = 1.0;
    D1 F[4], G[4], Ft[4], Gt[4];
    nodal_flux(gd, x, x + 4, x + 8, F, G, Ft, Gt);
    double acc = 0.0;
    for (int k = 0; k < 4; ++k)
      acc += F[k].d[0] * ob[k] + G[k].d[0] * ob[4 + k] + Ft[k].d[0] * ob[8 + k] + Gt[k].d[0] * ob[12 + k];
    dual[m] = acc;
  }
}

}  // extern "C"
