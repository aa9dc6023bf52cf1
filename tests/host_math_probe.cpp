// Host instantiation of the device arithmetic in fdcgks_math.cuh.
//
// Test instrumentation only: lets the CPU test suite check the kernels'
// formulas (reconstruction, kinetic interface solve, nodal flux) against the
// oracle without a GPU.  The library and its Python binding never call it;
// the product path runs only in the CUDA kernels.
#include <cmath>

#include "fdcgks_math.cuh"

using namespace fdk;

namespace {

template <class R>
GenoK<R> geno_of(int variant) {
  GenoK<R> g;
  g.linear = variant == 2;
  g.C = (R)20.0;
  g.tanhC = (R)std::tanh(20.0);
  g.inv_tanhC = (R)(1.0 / std::tanh(20.0));
  g.eps_w = (R)1e-6;
  if (variant == 1) {
    g.r = 3; g.eps_a = (R)1e-15;
    g.d_iface[0] = 1; g.d_iface[1] = 8; g.d_iface[2] = 1;
  } else {
    g.r = 2; g.eps_a = (R)1e-12;
    g.d_iface[0] = 8; g.d_iface[1] = 1; g.d_iface[2] = 1;
  }
  g.d_node[0] = 8; g.d_node[1] = 1; g.d_node[2] = 1;
  return g;
}

template <class R>
GasK<R> gas_of(double gamma, double mu, double Pr, double c1, double c2, double dt) {
  GasK<R> g;
  const double K = (4.0 - 2.0 * gamma) / (gamma - 1.0);
  g.K = (R)K;
  g.gm1 = (R)(gamma - 1.0);
  g.c4K = (R)(4.0 / (K + 2.0));
  g.prfix = (R)(1.0 / Pr - 1.0);
  g.mu = mu; g.c1 = c1; g.c2 = c2; g.dt = dt; g.inv_dt = 1.0 / dt;
  g.mu_r = (R)mu; g.c1_r = (R)c1; g.c2_r = (R)c2; g.dt_r = (R)dt; g.inv_dt_r = (R)(1.0 / dt);
  return g;
}

template <class R>
void iface(double gamma, double mu, double Pr, double c1, double c2, double dt, int normal, int n, const double* in,
           double* out) {
  GasK<R> gas = gas_of<R>(gamma, mu, Pr, c1, c2, dt);
  for (int t = 0; t < n; ++t) {
    R v[20];
    for (int k = 0; k < 20; ++k) v[k] = (R)in[t * 20 + k];
    IfaceOut<R> o;
    iface_solve(gas, normal, v, v + 4, v + 8, v + 12, v + 16, true, o);
    double* q = out + t * 24;
    for (int k = 0; k < 4; ++k) {
      q[k] = o.F[k]; q[4 + k] = o.Ft[k]; q[8 + k] = o.Wl[k];
      q[12 + k] = o.Wr[k]; q[16 + k] = o.Wlt[k]; q[20 + k] = o.Wrt[k];
    }
  }
}

}  // namespace

extern "C" {

// path-function values chi^l, chi^r of the interface reconstruction of n
// 4-point lines (Q[n][4], Qx[n][4]) in FP32 (precision 1) or FP64
void probe_recon_chi(int precision, int variant, int n, const double* Q, const double* Qx, double h, double* chi) {
  for (int t = 0; t < n; ++t) {
    if (precision == 1) {
      const GenoK<float> g = geno_of<float>(variant);
      float q[4], qx[4], vl, dl, cl, vr, dr, cr;
      for (int k = 0; k < 4; ++k) { q[k] = (float)Q[t * 4 + k]; qx[k] = (float)Qx[t * 4 + k]; }
      recon_interface(g, q, qx, (float)h, (float)(1.0 / h), vl, dl, cl, vr, dr, cr);
      chi[2 * t] = cl; chi[2 * t + 1] = cr;
    } else {
      const GenoK<double> g = geno_of<double>(variant);
      double vl, dl, cl, vr, dr, cr;
      recon_interface(g, Q + t * 4, Qx + t * 4, h, 1.0 / h, vl, dl, cl, vr, dr, cr);
      chi[2 * t] = cl; chi[2 * t + 1] = cr;
    }
  }
}

void probe_iface(int precision, double gamma, double mu, double Pr, double c1, double c2, double dt, int normal, int n,
                 const double* in, double* out) {
  if (precision == 1) iface<float>(gamma, mu, Pr, c1, c2, dt, normal, n, in, out);
  else iface<double>(gamma, mu, Pr, c1, c2, dt, normal, n, in, out);
}

void probe_nodal(double gamma, double mu, double Pr, double c1, double dt, int n, const double* in, double* out) {
  GasK<double> gas = gas_of<double>(gamma, mu, Pr, c1, 0.0, dt);
  for (int t = 0; t < n; ++t) {
    double F[4], G[4], Ft[4], Gt[4];
    nodal_flux(gas, in + t * 12, in + t * 12 + 4, in + t * 12 + 8, F, G, Ft, Gt);
    for (int k = 0; k < 4; ++k) {
      out[t * 16 + k] = F[k]; out[t * 16 + 4 + k] = G[k];
      out[t * 16 + 8 + k] = Ft[k]; out[t * 16 + 12 + k] = Gt[k];
    }
  }
}

// FP32 erfc of the mixed path (host build of the same source), for checks
// against the approximation's published error bound
void probe_erfc32(int n, const double* x, double* out) {
  for (int t = 0; t < n; ++t) {
    float xf = (float)x[t];
    out[t] = (double)s_erfc_e(xf, std::exp(-xf * xf));
  }
}

void probe_recon(int variant, int kind, double h, int n, const double* in, double* out) {
  GenoK<double> g = geno_of<double>(variant);
  for (int t = 0; t < n; ++t) {
    if (kind == 0) {
      double vl, dl, cl, vr, dr, cr;
      recon_interface(g, in + t * 8, in + t * 8 + 4, h, 1.0 / h, vl, dl, cl, vr, dr, cr);
      double* q = out + t * 6;
      q[0] = vl; q[1] = dl; q[2] = cl; q[3] = vr; q[4] = dr; q[5] = cr;
    } else {
      out[t * 6] = recon_node(g, in + t * 6, in + t * 6 + 3, h, 1.0 / h);
      for (int k = 1; k < 6; ++k) out[t * 6 + k] = 0.0;
    }
  }
}

}  // extern "C"
