// Internal declarations shared by the CUDA translation units of the FD-CGKS
// library: padded data layout, kernel argument block and launchers.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "../../include/fdcgks.h"
#include "fdcgks_math.cuh"

namespace fdk {

const int GH = 3;        // ghost layers of every state plane
const int NFLD = 12;     // fields per grid: W[4], averaged x-gradient[4], averaged y-gradient[4]
const int NNF = 16;      // nodal outputs: F[4], G[4], F_t[4], G_t[4]
const int NPS = 25;      // outputs of one interface solve (see PO_* below)
const int NPT = 2 * NPS; // outputs of one virtual-interface point (primary solve, dual solve)

// field offsets inside one solve's 25 outputs
enum { PO_F = 0, PO_FT = 4, PO_CHI = 8, PO_WL = 9, PO_WR = 13, PO_WLT = 17, PO_WRT = 21 };

// Both grids share one padded plane geometry.  A state buffer holds
// [grid 2][field 12][plane]; node (i, j) of a grid sits at
// (j + GH) * pitch + (i + GH), i in [-GH, n + GH).
// Interface-point arrays (Type A: (i+1/2, j), Type B: (i, j+1/2)) hold
// [NPT][pplane] with point (i, j) at (j + 2) * ppitch + (i + 2).
struct Layout {
  int nx, ny, nxd, nyd;
  int pitch, rows;
  long plane;
  int ppitch, prows;
  long pplane;
};

FD_HD long cell(const Layout& L, int i, int j) { return (long)(j + GH) * L.pitch + (i + GH); }
FD_HD long pcell(const Layout& L, int i, int j) { return (long)(j + 2) * L.ppitch + (i + 2); }

// padded layout of a run: rows padded to multiples of 32 entries
inline Layout make_layout(const fdcgks_params& p) {
  Layout L;
  L.nx = p.nx;
  L.ny = p.ny;
  L.nxd = p.nx + (p.bc[0] == FDCGKS_BC_PERIODIC ? 0 : 1);
  L.nyd = p.ny + (p.bc[2] == FDCGKS_BC_PERIODIC ? 0 : 1);
  const int mx = L.nx > L.nxd ? L.nx : L.nxd, my = L.ny > L.nyd ? L.ny : L.nyd;
  L.pitch = ((mx + 2 * GH) + 31) / 32 * 32;
  L.rows = my + 2 * GH;
  L.plane = (long)L.pitch * L.rows;
  L.ppitch = ((mx + 3) + 31) / 32 * 32;
  L.prows = my + 3;
  L.pplane = (long)L.ppitch * L.prows;
  return L;
}

// CFL rates of one node (Sec. 5 time step): the larger of (|U| + c)/hx and
// (|V| + c)/hy, and the kinematic viscosity mu/rho, folded into running
// maxima (fmax: a NaN never replaces a number)
FD_HD void cfl_rates(double r, double ru, double rv, double E, double gamma, double mu, double ihx, double ihy,
                     double& rate, double& numax) {
  const double ir = 1.0 / r;
  const double U = ru * ir, V = rv * ir;
  const double p = (gamma - 1.0) * (E - 0.5 * r * (U * U + V * V));
  const double cs = sqrt(gamma * p * ir);
  rate = fmax(rate, fmax((fabs(U) + cs) * ihx, (fabs(V) + cs) * ihy));
  numax = fmax(numax, mu * ir);
}

#ifdef __CUDACC__
// FP32 estimate of one node's CFL rate (the form of cfl_rates, or with sum
// set the two directions' rates added) and of mu/rho, from FP32 roundings
// (relative error <= u = 2^-24) of the node's conservative variables; used
// to screen out the nodes that cannot hold the FP64 maxima.  Reliable, i.e.
// within a relative 1e-5 of the FP64 formula on the unrounded values, while
// 1e-30 < rho < 1e30 and p > 0.05 E: U and V carry about 5u, the kinetic
// energy about 12u of itself, so E - rho (U^2+V^2)/2 carries at most about
// (u E + 12u (E - p))/p < 250u of p (E/p < 20); the sound speed halves that,
// giving < 130u ~ 7.8e-6 in the rate.  Otherwise ok is false.
__device__ __forceinline__ void cfl_estimate_f(float r, float ru, float rv, float E, float gf, float muf, float ihxf,
                                               float ihyf, bool sum, float& rt, float& nu, bool& ok) {
  const float ir = __fdividef(1.0f, r), U = ru * ir, V = rv * ir;
  const float p = (gf - 1.0f) * (E - 0.5f * r * (U * U + V * V));
  const float c = sqrtf(fmaxf(gf * p * ir, 0.0f));
  const float ax = (fabsf(U) + c) * ihxf, ay = (fabsf(V) + c) * ihyf;
  rt = sum ? ax + ay : fmaxf(ax, ay);
  nu = muf * ir;
  ok = r > 1e-30f && r < 1e30f && p > 0.05f * E && rt < INFINITY && nu < INFINITY;
}

// Margin of the screening: a node is evaluated in FP64 when its estimate is
// not below the largest reliable estimate by more than this fraction.  With
// the estimates' bound b = 1e-5, (1 - margin)(1 + b)^2 < 1, so a node left
// out has an FP64 rate below that of the node holding the largest estimate:
// the maxima are exactly those of evaluating every node.
const float CFL_SCREEN_MARGIN = 5e-5f;
#endif

template <class R>
struct KArgs {
  Layout L;
  const R* Sr;           // state read by the nodal and point kernels, in the compute type
                         // (the FP64 state itself, or the high parts in the mixed path)
  // mixed path: the state and the S2O4 accumulators are float-float pairs
  const R* Sn_hi;        // state at t^n [2][12][plane], high and low parts
  const R* Sn_lo;
  R* Out_hi;             // stage 1: W*, grad* (high parts only); stage 2: the new state
  R* Out_lo;             // stage 2: low parts of the new state (null at stage 1)
  R* Acc_hi;             // W_acc pairs [2][4][plane]
  R* Acc_lo;
  R* Gb_hi;              // gradient-base pairs [2][8][plane]
  R* Gb_lo;
  const double* S;       // state read by this stage [2][12][plane] (FP64 path)
  const double* Sn;      // state at t^n (stage 1 base, reading-A gradient base)
  double* Sout;          // stage 1: W*, grad*;  stage 2: W^{n+1}, grad^{n+1}
  double* Wacc;          // [2][4][plane]  W^n + dt L + dt^2/6 L_t
  double* gB;            // [2][8][plane]  gradient base of Eq. (eq-interface-update)
  R* NF;                 // [2][16][plane] nodal fluxes
  R* PA;                 // [50][pplane]   Type A point outputs
  R* PB;                 // [50][pplane]   Type B point outputs
  GenoK<R> geno;
  GasK<R> gas;
  R h[2], ih[2];
  double hd[2], ihd[2];
  int bc[4];
  int flux_variant, grad_base, want_n;
  int recon_vars;        // 0 conservative, 1 characteristic interface reconstruction
  double dt;
  int* flag;             // bit 0: non-physical state found
  double* op[8];         // operator outputs (Lp, Ltp, gbp, gtp, Ld, Ltd, gbd, gtd), interior layout
};

// Ghost layers of one grid g of a padded state (W, x- and y-gradients):
// periodic wrap, mirror (symmetry: normal momentum odd; no-slip: both momenta
// odd; gradients take the field's parity times -1 along the mirror normal) or
// constant extrapolation with zero gradients (transmissive).  Work item idx
// covers (row or column t, side, layer k); dir 0 fills x ghosts of interior
// rows, dir 1 y ghosts of all columns (so corners are consistent).
// ghost_map gives the ghost cell, its source cell and the boundary kind of
// item idx (false when idx is out of range); ghost_sign the parity of field
// component c (of W and of the x- and y-gradients; 0 = set to zero).
FD_HD bool ghost_map(const Layout& L, int bc0, int bc1, int dir, int g, int idx, long& gc, long& sc, int& b) {
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  const int n = dir == 0 ? nxg : nyg;
  const int tcount = dir == 0 ? nyg : nxg + 2 * GH;
  const int toff = dir == 0 ? 0 : -GH;
  if (idx < 0 || idx >= tcount * 2 * GH) return false;
  const int k = 1 + idx % GH;
  const int side = (idx / GH) % 2;
  const int t = idx / (2 * GH) + toff;
  b = side == 0 ? bc0 : bc1;
  const int ghost = side == 0 ? -k : n - 1 + k;
  int src;
  if (b == 0) src = ((ghost % n) + n) % n;                 // periodic, also for n < GH
  else if (b == 1) src = side == 0 ? 0 : n - 1;            // transmissive
  else if (g == 0) src = side == 0 ? k - 1 : n - k;        // mirror about the boundary line
  else src = side == 0 ? k : n - 1 - k;
  gc = dir == 0 ? cell(L, ghost, t) : cell(L, t, ghost);
  sc = dir == 0 ? cell(L, src, t) : cell(L, t, src);
  return true;
}

FD_HD void ghost_sign(int b, int dir, int c, int& sW, int& sgx, int& sgy) {
  if (b == 0) { sW = sgx = sgy = 1; return; }
  if (b == 1) { sW = 1; sgx = sgy = 0; return; }
  sW = 1;
  if (c == 1 + dir) sW = -1;
  if (c == 2 - dir && b == 3) sW = -1;
  sgx = dir == 0 ? -sW : sW;
  sgy = dir == 1 ? -sW : sW;
}

// copy the source node into the ghost node with the parities of kind b
template <class T>
__device__ __forceinline__ void ghost_apply(T* Sg, const Layout& L, int b, int dir, long gc, long sc) {
  for (int c = 0; c < 4; ++c) {
    int sW, sgx, sgy;
    ghost_sign(b, dir, c, sW, sgx, sgy);
    T w = Sg[(long)c * L.plane + sc];
    T gx = Sg[(long)(4 + c) * L.plane + sc];
    T gy = Sg[(long)(8 + c) * L.plane + sc];
    if (b == 1) {
      gx = 0;
      gy = 0;
    } else if (b != 0) {
      w *= (T)sW;
      gx *= (T)sgx;
      gy *= (T)sgy;
    }
    Sg[(long)c * L.plane + gc] = w;
    Sg[(long)(4 + c) * L.plane + gc] = gx;
    Sg[(long)(8 + c) * L.plane + gc] = gy;
  }
}

template <class T>
__device__ __forceinline__ void ghost_body(T* S, const Layout& L, int bc0, int bc1, int dir, int g, int idx) {
  long gc, sc;
  int b;
  if (!ghost_map(L, bc0, bc1, dir, g, idx, gc, sc, b)) return;
  ghost_apply(S + (long)g * NFLD * L.plane, L, b, dir, gc, sc);
}

// Split sides (fdcgks_set_sides), at one stage time: kind of each part, the
// split position along the side, the fixed conservative states, the node
// geometry for the coordinate along the side.
struct GhostSides {
  int kind[4][2];
  double split[4];
  double W[4][2][4];
  double x0, y0, hx, hy;
};

template <class T>
__device__ __forceinline__ void ghost_body_sides(T* S, const Layout& L, const GhostSides& gs, int dir, int g,
                                                 int idx) {
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  const int tcount = dir == 0 ? nyg : nxg + 2 * GH;
  if (idx < 0 || idx >= tcount * 2 * GH) return;
  const int side = (idx / GH) % 2;
  const int t = idx / (2 * GH) + (dir == 0 ? 0 : -GH);
  const int sd = 2 * dir + side;
  // coordinate along the side of the ghost's row (x sides) or column (y
  // sides), a single-rounded fused product like the split point, so that a
  // node lying on the split is classified independently of contraction
  const double pos = t + (g == 0 ? 0.5 : 0.0);
  const double coord = dir == 0 ? fma(pos, gs.hy, gs.y0) : fma(pos, gs.hx, gs.x0);
  const int part = coord < gs.split[sd] ? 0 : 1;
  const int kind = gs.kind[sd][part];
  long gc, sc;
  int b;
  if (!ghost_map(L, kind, kind, dir, g, idx, gc, sc, b)) return;
  T* Sg = S + (long)g * NFLD * L.plane;
  if (kind == 4) {   // FIXED
    for (int c = 0; c < 4; ++c) {
      Sg[(long)c * L.plane + gc] = (T)gs.W[sd][part][c];
      Sg[(long)(4 + c) * L.plane + gc] = 0;
      Sg[(long)(8 + c) * L.plane + gc] = 0;
    }
    return;
  }
  ghost_apply(Sg, L, b, dir, gc, sc);
}

enum { UPD_STAGE1 = 0, UPD_STAGE2 = 1, UPD_OPERATOR = 2 };

// message returned by fdcgks_last_error(NULL)
void set_global_error(const char* msg);

// what other translation units of the library see of a context
struct CtxView {
  fdcgks_params p;
  Layout L;
  double hx, hy;
  cudaStream_t stream;
  double* S;        // FP64 state [2][12][plane] (the state itself on the FP64 path)
  bool has_state;
  bool has_sides;   // fdcgks_set_sides in force
};
bool ctx_view(fdcgks_t c, CtxView* v);
void ctx_set_error(fdcgks_t c, const char* msg);

// validation of user parameters (nullptr when valid)
const char* check_params(const fdcgks_params* p);

// run constants in the compute type
template <class R>
inline GenoK<R> make_geno(int variant) {
  GenoK<R> g;
  g.linear = variant == 2;
  g.C = (R)20.0;
  g.tanhC = (R)std::tanh(20.0);
  g.inv_tanhC = (R)(1.0 / std::tanh(20.0));
  g.eps_w = (R)1e-6;
  if (variant == 1) {
    g.r = 3;
    g.eps_a = (R)1e-15;
    g.d_iface[0] = 1; g.d_iface[1] = 8; g.d_iface[2] = 1;
  } else {
    g.r = 2;
    g.eps_a = (R)1e-12;
    g.d_iface[0] = 8; g.d_iface[1] = 1; g.d_iface[2] = 1;
  }
  g.d_node[0] = 8; g.d_node[1] = 1; g.d_node[2] = 1;
  return g;
}

template <class R>
inline GasK<R> make_gas(const fdcgks_params& p, double dt) {
  GasK<R> g;
  const double K = (4.0 - 2.0 * p.gamma) / (p.gamma - 1.0);
  g.K = (R)K;
  g.gm1 = (R)(p.gamma - 1.0);
  g.c4K = (R)(4.0 / (K + 2.0));
  g.prfix = (R)(1.0 / p.Pr - 1.0);
  g.mu = p.mu;
  g.c1 = p.tau_c1;
  g.c2 = p.tau_c2;
  g.dt = dt;
  g.inv_dt = 1.0 / dt;
  g.mu_r = (R)p.mu;
  g.c1_r = (R)p.tau_c1;
  g.c2_r = (R)p.tau_c2;
  g.dt_r = (R)dt;
  g.inv_dt_r = (R)(1.0 / dt);
  return g;
}


// whole-plane helpers of the host runtime (fdcgks_api.cu), on stream s:
// positivity/finiteness check of the interior of an FP64 state (sets bit 0 of
// *flag), and the FP64 <-> float-float conversion of n entries
cudaError_t launch_validate(const double* S, const Layout& L, double gamma, int* flag, cudaStream_t s);
cudaError_t launch_split_ff(const double* S, float* hi, float* lo, long n, cudaStream_t s);
cudaError_t launch_join_ff(const float* hi, const float* lo, double* S, long n, cudaStream_t s);

template <class R> cudaError_t launch_nodal(const KArgs<R>& a, cudaStream_t s);
template <class R> cudaError_t launch_points(const KArgs<R>& a, cudaStream_t s);
template <class R> cudaError_t launch_update(const KArgs<R>& a, int mode, cudaStream_t s);

// component-level batches (device arrays), for parity tests of the kernels' arithmetic
template <class R> cudaError_t launch_iface_batch(const GasK<R>& gas, int normal, int n, const double* in,
                                                  double* out, cudaStream_t s);
template <class R> cudaError_t launch_nodal_batch(const GasK<R>& gas, int n, const double* in, double* out,
                                                  cudaStream_t s);
template <class R> cudaError_t launch_recon_batch(const GenoK<R>& g, int kind, double h, int n, const double* in,
                                                  double* out, cudaStream_t s);

}  // namespace fdk
