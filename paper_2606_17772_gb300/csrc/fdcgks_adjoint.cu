// Adjoint (reverse mode) of the FP64 FD-CGKS step: the gradient of a scalar
// function of the state after n steps with respect to the initial state.
//
// The step is a composition of local maps: the ghost fill, the nodal map
// (node stencil -> nodal fluxes), the point map (two 4-node lines -> the 50
// outputs of a virtual-interface point), and the update (compact fluxes of
// point and nodal outputs -> stage operator -> S2O4 combination, no-slip
// reset).  Its adjoint runs these in reverse:
//   update:  written out by hand (linear in the fluxes given chi, bilinear in
//            chi; the reset's Jacobian explicitly), scattering the adjoints of
//            the point and nodal outputs with atomicAdd;
//   points, nodes: written out by hand as well (fdcgks_reverse.cuh: the
//            reverse passes of the GENO reconstructions, the kinetic solve and
//            the nodal flux), scattered into the adjoint state with atomicAdd;
//   ghost fill: each ghost's adjoint folded back into its source (y pass,
//            then x pass, the reverse of the forward order).
// The forward states are recomputed from checkpoints taken every
// `checkpoint_every` steps; each step's intermediates (stage state, point and
// nodal outputs of both stages, S2O4 accumulators) are recomputed once more
// right before its reverse pass.
// On a mixed-precision context the trajectory (checkpoints, segment states,
// the final state) is the context's own mixed run, replayed through FP64
// buffers that hold its float-float pairs to FP64 rounding; each step's intermediates
// and reverse pass are the FP64 step's at those states, so the adjoint state
// accumulates in FP64 and the result is the FP64 step's derivative along the
// mixed trajectory.  Where the data vary by less than about 4e-6 of their
// size the mixed step's GENO takes them as smooth (its FP32 rounding floor)
// and the FP64 step's does not; there the two derivatives differ.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/fdcgks.h"
#include "fdcgks_kernels.cuh"
#include "fdcgks_reverse.cuh"
#include "fdcgks_replay.h"

namespace fdk {
// the forward FP64 kernels are instantiated in fdcgks_fp64.cu
extern template cudaError_t launch_nodal<double>(const KArgs<double>&, cudaStream_t);
extern template cudaError_t launch_points<double>(const KArgs<double>&, cudaStream_t);
extern template cudaError_t launch_update<double>(const KArgs<double>&, int, cudaStream_t);
}  // namespace fdk

using namespace fdk;

namespace {

// ---------------------------------------------------------------------------
// out-of-line copies of the reverse passes (one code copy per kernel)
// ---------------------------------------------------------------------------
__device__ __noinline__ void solve_adj_call(const GasK<double>& gas, int normal, const double* Wl, const double* Wr,
                                            const double* Wln, const double* Wrn, const double* Wt, bool want_n,
                                            const IfaceOut<double>& ob, double* Wlb, double* Wrb, double* Wlnb,
                                            double* Wrnb, double* Wtb) {
  rev::iface_solve_adj(gas, normal, Wl, Wr, Wln, Wrn, Wt, want_n, ob, Wlb, Wrb, Wlnb, Wrnb, Wtb);
}

__device__ __noinline__ void recon_adj_call(const GenoK<double>& g, const double* Q, const double* Qx, double h,
                                            double ih, double vlb, double dlb, double chilb, double vrb, double drb,
                                            double chirb, double* Qb, double* Qxb, double fscale) {
  rev::recon_interface_adj(g, Q, Qx, h, ih, vlb, dlb, chilb, vrb, drb, chirb, Qb, Qxb, fscale);
}

// ---------------------------------------------------------------------------
// point map adjoint: inputs are the 64 values (2 lines x 4 entries x (4 W +
// 4 gradients along the line)) the point reads; outputs its 50 values.
// Reverse order of point_compute: W~ assembly (linear) <- two kinetic solves
// <- tangential derivatives (means) <- two line reconstructions, each step
// by its hand-written reverse pass (fdcgks_reverse.cuh).  fscale > 0 (mixed
// contexts): GENO's path function takes the FP32 path's rounding floor
// (64 u max|Q|)^2, so that the reverse pass linearises the map the mixed
// step computes, in which data varying below the floor count as smooth.
// ---------------------------------------------------------------------------
template <int TYPE>
__global__ void __launch_bounds__(128) point_vjp_kernel(KArgs<double> a, const double* __restrict__ Pa,
                                                        double* Sa, double fscale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 2, j = blockIdx.y * blockDim.y + threadIdx.y - 2;
  const Layout& L = a.L;
  const int imax = TYPE == 0 ? L.nx : L.nxd, jmax = TYPE == 0 ? L.nyd : L.ny;
  if (i < -2 || j < -2 || i > imax || j > jmax) return;
  const long pp = L.pplane, pc = pcell(L, i, j);
  double ah[NPT];
  bool any = false;
  for (int k = 0; k < NPT; ++k) {
    ah[k] = Pa[(long)k * pp + pc];
    any = any || ah[k] != 0.0;
  }
  if (!any) return;
  const PointLines pl = point_lines<TYPE>(L, i, j);
  auto addr = [&](int s) -> long {
    const int l = s / 32, e = (s / 8) % 4, f = s % 8;
    const int field = f < 4 ? f : pl.gfield[l] + (f - 4);
    return ((long)l * NFLD + field) * L.plane + pl.base[l] + e * pl.stride[l];
  };
  double x[64];
  for (int s = 0; s < 64; ++s) x[s] = a.Sr[addr(s)];
  const bool wn = a.want_n != 0;
  const int n0 = TYPE;                                  // normal of solve 0 (primary line); solve 1: 1 - n0
  const double hl[2] = {a.h[n0], a.h[1 - n0]}, ihl[2] = {a.ih[n0], a.ih[1 - n0]};

  // forward values of the reconstructions and tangential derivatives
  double v[2][4][4], chi[2];                            // v[line][vl, dl, vr, dr][component]
  for (int l = 0; l < 2; ++l) {
    double cl0, cr0;
    bool fl, fr;
    rev::recon_line_fwd(a.geno, x + 32 * l, hl[l], ihl[l], fscale, v[l], chi[l], cl0, cr0, fl, fr);
  }
  double tg[2][4];
  for (int c = 0; c < 4; ++c) {
    tg[0][c] = 0.5 * (v[1][1][c] + v[1][3][c]);
    tg[1][c] = 0.5 * (v[0][1][c] + v[0][3][c]);
  }

  // adjoints of the solves' outputs from the point outputs (W~ of Eq. eq:W-model-2d)
  IfaceOut<double> ao[2];
  for (int sv = 0; sv < 2; ++sv) {
    const int b = sv * NPS, o = (1 - sv) * NPS;
    for (int c = 0; c < 4; ++c) {
      ao[sv].F[c] = wn ? ah[b + PO_F + c] : 0.0;
      ao[sv].Ft[c] = ah[b + PO_FT + c];
      ao[sv].Wl[c] = wn ? 0.5 * ah[b + PO_WL + c] + 0.25 * (ah[o + PO_WL + c] + ah[o + PO_WR + c]) : 0.0;
      ao[sv].Wr[c] = wn ? 0.5 * ah[b + PO_WR + c] + 0.25 * (ah[o + PO_WL + c] + ah[o + PO_WR + c]) : 0.0;
      ao[sv].Wlt[c] = 0.5 * ah[b + PO_WLT + c] + 0.25 * (ah[o + PO_WLT + c] + ah[o + PO_WRT + c]);
      ao[sv].Wrt[c] = 0.5 * ah[b + PO_WRT + c] + 0.25 * (ah[o + PO_WLT + c] + ah[o + PO_WRT + c]);
    }
  }

  // solves: their reverse passes give the adjoints of W^l, W^r, the normal
  // derivatives and the tangential derivative
  double av[2][4][4] = {}, at[2][4] = {};
  for (int sv = 0; sv < 2; ++sv)
    solve_adj_call(a.gas, sv == 0 ? n0 : 1 - n0, v[sv][0], v[sv][2], v[sv][1], v[sv][3], tg[sv], wn, ao[sv],
                   av[sv][0], av[sv][2], av[sv][1], av[sv][3], at[sv]);
  // the tangential derivative of each solve is the mean of the other line's derivatives
  for (int c = 0; c < 4; ++c) {
    av[1][1][c] += 0.5 * at[0][c];
    av[1][3][c] += 0.5 * at[0][c];
    av[0][1][c] += 0.5 * at[1][c];
    av[0][3][c] += 0.5 * at[1][c];
  }
  // line reconstructions
  double ax[64] = {};
  for (int l = 0; l < 2; ++l)
    rev::recon_line_adj(a.geno, x + 32 * l, hl[l], ihl[l], av[l], ah[l * NPS + PO_CHI], ax + 32 * l,
                        [&](const double* Q, const double* Qx, double vlb, double dlb, double chilb, double vrb,
                            double drb, double chirb, double* Qb, double* Qxb) {
                          recon_adj_call(a.geno, Q, Qx, hl[l], ihl[l], vlb, dlb, chilb, vrb, drb, chirb, Qb, Qxb,
                                         fscale);
                        },
                        fscale);
  for (int s = 0; s < 64; ++s)
    if (ax[s] != 0.0) atomicAdd(Sa + addr(s), ax[s]);
}

// ---------------------------------------------------------------------------
// nodal map adjoint: 44 inputs (the node's 12 fields; W and the x-gradient of
// its x neighbours; W and the y-gradient of its y neighbours), 16 outputs
// ---------------------------------------------------------------------------
const int NODAL_IN = 44;

// slot of (stencil node e, field f) in the 44 inputs, and back
FD_HD int nodal_slot(int e, int f) {
  if (e == 0) return f;
  const int base = 12 + (e - 1) * 8;
  if (e <= 2) return base + f;             // fields 0-7
  return base + (f < 4 ? f : f - 4);       // fields 0-3, 8-11
}
FD_HD void nodal_unslot(int s, int& e, int& f) {
  if (s < 12) {
    e = 0;
    f = s;
    return;
  }
  e = 1 + (s - 12) / 8;
  const int r = (s - 12) % 8;
  f = (e <= 2 || r < 4) ? r : r + 4;
}

__device__ __noinline__ void nodal_adj_call(const GasK<double>& gas, const double* W, const double* Wx,
                                            const double* Wy, const double* ah, double* Wb, double* Wxb,
                                            double* Wyb) {
  rev::nodal_flux_adj(gas, W, Wx, Wy, ah, ah + 4, ah + 8, ah + 12, Wb, Wxb, Wyb);
}

__global__ void __launch_bounds__(128) nodal_vjp_kernel(KArgs<double> a, const double* __restrict__ NFa, double* Sa,
                                                        double fscale) {
  const int g = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1, j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  const Layout& L = a.L;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  if (i < -1 || j < -1 || i > nxg || j > nyg) return;
  const long c0 = cell(L, i, j);
  double ah[NNF];
  bool any = false;
  for (int k = 0; k < NNF; ++k) {
    ah[k] = NFa[((long)g * NNF + k) * L.plane + c0];
    any = any || ah[k] != 0.0;
  }
  if (!any) return;
  const long gbase = (long)g * NFLD * L.plane;
  auto addr = [&](int s) -> long {
    int e, f;
    nodal_unslot(s, e, f);
    return gbase + (long)f * L.plane + c0 + nodal_offset(L, e);
  };
  double x[NODAL_IN];
  for (int s = 0; s < NODAL_IN; ++s) x[s] = a.Sr[addr(s)];
  auto X = [&](int e, int f) { return x[nodal_slot(e, f)]; };
  // forward values of the node derivatives (dir 0: x with neighbours 1, 2; dir 1: y with 3, 4)
  double W[4], D[2][4];
  for (int c = 0; c < 4; ++c) {
    W[c] = X(0, c);
    for (int d = 0; d < 2; ++d) {
      const int em = 1 + 2 * d, ep = 2 + 2 * d, gf = 4 + 4 * d + c;
      const double q[3] = {X(em, c), W[c], X(ep, c)}, gq[3] = {X(em, gf), X(0, gf), X(ep, gf)};
      D[d][c] = recon_node(a.geno, q, gq, a.h[d], a.ih[d], fscale);
    }
  }
  // nodal flux reverse pass: adjoints of W, W_x, W_y
  double aW[4] = {0, 0, 0, 0}, aD[2][4] = {};
  nodal_adj_call(a.gas, W, D[0], D[1], ah, aW, aD[0], aD[1]);
  // node derivatives reverse passes
  double ax[NODAL_IN] = {};
  for (int c = 0; c < 4; ++c) ax[nodal_slot(0, c)] += aW[c];
  for (int d = 0; d < 2; ++d)
    for (int c = 0; c < 4; ++c) {
      const int em = 1 + 2 * d, ep = 2 + 2 * d, gf = 4 + 4 * d + c;
      const int ent[3] = {em, 0, ep};
      const double q[3] = {X(em, c), W[c], X(ep, c)}, gq[3] = {X(em, gf), X(0, gf), X(ep, gf)};
      double qb[3] = {0.0, 0.0, 0.0}, gqb[3] = {0.0, 0.0, 0.0};
      rev::recon_node_adj(a.geno, q, gq, a.h[d], a.ih[d], aD[d][c], qb, gqb, fscale);
      for (int t = 0; t < 3; ++t) {
        ax[nodal_slot(ent[t], c)] += qb[t];
        ax[nodal_slot(ent[t], gf)] += gqb[t];
      }
    }
  for (int s = 0; s < NODAL_IN; ++s)
    if (ax[s] != 0.0) atomicAdd(Sa + addr(s), ax[s]);
}

// ---------------------------------------------------------------------------
// update adjoint
// ---------------------------------------------------------------------------
// adjoint of compact_flux (Eqs. fd-conservative-flux-1/-2) times bar
__device__ __forceinline__ void compact_flux_adj(int fv, double chi, double Fim, double Fi0, double Fip, double Fn0,
                                                 double Fn1, double bar, double& dchi, double& dim, double& di0,
                                                 double& dip, double& dn) {
  const double Fbar = (Fim + 46.0 * Fi0 + Fip - 9.0 * (Fn0 + Fn1)) * (1.0 / 30.0);
  const double Flow = fv == 62 ? Fi0 : (8.0 * Fi0 - Fn0 - Fn1) * (1.0 / 6.0);
  dchi = bar * (Fbar - Flow);
  dim = bar * chi * (1.0 / 30.0);
  dip = dim;
  di0 = bar * (chi * (46.0 / 30.0) + (1.0 - chi) * (fv == 62 ? 1.0 : 8.0 / 6.0));
  dn = bar * (-9.0 / 30.0 * chi + (1.0 - chi) * (fv == 62 ? 0.0 : -1.0 / 6.0));
}

__device__ __forceinline__ void aadd(double* p, double v) {
  if (v != 0.0) atomicAdd(p, v);
}

// one compact flux's adjoint scattered into the point (field fpt of the three
// points im, i0, ip, chi at chip) and nodal (the two nodes n0, n1) adjoints
__device__ __forceinline__ void cf_scatter(int fv, const double* P, double* Pa, long pp, int fpt, long im, long i0,
                                           long ip, long chip, const double* N, double* Na, long n0, long n1,
                                           double bar) {
  if (bar == 0.0) return;
  double dchi, dim, di0, dip, dn;
  compact_flux_adj(fv, P[PO_CHI * pp + chip], P[fpt * pp + im], P[fpt * pp + i0], P[fpt * pp + ip], N[n0], N[n1],
                   bar, dchi, dim, di0, dip, dn);
  aadd(Pa + PO_CHI * pp + chip, dchi);
  aadd(Pa + fpt * pp + im, dim);
  aadd(Pa + fpt * pp + i0, di0);
  aadd(Pa + fpt * pp + ip, dip);
  aadd(Na + n0, dn);
  aadd(Na + n1, dn);
}

// stage = 0: stage 1 (UPD_STAGE1), 1: stage 2 (UPD_STAGE2).
// Aout: adjoint of this stage's output state; Aacc, AgB: adjoints of the
// S2O4 accumulator and the gradient base (written by stage 2, read by stage
// 1); Ain: stage 1 writes the direct part of the adjoint of the step's input
// state; PAa, PBa, NFa: adjoints of this stage's point and nodal outputs.
__global__ void __launch_bounds__(128) update_adj_kernel(KArgs<double> a, int stage, const double* Aout,
                                                         double* Aacc, double* AgB, double* Ain, double* PAa,
                                                         double* PBa, double* NFa) {
  const int g = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const Layout& L = a.L;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  if (i < 0 || j < 0 || i >= nxg || j >= nyg) return;
  const long P = L.plane, c0 = cell(L, i, j), pp = L.pplane;
  const double dt = a.dt;
  const bool want_n = stage == 0;
  NodeOp<double> o;
  node_operator(a, g, i, j, want_n, o);
  const double* Ao = Aout + (long)g * NFLD * P;
  double Wb[4], Gb[8];
  for (int c = 0; c < 4; ++c) Wb[c] = Ao[(long)c * P + c0];
  for (int f = 0; f < 8; ++f) Gb[f] = Ao[(long)(4 + f) * P + c0];
  const bool xwall = g == 1 && ((a.bc[0] == 3 && i == 0) || (a.bc[1] == 3 && i == nxg - 1));
  const bool ywall = g == 1 && ((a.bc[2] == 3 && j == 0) || (a.bc[3] == 3 && j == nyg - 1));
  double* Ac = Aacc + (long)g * 4 * P;
  double* Ag = AgB + (long)g * 8 * P;
  if (xwall || ywall) {
    // the reset W' = (W0, 0, 0, W3 - (W1^2 + W2^2)/(2 W0)) of the pre-reset stage result
    double W[4];
    for (int c = 0; c < 4; ++c)
      W[c] = stage == 0 ? a.Sn[(long)g * NFLD * P + (long)c * P + c0] + 0.5 * dt * o.L[c] + 0.125 * dt * dt * o.Lt[c]
                        : a.Wacc[(long)g * 4 * P + (long)c * P + c0] + dt * dt / 3.0 * o.Lt[c];
    const double iw = 1.0 / W[0], e3 = Wb[3];
    Wb[0] += e3 * 0.5 * (W[1] * W[1] + W[2] * W[2]) * iw * iw;
    Wb[1] = -e3 * W[1] * iw;
    Wb[2] = -e3 * W[2] * iw;
  }
  if (xwall) { Gb[4 + 1] = 0.0; Gb[4 + 2] = 0.0; }   // y-gradients of rho U, rho V set to 0
  if (ywall) { Gb[1] = 0.0; Gb[2] = 0.0; }           // x-gradients of rho U, rho V set to 0
  double Lb[4], Ltb[4], gbxb[4], gbyb[4], gtxb[4], gtyb[4];
  if (stage == 1) {
    for (int c = 0; c < 4; ++c) {
      Ac[(long)c * P + c0] = Wb[c];
      Lb[c] = 0.0;
      Ltb[c] = dt * dt / 3.0 * Wb[c];
      gbxb[c] = gbyb[c] = 0.0;
      gtxb[c] = dt * Gb[c];
      gtyb[c] = dt * Gb[4 + c];
    }
    for (int f = 0; f < 8; ++f) Ag[(long)f * P + c0] = Gb[f];
  } else {
    double* Ai = Ain + (long)g * NFLD * P;
    for (int c = 0; c < 4; ++c) {
      const double wa = Ac[(long)c * P + c0];
      Ai[(long)c * P + c0] = Wb[c] + wa;
      Lb[c] = 0.5 * dt * Wb[c] + dt * wa;
      Ltb[c] = 0.125 * dt * dt * Wb[c] + dt * dt / 6.0 * wa;
      gtxb[c] = 0.5 * dt * Gb[c];
      gtyb[c] = 0.5 * dt * Gb[4 + c];
    }
    for (int f = 0; f < 8; ++f) {
      const double bb = Ag[(long)f * P + c0] + Gb[f];
      Ai[(long)(4 + f) * P + c0] = a.grad_base ? bb : 0.0;
      const double gb = a.grad_base ? 0.0 : bb;
      if (f < 4) gbxb[f] = gb;
      else gbyb[f - 4] = gb;
    }
  }
  // adjoint of node_operator: the same points and nodal fluxes as the forward
  const double* PX = g == 0 ? a.PA : a.PB + NPS * pp;
  const double* PY = g == 0 ? a.PB : a.PA + NPS * pp;
  double* PXa = g == 0 ? PAa : PBa + NPS * pp;
  double* PYa = g == 0 ? PBa : PAa + NPS * pp;
  auto xi = [&](int k) { return g == 0 ? pcell(L, k, j) : pcell(L, k, j - 1); };
  auto yi = [&](int k) { return g == 0 ? pcell(L, i, k) : pcell(L, i - 1, k); };
  const double* NF = a.NF + (long)g * NNF * P;
  double* NFg = NFa + (long)g * NNF * P;
  const int fv = a.flux_variant;
  const double ihx = a.ih[0], ihy = a.ih[1];
  const long xm2 = xi(i - 2), xm1 = xi(i - 1), x0 = xi(i), xp1 = xi(i + 1);
  const long ym2 = yi(j - 2), ym1 = yi(j - 1), y0 = yi(j), yp1 = yi(j + 1);
  const long cE = c0 + 1, cW = c0 - 1, cN = c0 + L.pitch, cS = c0 - L.pitch;
  for (int c = 0; c < 4; ++c) {
    // L_t = -(fp - fm)/hx - (gp - gm)/hy on the time-derivative fluxes
    const double* nFt = NF + (long)(8 + c) * P;
    const double* nGt = NF + (long)(12 + c) * P;
    double* nFta = NFg + (long)(8 + c) * P;
    double* nGta = NFg + (long)(12 + c) * P;
    cf_scatter(fv, PX, PXa, pp, PO_FT + c, xm1, x0, xp1, x0, nFt, nFta, c0, cE, -ihx * Ltb[c]);
    cf_scatter(fv, PX, PXa, pp, PO_FT + c, xm2, xm1, x0, xm1, nFt, nFta, cW, c0, ihx * Ltb[c]);
    cf_scatter(fv, PY, PYa, pp, PO_FT + c, ym1, y0, yp1, y0, nGt, nGta, c0, cN, -ihy * Ltb[c]);
    cf_scatter(fv, PY, PYa, pp, PO_FT + c, ym2, ym1, y0, ym1, nGt, nGta, cS, c0, ihy * Ltb[c]);
    if (want_n) {
      const double* nF = NF + (long)c * P;
      const double* nG = NF + (long)(4 + c) * P;
      double* nFa = NFg + (long)c * P;
      double* nGa = NFg + (long)(4 + c) * P;
      cf_scatter(fv, PX, PXa, pp, PO_F + c, xm1, x0, xp1, x0, nF, nFa, c0, cE, -ihx * Lb[c]);
      cf_scatter(fv, PX, PXa, pp, PO_F + c, xm2, xm1, x0, xm1, nF, nFa, cW, c0, ihx * Lb[c]);
      cf_scatter(fv, PY, PYa, pp, PO_F + c, ym1, y0, yp1, y0, nG, nGa, c0, cN, -ihy * Lb[c]);
      cf_scatter(fv, PY, PYa, pp, PO_F + c, ym2, ym1, y0, ym1, nG, nGa, cS, c0, ihy * Lb[c]);
      // averaged gradients re-evaluated from W~ (Eq. define-averaged-gradient)
      aadd(PXa + (PO_WL + c) * pp + x0, ihx * gbxb[c]);
      aadd(PXa + (PO_WR + c) * pp + xm1, -ihx * gbxb[c]);
      aadd(PYa + (PO_WL + c) * pp + y0, ihy * gbyb[c]);
      aadd(PYa + (PO_WR + c) * pp + ym1, -ihy * gbyb[c]);
    }
    aadd(PXa + (PO_WLT + c) * pp + x0, ihx * gtxb[c]);
    aadd(PXa + (PO_WRT + c) * pp + xm1, -ihx * gtxb[c]);
    aadd(PYa + (PO_WLT + c) * pp + y0, ihy * gtyb[c]);
    aadd(PYa + (PO_WRT + c) * pp + ym1, -ihy * gtyb[c]);
  }
}

// ---------------------------------------------------------------------------
// ghost fill: forward (as the library's) and its adjoint
// ---------------------------------------------------------------------------
__global__ void ghost_fwd_kernel(double* S, Layout L, int bc0, int bc1, int dir) {
  ghost_body(S, L, bc0, bc1, dir, blockIdx.z, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void ghost_adj_kernel(double* Sa, Layout L, int bc0, int bc1, int dir) {
  const int g = blockIdx.z;
  long gc, sc;
  int b;
  if (!ghost_map(L, bc0, bc1, dir, g, blockIdx.x * blockDim.x + threadIdx.x, gc, sc, b)) return;
  double* Sg = Sa + (long)g * NFLD * L.plane;
  for (int c = 0; c < 4; ++c) {
    int sW, sgx, sgy;
    ghost_sign(b, dir, c, sW, sgx, sgy);
    const int sgn[3] = {sW, sgx, sgy};
    for (int q = 0; q < 3; ++q) {
      const long f = (long)(4 * q + c) * L.plane;
      const double v = Sg[f + gc];
      Sg[f + gc] = 0.0;
      if (sgn[q] != 0 && v != 0.0) atomicAdd(Sg + f + sc, sgn[q] * v);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Work {
  CtxView v;
  size_t fs = 0;             // bytes of one padded state [2][12][plane]
  std::vector<double*> ck;   // checkpoints
  std::vector<double*> seg;  // states of one segment
  double *Sn = nullptr, *S2 = nullptr, *Snext = nullptr, *Wacc = nullptr, *gB = nullptr;
  double *P1A = nullptr, *P1B = nullptr, *P2A = nullptr, *P2B = nullptr, *NF1 = nullptr, *NF2 = nullptr;
  double *A0 = nullptr, *A1 = nullptr, *As = nullptr, *Aacc = nullptr, *AgB = nullptr;
  double *PAa = nullptr, *PBa = nullptr, *NFa = nullptr;
  double* fin = nullptr;     // final state (mixed contexts: loaded back at the end)
  int* flag = nullptr;
  char* arena = nullptr;
};

cudaError_t fill_ghosts_fwd(const Work& w, double* S) {
  const Layout& L = w.v.L;
  const int tx = (L.ny > L.nyd ? L.ny : L.nyd) * 2 * GH;
  ghost_fwd_kernel<<<dim3((tx + 127) / 128, 1, 2), 128, 0, w.v.stream>>>(S, L, w.v.p.bc[0], w.v.p.bc[1], 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ty = ((L.nx > L.nxd ? L.nx : L.nxd) + 2 * GH) * 2 * GH;
  ghost_fwd_kernel<<<dim3((ty + 127) / 128, 1, 2), 128, 0, w.v.stream>>>(S, L, w.v.p.bc[2], w.v.p.bc[3], 1);
  return cudaGetLastError();
}

// adjoint of the ghost fill: the y pass first (its sources include x ghosts)
cudaError_t fold_ghosts(const Work& w, double* Sa) {
  const Layout& L = w.v.L;
  const int ty = ((L.nx > L.nxd ? L.nx : L.nxd) + 2 * GH) * 2 * GH;
  ghost_adj_kernel<<<dim3((ty + 127) / 128, 1, 2), 128, 0, w.v.stream>>>(Sa, L, w.v.p.bc[2], w.v.p.bc[3], 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int tx = (L.ny > L.nyd ? L.ny : L.nyd) * 2 * GH;
  ghost_adj_kernel<<<dim3((tx + 127) / 128, 1, 2), 128, 0, w.v.stream>>>(Sa, L, w.v.p.bc[0], w.v.p.bc[1], 0);
  return cudaGetLastError();
}

KArgs<double> stage_args(const Work& w, double dt, int stage) {
  KArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.L = w.v.L;
  a.geno = make_geno<double>(w.v.p.geno_variant);
  a.gas = make_gas<double>(w.v.p, dt);
  a.hd[0] = a.h[0] = w.v.hx;
  a.hd[1] = a.h[1] = w.v.hy;
  a.ihd[0] = a.ih[0] = 1.0 / w.v.hx;
  a.ihd[1] = a.ih[1] = 1.0 / w.v.hy;
  for (int k = 0; k < 4; ++k) a.bc[k] = w.v.p.bc[k];
  a.flux_variant = w.v.p.flux_variant;
  a.grad_base = w.v.p.grad_base;
  a.want_n = stage == 0 ? 1 : 0;
  a.dt = dt;
  a.flag = w.flag;
  a.Sn = w.Sn;
  a.Wacc = w.Wacc;
  a.gB = w.gB;
  if (stage == 0) {
    a.S = w.Sn;
    a.Sout = w.S2;
    a.NF = w.NF1;
    a.PA = w.P1A;
    a.PB = w.P1B;
  } else {
    a.S = w.S2;
    a.Sout = w.Snext;
    a.NF = w.NF2;
    a.PA = w.P2A;
    a.PB = w.P2B;
  }
  a.Sr = a.S;
  return a;
}

// one forward step from `in` (padded, interior valid) into `out`, keeping the
// stage intermediates in the work buffers (Sn holds `in` with ghosts)
cudaError_t forward_step(const Work& w, double dt, const double* in, double* out) {
  cudaStream_t s = w.v.stream;
  cudaError_t e = cudaMemcpyAsync(w.Sn, in, w.fs, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  for (int stage = 0; stage < 2; ++stage) {
    KArgs<double> a = stage_args(w, dt, stage);
    if ((e = fill_ghosts_fwd(w, const_cast<double*>(a.Sr))) != cudaSuccess) return e;
    if ((e = launch_nodal<double>(a, s)) != cudaSuccess) return e;
    if ((e = launch_points<double>(a, s)) != cudaSuccess) return e;
    if ((e = launch_update<double>(a, stage == 0 ? UPD_STAGE1 : UPD_STAGE2, s)) != cudaSuccess) return e;
  }
  if (out != w.Snext) e = cudaMemcpyAsync(out, w.Snext, w.fs, cudaMemcpyDeviceToDevice, s);
  return e;
}

// reverse of one step: Aout (adjoint of the step's output) -> Ain (of its
// input), given the intermediates of that step in the work buffers
cudaError_t adjoint_step(const Work& w, double dt, const double* Aout, double* Ain) {
  cudaStream_t s = w.v.stream;
  const Layout& L = w.v.L;
  const size_t pbytes = sizeof(double) * NPT * L.pplane, nbytes = sizeof(double) * 2 * NNF * L.plane;
  const dim3 b(32, 4);
  const int mx = L.nx > L.nxd ? L.nx : L.nxd, my = L.ny > L.nyd ? L.ny : L.nyd;
  const dim3 gu = grid2(mx, my, b, 2), gn = grid2(mx + 2, my + 2, b, 2);
  const dim3 gA = grid2(L.nx + 3, L.nyd + 3, b, 1), gB = grid2(L.nxd + 3, L.ny + 3, b, 1);
  cudaError_t e;
  // the FP32 path's GENO rounding floor (64 u, u = 2^-24) for mixed contexts
  const double fscale = w.v.p.precision == FDCGKS_MIXED ? 64.0 * 5.9604644775390625e-8 : 0.0;
  for (int stage = 1; stage >= 0; --stage) {
    const KArgs<double> a = stage_args(w, dt, stage);
    double* target = stage == 1 ? w.As : Ain;   // adjoint of this stage's input state
    const double* aout = stage == 1 ? Aout : w.As;
    if ((e = cudaMemsetAsync(w.PAa, 0, pbytes, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.PBa, 0, pbytes, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.NFa, 0, nbytes, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(target, 0, w.fs, s)) != cudaSuccess) return e;
    update_adj_kernel<<<gu, b, 0, s>>>(a, stage, aout, w.Aacc, w.AgB, Ain, w.PAa, w.PBa, w.NFa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    point_vjp_kernel<0><<<gA, b, 0, s>>>(a, w.PAa, target, fscale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    point_vjp_kernel<1><<<gB, b, 0, s>>>(a, w.PBa, target, fscale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    nodal_vjp_kernel<<<gn, b, 0, s>>>(a, w.NFa, target, fscale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = fold_ghosts(w, target)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// dense [4][ny][nx] / [2][4][ny][nx] <-> padded planes of one grid
cudaError_t dense_copy(const Work& w, double* pad, const double* Wsrc, const double* Gsrc, double* Wdst,
                       double* Gdst, int g) {
  const Layout& L = w.v.L;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  const long NN = (long)nxg * nyg;
  for (int f = 0; f < NFLD; ++f) {
    double* p = pad + ((long)g * NFLD + f) * L.plane + cell(L, 0, 0);
    cudaError_t e;
    if (Wsrc) {
      const double* src = f < 4 ? Wsrc + f * NN : Gsrc + (f - 4) * NN;
      e = cudaMemcpy2DAsync(p, sizeof(double) * L.pitch, src, sizeof(double) * nxg, sizeof(double) * nxg, nyg,
                            cudaMemcpyDeviceToDevice, w.v.stream);
    } else {
      double* dst = f < 4 ? Wdst + f * NN : Gdst + (f - 4) * NN;
      e = cudaMemcpy2DAsync(dst, sizeof(double) * nxg, p, sizeof(double) * L.pitch, sizeof(double) * nxg, nyg,
                            cudaMemcpyDeviceToDevice, w.v.stream);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

fdcgks_status afail(fdcgks_t c, fdcgks_status s, const char* what, cudaError_t e = cudaSuccess) {
  char m[400];
  if (e != cudaSuccess) snprintf(m, sizeof(m), "%s: %s", what, cudaGetErrorString(e));
  else snprintf(m, sizeof(m), "%s", what);
  ctx_set_error(c, m);
  return s;
}

}  // namespace

extern "C" fdcgks_status fdcgks_vjp_steps(fdcgks_t ctx, double dt, int nsteps, int checkpoint_every,
                                          const double* Wp0, const double* Gp0, const double* Wd0, const double* Gd0,
                                          const double* aWp, const double* aGp, const double* aWd, const double* aGd,
                                          double* gWp, double* gGp, double* gWd, double* gGd) {
  Work w;
  if (!ctx_view(ctx, &w.v)) return afail(nullptr, FDCGKS_ERR_ARG, "ctx is NULL");
  if (w.v.p.recon_vars != 0)
    return afail(ctx, FDCGKS_ERR_ARG, "the adjoint reconstructs conservative components only");
  if (w.v.has_sides) return afail(ctx, FDCGKS_ERR_ARG, "the adjoint takes the boundary kinds of params.bc only");
  if (!(dt > 0.0) || !std::isfinite(dt)) return afail(ctx, FDCGKS_ERR_ARG, "dt must be positive and finite");
  if (nsteps < 0 || checkpoint_every < 1) return afail(ctx, FDCGKS_ERR_ARG, "nsteps >= 0 and checkpoint_every >= 1");
  const void* ptrs[] = {Wp0, Gp0, Wd0, Gd0, aWp, aGp, aWd, aGd, gWp, gGp, gWd, gGd};
  for (const void* q : ptrs)
    if (!q) return afail(ctx, FDCGKS_ERR_ARG, "NULL array");
  fdcgks_status st = fdcgks_set_state(ctx, Wp0, Gp0, Wd0, Gd0, 1);
  if (st != FDCGKS_OK) return st;
  ctx_view(ctx, &w.v);
  const Layout& L = w.v.L;
  cudaStream_t s = w.v.stream;
  w.fs = sizeof(double) * 2 * NFLD * L.plane;
  const int nck = nsteps == 0 ? 1 : (nsteps + checkpoint_every - 1) / checkpoint_every;
  const int nseg = std::max(1, std::min(nsteps, checkpoint_every));
  const size_t pb = sizeof(double) * NPT * L.pplane, nb = sizeof(double) * 2 * NNF * L.plane;
  const size_t acc = sizeof(double) * 2 * 4 * L.plane, gbb = sizeof(double) * 2 * 8 * L.plane;
  const bool mixed = w.v.p.precision == FDCGKS_MIXED;
  const size_t sizes[] = {w.fs, w.fs, w.fs, acc, gbb, pb, pb, pb, pb, nb, nb,
                          w.fs, w.fs, w.fs, acc, gbb, pb, pb, nb, 256, mixed ? w.fs : 0};
  double** slots[] = {&w.Sn, &w.S2, &w.Snext, &w.Wacc, &w.gB, &w.P1A, &w.P1B, &w.P2A, &w.P2B, &w.NF1, &w.NF2,
                      &w.A0, &w.A1, &w.As, &w.Aacc, &w.AgB, &w.PAa, &w.PBa, &w.NFa, (double**)&w.flag, &w.fin};
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t total = 0;
  for (size_t b : sizes) total += r256(b);
  total += (size_t)(nck + nseg) * r256(w.fs);
  cudaError_t e = cudaMalloc((void**)&w.arena, total);
  if (e != cudaSuccess) return afail(ctx, FDCGKS_ERR_NOMEM, "adjoint workspace", e);
  size_t off = 0;
  for (size_t k = 0; k < sizeof(sizes) / sizeof(sizes[0]); ++k) {
    *slots[k] = (double*)(w.arena + off);
    off += r256(sizes[k]);
  }
  for (int k = 0; k < nck; ++k, off += r256(w.fs)) w.ck.push_back((double*)(w.arena + off));
  for (int k = 0; k < nseg; ++k, off += r256(w.fs)) w.seg.push_back((double*)(w.arena + off));

  // one step of the trajectory: the FP64 step itself, or the context's mixed
  // step replayed between FP64 buffers
  auto advance = [&](const double* in, double* out) -> fdcgks_status {
    if (mixed) return ctx_replay_step(ctx, dt, in, out);
    cudaError_t r = forward_step(w, dt, in, out);
    return r == cudaSuccess ? FDCGKS_OK : afail(ctx, FDCGKS_ERR_CUDA, "forward", r);
  };
  auto run = [&]() -> fdcgks_status {
    cudaError_t r = cudaMemsetAsync(w.arena, 0, total, s);
    if (r != cudaSuccess) return afail(ctx, FDCGKS_ERR_CUDA, "workspace clear", r);
    // forward sweep with checkpoints
    if ((r = cudaMemcpyAsync(w.ck[0], w.v.S, w.fs, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return afail(ctx, FDCGKS_ERR_CUDA, "checkpoint", r);
    const double* cur = w.ck[0];
    fdcgks_status fs;
    for (int m = 0; m < nsteps; ++m) {
      if ((fs = advance(cur, w.Snext)) != FDCGKS_OK) return fs;
      const int k = (m + 1) / checkpoint_every;
      double* dst = ((m + 1) % checkpoint_every == 0 && k < nck) ? w.ck[k] : w.seg[0];
      if ((r = cudaMemcpyAsync(dst, w.Snext, w.fs, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return afail(ctx, FDCGKS_ERR_CUDA, "forward", r);
      cur = dst;
    }
    // the context keeps the final state (a mixed context's buffers are reused
    // by the replays below, so its final state is loaded back at the end)
    if ((r = cudaMemcpyAsync(mixed ? w.fin : w.v.S, cur, w.fs, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return afail(ctx, FDCGKS_ERR_CUDA, "final state", r);
    // adjoint of the final state
    double* Aout = w.A0;
    double* Ain = w.A1;
    if ((r = dense_copy(w, Aout, aWp, aGp, nullptr, nullptr, 0)) != cudaSuccess ||
        (r = dense_copy(w, Aout, aWd, aGd, nullptr, nullptr, 1)) != cudaSuccess)
      return afail(ctx, FDCGKS_ERR_CUDA, "adjoint seed", r);
    // reverse sweep, one checkpoint segment at a time
    for (int k = nck - 1; k >= 0; --k) {
      const int m0 = k * checkpoint_every, m1 = std::min(nsteps, m0 + checkpoint_every);
      if (m1 <= m0) continue;
      if ((r = cudaMemcpyAsync(w.seg[0], w.ck[k], w.fs, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return afail(ctx, FDCGKS_ERR_CUDA, "segment", r);
      for (int m = m0; m + 1 < m1; ++m)
        if ((fs = advance(w.seg[m - m0], w.seg[m - m0 + 1])) != FDCGKS_OK) return fs;
      for (int m = m1 - 1; m >= m0; --m) {
        if ((r = forward_step(w, dt, w.seg[m - m0], w.Snext)) != cudaSuccess)
          return afail(ctx, FDCGKS_ERR_CUDA, "recompute", r);
        if ((r = adjoint_step(w, dt, Aout, Ain)) != cudaSuccess) return afail(ctx, FDCGKS_ERR_CUDA, "adjoint", r);
        std::swap(Aout, Ain);
      }
    }
    if ((r = dense_copy(w, Aout, nullptr, nullptr, gWp, gGp, 0)) != cudaSuccess ||
        (r = dense_copy(w, Aout, nullptr, nullptr, gWd, gGd, 1)) != cudaSuccess)
      return afail(ctx, FDCGKS_ERR_CUDA, "gradient copy", r);
    if (mixed && (fs = ctx_load_padded(ctx, w.fin)) != FDCGKS_OK) return fs;
    if ((r = cudaStreamSynchronize(s)) != cudaSuccess) return afail(ctx, FDCGKS_ERR_CUDA, "adjoint", r);
    return FDCGKS_OK;
  };
  st = run();
  cudaStreamSynchronize(s);
  cudaFree(w.arena);
  return st;
}
