// Templated CUDA kernels of the FD-CGKS stage (Sec. 4 of the paper): nodal
// reconstruction + flux, virtual-interface points (two line reconstructions
// shared by the primary-grid and dual-grid solves), and the fused compact
// finite-difference + S2O4 update.  Included by one translation unit per
// compute precision.
#pragma once

#include "fdcgks_internal.cuh"

// Tuning knobs of the interface-point kernel (defaults are the tuned values):
// FDK_POINT_MINB   minimum resident blocks per SM in the launch bounds
//                  (caps registers per thread), per compute type
// FDK_UPDATE_MINB_F32, FDK_NODAL_MINB_F32  the same for the FP32 update and
//                  nodal kernels (the FP64 kernels are FP64-pipe bound and
//                  are left uncapped).  1024^2 vortex, ms per mixed step:
//                  update 4, 5, 6, 8 gave 0.448, 0.411, 0.382, 0.437; nodal
//                  5, 6, 8, 10, 12, 16 gave 0.303, 0.264, 0.234, 0.221, 0.225,
//                  0.332
// FDK_SOLVE_NOINLINE  1: the kinetic solve is an out-of-line function called
//                  twice (one code copy per kernel), 0: inlined twice.  With the
//                  reconstruction also out of line (below) the smaller code
//                  runs 3.6 % (mixed) and 0.8 % (FP64) faster per step on the
//                  1024^2 vortex than both inlined
#ifndef FDK_POINT_MINB_F64
#define FDK_POINT_MINB_F64 1
#endif
#ifndef FDK_POINT_MINB_F32
#define FDK_POINT_MINB_F32 4
#endif
#ifndef FDK_UPDATE_MINB_F32
#define FDK_UPDATE_MINB_F32 6
#endif
#ifndef FDK_NODAL_MINB_F32
#define FDK_NODAL_MINB_F32 10
#endif
#ifndef FDK_SOLVE_NOINLINE_F64
#define FDK_SOLVE_NOINLINE_F64 1
#endif
#ifndef FDK_SOLVE_NOINLINE_F32
#define FDK_SOLVE_NOINLINE_F32 1
#endif
// FDK_RECON_NOINLINE_F32 / _F64  1: the per-component interface reconstruction
//                  of the point kernels is an out-of-line function (one code copy
//                  instead of eight inlined ones), 0: inlined
#ifndef FDK_RECON_NOINLINE_F32
#define FDK_RECON_NOINLINE_F32 1
#endif
#ifndef FDK_RECON_NOINLINE_F64
#define FDK_RECON_NOINLINE_F64 1
#endif
// FDK_POINT_PAIR_F32 / _F64  1: two threads per interface point (one line and
//                  one solve each, coupled by warp shuffles; point_pair_kernel),
//                  0: one thread per point (point_kernel).  On the 1024^2 vortex
//                  the pair form takes the mixed point phase from 1.019 to
//                  0.903 ms per step and the FP64 one from 32.06 to 31.41 ms
// FDK_POINT_PAIR_MINB_F32 / _F64  minimum resident blocks per SM of the pair
//                  kernel (FP32 without preload: 2, 3, 4, 5 gave 1.43, 1.06,
//                  0.915, 0.903 ms; with preload 4 and 5 give 0.822 and 0.840)
#ifndef FDK_POINT_PAIR_F32
#define FDK_POINT_PAIR_F32 1
#endif
#ifndef FDK_POINT_PAIR_F64
#define FDK_POINT_PAIR_F64 1
#endif
#ifndef FDK_POINT_PAIR_MINB_F32
#define FDK_POINT_PAIR_MINB_F32 4
#endif
#ifndef FDK_POINT_PAIR_MINB_F64
#define FDK_POINT_PAIR_MINB_F64 1
#endif
// FDK_PAIR_PRELOAD_F32  1: a pair-kernel thread loads its line's 32 values (4
//                  entries x W and the gradient along the line) into registers
//                  before the first reconstruction, so the loads are not issued
//                  between the out-of-line reconstruction calls (mixed point
//                  phase 0.903 -> 0.840 ms per step at 5 blocks/SM, 0.822 at 4;
//                  the inlined reconstruction at 4 blocks/SM: 0.914)
#ifndef FDK_PAIR_PRELOAD_F32
#define FDK_PAIR_PRELOAD_F32 1
#endif

namespace fdk {

template <class R> struct PointTune;
template <> struct PointTune<double> {
  static constexpr int minb = FDK_POINT_MINB_F64;
  static constexpr int update_minb = 1;
  static constexpr int nodal_minb = 1;
  static constexpr bool noinline = FDK_SOLVE_NOINLINE_F64;
  static constexpr bool pair = FDK_POINT_PAIR_F64;
  static constexpr int pair_minb = FDK_POINT_PAIR_MINB_F64;
};
template <> struct PointTune<float> {
  static constexpr int minb = FDK_POINT_MINB_F32;
  static constexpr int update_minb = FDK_UPDATE_MINB_F32;
  static constexpr int nodal_minb = FDK_NODAL_MINB_F32;
  static constexpr bool noinline = FDK_SOLVE_NOINLINE_F32;
  static constexpr bool pair = FDK_POINT_PAIR_F32;
  static constexpr int pair_minb = FDK_POINT_PAIR_MINB_F32;
};

// interface reconstruction of one component, inlined or out of line (the
// adjoint's dual numbers always inline)
template <class R> struct ReconCall { static constexpr bool noinline = false; };
template <> struct ReconCall<float> { static constexpr bool noinline = FDK_RECON_NOINLINE_F32; };
template <> struct ReconCall<double> { static constexpr bool noinline = FDK_RECON_NOINLINE_F64; };

template <class R>
struct ReconOne { R vl, dl, cl, vr, dr, cr; };

template <class R>
__device__ __noinline__ ReconOne<R> recon_interface_call(const GenoK<R>& g, R q0, R q1, R q2, R q3, R x0, R x1, R x2,
                                                         R x3, R h, R ih) {
  const R Q[4] = {q0, q1, q2, q3}, Qx[4] = {x0, x1, x2, x3};
  ReconOne<R> o;
  recon_interface(g, Q, Qx, h, ih, o.vl, o.dl, o.cl, o.vr, o.dr, o.cr);
  return o;
}

template <class R>
FD_HD void recon_interface_sel(const GenoK<R>& g, const R Q[4], const R Qx[4], R h, R ih, R& vl, R& dl, R& cl, R& vr,
                               R& dr, R& cr) {
#ifdef __CUDA_ARCH__
  if constexpr (ReconCall<R>::noinline) {
    const ReconOne<R> o = recon_interface_call(g, Q[0], Q[1], Q[2], Q[3], Qx[0], Qx[1], Qx[2], Qx[3], h, ih);
    vl = o.vl; dl = o.dl; cl = o.cl; vr = o.vr; dr = o.dr; cr = o.cr;
    return;
  }
#endif
  recon_interface(g, Q, Qx, h, ih, vl, dl, cl, vr, dr, cr);
}

template <class R>
__device__ __noinline__ void iface_solve_call(const GasK<R>& gas, int normal, const R* Wl, const R* Wr, const R* Wln,
                                             const R* Wrn, const R* Wt, bool want_n, IfaceOut<R>& o) {
  iface_solve(gas, normal, Wl, Wr, Wln, Wrn, Wt, want_n, o);
}

// ---------------------------------------------------------------------------
// nodal reconstruction and flux (Sec. 4 item 2; Sec. 2.1 nodal fluxes)
// one thread per node, nodes i in [-1, n_x], j in [-1, n_y] of grid blockIdx.z
// ---------------------------------------------------------------------------
// One node: GENO node derivatives along x and y, then the nodal flux.
// ld(e, f): field f (0-3 W, 4-7 x-gradient, 8-11 y-gradient) of node e (0 the
// node, 1/2 its x neighbours -/+, 3/4 its y neighbours -/+); st(k, v): output
// k (F[4], G[4], F_t[4], G_t[4]); want_n = false (second S2O4 stage): F_t and
// G_t only, F and G are neither computed nor stored.
template <class R, class LD, class ST>
FD_HD void nodal_compute(const GenoK<R>& geno, const GasK<R>& gas, const R h[2], const R ih[2], LD ld, ST st,
                         bool want_n = true) {
  R W[4], Wx[4], Wy[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    W[c] = ld(0, c);
    R qx[3] = {ld(1, c), W[c], ld(2, c)};
    R gxv[3] = {ld(1, 4 + c), ld(0, 4 + c), ld(2, 4 + c)};
    Wx[c] = recon_node(geno, qx, gxv, h[0], ih[0]);
    R qy[3] = {ld(3, c), W[c], ld(4, c)};
    R gyv[3] = {ld(3, 8 + c), ld(0, 8 + c), ld(4, 8 + c)};
    Wy[c] = recon_node(geno, qy, gyv, h[1], ih[1]);
  }
  R F[4], G[4], Ft[4], Gt[4];
  nodal_flux(gas, W, Wx, Wy, F, G, Ft, Gt, want_n);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (want_n) {
      st(c, F[c]);
      st(4 + c, G[c]);
    }
    st(8 + c, Ft[c]);
    st(12 + c, Gt[c]);
  }
}

// offset of node e of the nodal stencil (see nodal_compute) from the node
FD_HD long nodal_offset(const Layout& L, int e) {
  return e == 0 ? 0 : e == 1 ? -1 : e == 2 ? 1 : e == 3 ? -(long)L.pitch : (long)L.pitch;
}

template <class R>
__device__ __forceinline__ void nodal_body(const KArgs<R>& a, int g, int i, int j) {
  const Layout& L = a.L;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  if (i < -1 || j < -1 || i > nxg || j > nyg) return;
  const R* S = a.Sr + (long)g * NFLD * L.plane;
  const long c0 = cell(L, i, j);
  R* NF = a.NF + (long)g * NNF * L.plane + c0;
  nodal_compute<R>(
      a.geno, a.gas, a.h, a.ih, [&](int e, int f) -> R { return S[(long)f * L.plane + c0 + nodal_offset(L, e)]; },
      [&](int k, R v) { NF[(long)k * L.plane] = v; }, a.want_n != 0);
}

template <class R>
__global__ void __launch_bounds__(128, PointTune<R>::nodal_minb) nodal_kernel(KArgs<R> a) {
  nodal_body(a, blockIdx.z, blockIdx.x * blockDim.x + threadIdx.x - 1, blockIdx.y * blockDim.y + threadIdx.y - 1);
}

// Positivity safeguard of the interface states (the paper describes none): a
// reconstructed state with non-positive or non-finite density or pressure
// (physical_state, fdcgks_math.cuh) is replaced by the state of the node on
// its side (line entries 1 and 2) with zero normal slope, and the interface's
// chi by 0, so its compact flux takes the low-order form.  Never triggered by
// smooth data.
// the safeguard applied to the left/right states of line l
template <class R, class LD>
FD_HD void positivity_fix(LD ld, int l, R vl[4], R dl[4], R vr[4], R dr[4], R& chi) {
  if (!physical_state(vl)) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      vl[c] = ld(l, 1, c);
      dl[c] = R(0);
    }
    chi = R(0);
  }
  if (!physical_state(vr)) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      vr[c] = ld(l, 2, c);
      dr[c] = R(0);
    }
    chi = R(0);
  }
}

// Reconstruct one 4-point line at its virtual interface (between entries 1
// and 2), with the safeguard above.  ld(l, e, f) = field f (0-3 W, 4-7 the
// averaged gradient along the line) of entry e (0-3) of line l.
template <class R, class LD>
FD_HD void recon_line_ld(const GenoK<R>& geno, LD ld, int l, R h, R ih, R vl[4], R dl[4], R vr[4], R dr[4],
                         R& chi) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    R Q[4] = {ld(l, 0, c), ld(l, 1, c), ld(l, 2, c), ld(l, 3, c)};
    R Qx[4] = {ld(l, 0, 4 + c), ld(l, 1, 4 + c), ld(l, 2, 4 + c), ld(l, 3, 4 + c)};
    R cl, cr;
    recon_interface_sel(geno, Q, Qx, h, ih, vl[c], dl[c], cl, vr[c], dr[c], cr);
    if (c == 0) chi = s_min(cl, cr);   // chi_{j+1/2} = min(chi^{l,rho}, chi^{r,rho})
  }
  positivity_fix(ld, l, vl, dl, vr, dr, chi);
}

// The same on characteristic components (Sec. 3.1, "characteristic component
// of W"; recon_vars = 1): the eigenvectors of the Euler flux Jacobian along
// the line's normal, frozen at the mean of entries 1 and 2, in the order
// (rho, m_n, m_t, E); rows of L / columns of R: U - c, entropy, shear, U + c.
// Values and gradients are projected with L, each component reconstructed,
// values and derivatives mapped back with R; chi of the flux is the smaller
// of the two acoustic fields' (Sec. 3.2).  A non-physical mean state falls
// back to conservative components.
template <class R, class LD>
FD_HD void recon_line_char(const GenoK<R>& geno, R gm1, int normal, LD ld, int l, R h, R ih, R vl[4], R dl[4],
                           R vr[4], R dr[4], R& chi) {
  const int in = normal == 0 ? 1 : 2, it = normal == 0 ? 2 : 1;
  const int perm[4] = {0, in, it, 3};
  const R r = R(0.5) * (ld(l, 1, 0) + ld(l, 2, 0));
  const R mn = R(0.5) * (ld(l, 1, in) + ld(l, 2, in)), mt = R(0.5) * (ld(l, 1, it) + ld(l, 2, it));
  const R E = R(0.5) * (ld(l, 1, 3) + ld(l, 2, 3));
  const R ir = s_div(R(1), r), u = mn * ir, v = mt * ir;
  const R q2 = u * u + v * v;
  const R p = gm1 * (E - R(0.5) * r * q2);
  if (!(r > R(0)) || !(p > R(0))) {
    recon_line_ld(geno, ld, l, h, ih, vl, dl, vr, dr, chi);
    return;
  }
  const R c = s_sqrt((gm1 + R(1)) * p * ir), ic = s_div(R(1), c), H = (E + p) * ir;
  const R b1 = gm1 * ic * ic, b2 = R(0.5) * b1 * q2;
  const R Lm[4][4] = {{R(0.5) * (b2 + u * ic), -R(0.5) * (b1 * u + ic), -R(0.5) * b1 * v, R(0.5) * b1},
                      {R(1) - b2, b1 * u, b1 * v, -b1},
                      {-v, R(0), R(1), R(0)},
                      {R(0.5) * (b2 - u * ic), -R(0.5) * (b1 * u - ic), -R(0.5) * b1 * v, R(0.5) * b1}};
  const R Rm[4][4] = {{R(1), R(1), R(0), R(1)},
                      {u - c, u, R(0), u + c},
                      {v, v, R(1), v},
                      {H - u * c, R(0.5) * q2, v, H + u * c}};
  R cvl[4], cdl[4], cvr[4], cdr[4], cl[4], cr[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    R Q[4], Qx[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      R a = R(0), b = R(0);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a += Lm[k][j] * ld(l, m, perm[j]);
        b += Lm[k][j] * ld(l, m, 4 + perm[j]);
      }
      Q[m] = a;
      Qx[m] = b;
    }
    recon_interface_sel(geno, Q, Qx, h, ih, cvl[k], cdl[k], cl[k], cvr[k], cdr[k], cr[k]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    R a = R(0), b = R(0), d = R(0), e = R(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a += Rm[j][k] * cvl[k];
      b += Rm[j][k] * cvr[k];
      d += Rm[j][k] * cdl[k];
      e += Rm[j][k] * cdr[k];
    }
    vl[perm[j]] = a;
    vr[perm[j]] = b;
    dl[perm[j]] = d;
    dr[perm[j]] = e;
  }
  chi = s_min(s_min(cl[0], cr[0]), s_min(cl[3], cr[3]));
  positivity_fix(ld, l, vl, dl, vr, dr, chi);
}

// One virtual-interface point: the two line reconstructions (with the
// safeguard), the tangential derivatives, the two kinetic solves and the W~
// combination.  ld(l, e, f) as for recon_line_ld, line 0 being the
// primary-grid line (normal TYPE, spacing h[TYPE]) and line 1 the dual-grid
// line (normal 1 - TYPE); st(k, v): output k (PO_* of solve 0, NPS + PO_* of
// solve 1; F and W~ values only when wn).  Shared by the kernel and its adjoint.
template <class R, int TYPE, bool CHAR = false, class LD, class ST>
FD_HD void point_compute(const GenoK<R>& geno, const GasK<R>& gas, const R h[2], const R ih[2], bool wn, LD ld,
                         ST st) {
  const int n0 = TYPE;        // normal of the primary-grid solve
  R l0v[4], l0d[4], r0v[4], r0d[4], chi0;
  R l1v[4], l1d[4], r1v[4], r1d[4], chi1;
  if constexpr (CHAR) {
    recon_line_char(geno, gas.gm1, n0, ld, 0, h[n0], ih[n0], l0v, l0d, r0v, r0d, chi0);
    recon_line_char(geno, gas.gm1, 1 - n0, ld, 1, h[1 - n0], ih[1 - n0], l1v, l1d, r1v, r1d, chi1);
  } else {
    recon_line_ld(geno, ld, 0, h[n0], ih[n0], l0v, l0d, r0v, r0d, chi0);
    recon_line_ld(geno, ld, 1, h[1 - n0], ih[1 - n0], l1v, l1d, r1v, r1d, chi1);
  }
  // tangential derivative of each solve: mean of the other line's l/r derivatives
  R t0[4], t1[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    t0[c] = R(0.5) * (l1d[c] + r1d[c]);
    t1[c] = R(0.5) * (l0d[c] + r0d[c]);
  }
  IfaceOut<R> o0, o1;
  if constexpr (PointTune<R>::noinline) {
    iface_solve_call(gas, n0, l0v, r0v, l0d, r0d, t0, wn, o0);
    iface_solve_call(gas, 1 - n0, l1v, r1v, l1d, r1d, t1, wn, o1);
  } else {
    iface_solve(gas, n0, l0v, r0v, l0d, r0d, t0, wn, o0);
    iface_solve(gas, 1 - n0, l1v, r1v, l1d, r1d, t1, wn, o1);
  }
  // W~ of Eq. (eq:W-model-2d): half of the own solve plus a quarter of each side of the other
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    R m1t = R(0.25) * (o1.Wlt[c] + o1.Wrt[c]), m0t = R(0.25) * (o0.Wlt[c] + o0.Wrt[c]);
    st(PO_FT + c, o0.Ft[c]);
    st(PO_WLT + c, R(0.5) * o0.Wlt[c] + m1t);
    st(PO_WRT + c, R(0.5) * o0.Wrt[c] + m1t);
    st(NPS + PO_FT + c, o1.Ft[c]);
    st(NPS + PO_WLT + c, R(0.5) * o1.Wlt[c] + m0t);
    st(NPS + PO_WRT + c, R(0.5) * o1.Wrt[c] + m0t);
    if (wn) {
      R m1 = R(0.25) * (o1.Wl[c] + o1.Wr[c]), m0 = R(0.25) * (o0.Wl[c] + o0.Wr[c]);
      st(PO_F + c, o0.F[c]);
      st(PO_WL + c, R(0.5) * o0.Wl[c] + m1);
      st(PO_WR + c, R(0.5) * o0.Wr[c] + m1);
      st(NPS + PO_F + c, o1.F[c]);
      st(NPS + PO_WL + c, R(0.5) * o1.Wl[c] + m0);
      st(NPS + PO_WR + c, R(0.5) * o1.Wr[c] + m0);
    }
  }
  st(PO_CHI, chi0);
  st(NPS + PO_CHI, chi1);
}

// Where the lines of point (i, j) lie in the padded state: entry e of line l
// is at base[l] + e * stride[l] of grid l (primary 0, dual 1), its gradient
// along the line in fields gfield[l]..gfield[l] + 3.
struct PointLines {
  long base[2], stride[2];
  int gfield[2];
};
template <int TYPE>
FD_HD PointLines point_lines(const Layout& L, int i, int j) {
  PointLines p;
  if (TYPE == 0) {
    // primary nodes (i-1..i+2, j) along x; dual nodes (i+1, j-1..j+2) along y
    p.base[0] = cell(L, i - 1, j); p.stride[0] = 1; p.gfield[0] = 4;
    p.base[1] = cell(L, i + 1, j - 1); p.stride[1] = L.pitch; p.gfield[1] = 8;
  } else {
    // primary nodes (i, j-1..j+2) along y; dual nodes (i-1..i+2, j+1) along x
    p.base[0] = cell(L, i, j - 1); p.stride[0] = L.pitch; p.gfield[0] = 8;
    p.base[1] = cell(L, i - 1, j + 1); p.stride[1] = 1; p.gfield[1] = 4;
  }
  return p;
}

// ---------------------------------------------------------------------------
// virtual-interface points (Sec. 4 item 1; App. A3).
// TYPE 0 = point A (i+1/2, j): primary x-interface, dual y-interface of dual column i+1
// TYPE 1 = point B (i, j+1/2): primary y-interface, dual x-interface of dual row j+1
// ---------------------------------------------------------------------------
template <class R, int TYPE, bool CHAR = false>
__device__ __forceinline__ void point_body(const KArgs<R>& a, int i, int j) {
  const Layout& L = a.L;
  const int imax = TYPE == 0 ? L.nx : L.nxd;
  const int jmax = TYPE == 0 ? L.nyd : L.ny;
  if (i < -2 || j < -2 || i > imax || j > jmax) return;
  const PointLines pl = point_lines<TYPE>(L, i, j);
  const R* S = a.Sr;
  R* P = (TYPE == 0 ? a.PA : a.PB) + pcell(L, i, j);
  const long pp = L.pplane;
  point_compute<R, TYPE, CHAR>(
      a.geno, a.gas, a.h, a.ih, a.want_n != 0,
      [&](int l, int e, int f) -> R {
        const int field = f < 4 ? f : pl.gfield[l] + (f - 4);
        return S[((long)l * NFLD + field) * L.plane + pl.base[l] + e * pl.stride[l]];
      },
      [&](int k, R v) { P[(long)k * pp] = v; });
}

template <class R, int TYPE, bool CHAR>
__global__ void __launch_bounds__(128, PointTune<R>::minb) point_kernel(KArgs<R> a) {
  point_body<R, TYPE, CHAR>(a, blockIdx.x * blockDim.x + threadIdx.x - 2,
                            blockIdx.y * blockDim.y + threadIdx.y - 2);
}

// ---------------------------------------------------------------------------
// The same point with two threads (lanes 2k and 2k + 1 of a warp): lane
// parity l reconstructs line l and runs solve l (l = 0 the primary-grid solve
// with normal TYPE, l = 1 the dual-grid solve).  What couples the two solves
// of a point travels between the partner lanes by warp shuffles: the
// tangential derivative of each solve (the mean of the other line's l/r
// derivatives) and the other solve's quarter in W~ (Eq. eq:W-model-2d).
// Each thread holds one line and one solve instead of two, so the solve runs
// inline without a local-memory call frame; the arithmetic is point_compute's,
// in the same order.  mask: the lanes of the warp that take part (pairs are
// valid together).
// ---------------------------------------------------------------------------
template <class R, int TYPE, bool CHAR, class LD, class ST>
__device__ __forceinline__ void point_compute_pair(const GenoK<R>& geno, const GasK<R>& gas, const R h[2],
                                                   const R ih[2], bool wn, int l, unsigned mask, LD ld, ST st) {
  const int n = l == 0 ? TYPE : 1 - TYPE;   // normal of this lane's solve
  R lv[4], ldv[4], rv[4], rdv[4], chi;
  if constexpr (CHAR)
    recon_line_char(geno, gas.gm1, n, ld, l, h[n], ih[n], lv, ldv, rv, rdv, chi);
  else
    recon_line_ld(geno, ld, l, h[n], ih[n], lv, ldv, rv, rdv, chi);
  R t[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) t[c] = R(0.5) * __shfl_xor_sync(mask, ldv[c] + rdv[c], 1);
  IfaceOut<R> o;
  iface_solve(gas, n, lv, rv, ldv, rdv, t, wn, o);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const R mt = R(0.25) * __shfl_xor_sync(mask, o.Wlt[c] + o.Wrt[c], 1);
    st(PO_FT + c, o.Ft[c]);
    st(PO_WLT + c, R(0.5) * o.Wlt[c] + mt);
    st(PO_WRT + c, R(0.5) * o.Wrt[c] + mt);
    if (wn) {
      const R m = R(0.25) * __shfl_xor_sync(mask, o.Wl[c] + o.Wr[c], 1);
      st(PO_F + c, o.F[c]);
      st(PO_WL + c, R(0.5) * o.Wl[c] + m);
      st(PO_WR + c, R(0.5) * o.Wr[c] + m);
    }
  }
  st(PO_CHI, chi);
}

// one thread of a point pair: point (i, j), line / solve l
template <class R, int TYPE, bool CHAR>
__device__ __forceinline__ void point_pair_body(const KArgs<R>& a, int i, int j, int l) {
  const Layout& L = a.L;
  const int imax = TYPE == 0 ? L.nx : L.nxd;
  const int jmax = TYPE == 0 ? L.nyd : L.ny;
  const bool valid = !(i < -2 || j < -2 || i > imax || j > jmax);
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const PointLines pl = point_lines<TYPE>(L, i, j);
  const R* S = a.Sr;
  R* P = (TYPE == 0 ? a.PA : a.PB) + pcell(L, i, j) + (long)l * NPS * L.pplane;
  const long pp = L.pplane;
  auto st = [&](int k, R v) { P[(long)k * pp] = v; };
  auto gl = [&](int ll, int e, int f) -> R {
    const int field = f < 4 ? f : pl.gfield[ll] + (f - 4);
    return S[((long)ll * NFLD + field) * L.plane + pl.base[ll] + e * pl.stride[ll]];
  };
#if FDK_PAIR_PRELOAD_F32
  if constexpr (IsF32<R>::v) {
  R xl[32];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int f = 0; f < 8; ++f) xl[e * 8 + f] = gl(l, e, f);
  point_compute_pair<R, TYPE, CHAR>(a.geno, a.gas, a.h, a.ih, a.want_n != 0, l, mask,
                                    [&](int, int e, int f) -> R { return xl[e * 8 + f]; }, st);
  } else {
    point_compute_pair<R, TYPE, CHAR>(a.geno, a.gas, a.h, a.ih, a.want_n != 0, l, mask, gl, st);
  }
#else
  point_compute_pair<R, TYPE, CHAR>(a.geno, a.gas, a.h, a.ih, a.want_n != 0, l, mask, gl, st);
#endif
}

// block (32, 4): 16 points per warp row, two lanes each
template <class R, int TYPE, bool CHAR>
__global__ void __launch_bounds__(128, PointTune<R>::pair_minb) point_pair_kernel(KArgs<R> a) {
  point_pair_body<R, TYPE, CHAR>(a, blockIdx.x * (blockDim.x / 2) + (threadIdx.x >> 1) - 2,
                                 blockIdx.y * blockDim.y + threadIdx.y - 2, threadIdx.x & 1);
}

// ---------------------------------------------------------------------------
// compact FD + S2O4 update (Eqs. eq-conservation-law-2d, fd-conservative-flux*,
// define-averaged-gradient, eq-nodal-update, eq-interface-update).
// One thread per interior node of grid blockIdx.z.
// ---------------------------------------------------------------------------

// one node's stage operator: L, dL/dt (per component), the averaged gradients
// re-evaluated from the interface solution (node's own side) and their time
// derivatives
template <class R>
struct NodeOp {
  R L[4], Lt[4], gbx[4], gby[4], gtx[4], gty[4];
};

template <class R>
__device__ __forceinline__ void node_operator(const KArgs<R>& a, int g, int i, int j, bool want_n, NodeOp<R>& o) {
  const Layout& L = a.L;
  const long pp = L.pplane;
  // x-interface k+1/2 of this grid's row and y-interface k+1/2 of its column
  const R* PX = g == 0 ? a.PA : a.PB + NPS * pp;   // primary: A points solve 0; dual: B points solve 1
  const R* PY = g == 0 ? a.PB : a.PA + NPS * pp;   // primary: B points solve 0; dual: A points solve 1
  auto xi = [&](int k) { return g == 0 ? pcell(L, k, j) : pcell(L, k, j - 1); };
  auto yi = [&](int k) { return g == 0 ? pcell(L, i, k) : pcell(L, i - 1, k); };
  const R* NF = a.NF + (long)g * NNF * L.plane;
  const long cN = cell(L, i, j);
  const int fv = a.flux_variant;
  const R ihx = a.ih[0], ihy = a.ih[1];
  const long xm2 = xi(i - 2), xm1 = xi(i - 1), x0 = xi(i), xp1 = xi(i + 1);
  const long ym2 = yi(j - 2), ym1 = yi(j - 1), y0 = yi(j), yp1 = yi(j + 1);
  const R chixm = PX[PO_CHI * pp + xm1], chix0 = PX[PO_CHI * pp + x0];
  const R chiym = PY[PO_CHI * pp + ym1], chiy0 = PY[PO_CHI * pp + y0];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const R* nF = NF + (long)c * L.plane;
    const R* nG = NF + (long)(4 + c) * L.plane;
    const R* nFt = NF + (long)(8 + c) * L.plane;
    const R* nGt = NF + (long)(12 + c) * L.plane;
    const R* pF = PX + (long)(PO_F + c) * pp;
    const R* pFt = PX + (long)(PO_FT + c) * pp;
    const R* qF = PY + (long)(PO_F + c) * pp;
    const R* qFt = PY + (long)(PO_FT + c) * pp;
    {
      R fp = compact_flux(fv, chix0, pFt[xm1], pFt[x0], pFt[xp1], nFt[cN], nFt[cN + 1]);
      R fm = compact_flux(fv, chixm, pFt[xm2], pFt[xm1], pFt[x0], nFt[cN - 1], nFt[cN]);
      R gp = compact_flux(fv, chiy0, qFt[ym1], qFt[y0], qFt[yp1], nGt[cN], nGt[cN + L.pitch]);
      R gm = compact_flux(fv, chiym, qFt[ym2], qFt[ym1], qFt[y0], nGt[cN - L.pitch], nGt[cN]);
      o.Lt[c] = -(fp - fm) * ihx - (gp - gm) * ihy;
    }
    o.L[c] = R(0);
    o.gbx[c] = R(0);
    o.gby[c] = R(0);
    if (want_n) {
      R fp = compact_flux(fv, chix0, pF[xm1], pF[x0], pF[xp1], nF[cN], nF[cN + 1]);
      R fm = compact_flux(fv, chixm, pF[xm2], pF[xm1], pF[x0], nF[cN - 1], nF[cN]);
      R gp = compact_flux(fv, chiy0, qF[ym1], qF[y0], qF[yp1], nG[cN], nG[cN + L.pitch]);
      R gm = compact_flux(fv, chiym, qF[ym2], qF[ym1], qF[y0], nG[cN - L.pitch], nG[cN]);
      o.L[c] = -(fp - fm) * ihx - (gp - gm) * ihy;
      o.gbx[c] = (PX[(PO_WL + c) * pp + x0] - PX[(PO_WR + c) * pp + xm1]) * ihx;
      o.gby[c] = (PY[(PO_WL + c) * pp + y0] - PY[(PO_WR + c) * pp + ym1]) * ihy;
    }
    o.gtx[c] = (PX[(PO_WLT + c) * pp + x0] - PX[(PO_WRT + c) * pp + xm1]) * ihx;
    o.gty[c] = (PY[(PO_WLT + c) * pp + y0] - PY[(PO_WRT + c) * pp + ym1]) * ihy;
  }
}

// float-float (double-word) accumulation for the mixed path: Knuth's TwoSum
// gives s + e = a + b exactly; Dekker's FastTwoSum renormalises hi + lo
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float v = s - a;
  e = (a - (s - v)) + (b - v);
}
__device__ __forceinline__ void ff_add(float& hi, float& lo, float b) {
  float s, e;
  two_sum(hi, b, s, e);
  e += lo;
  hi = s + e;
  lo = e - (hi - s);
}

template <class R>
__device__ __forceinline__ void update_body(const KArgs<R>& a, int mode, int g, int i, int j) {
  const Layout& L = a.L;
  const int nxg = g == 0 ? L.nx : L.nxd, nyg = g == 0 ? L.ny : L.nyd;
  if (i < 0 || j < 0 || i >= nxg || j >= nyg) return;
  NodeOp<R> o;
  node_operator(a, g, i, j, mode != UPD_STAGE2, o);
  const long c0 = cell(L, i, j);
  if (mode == UPD_OPERATOR) {
    const long NN = (long)nxg * nyg, oi = (long)j * nxg + i;
    double* const* op = a.op + 4 * g;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      op[0][c * NN + oi] = (double)o.L[c];
      op[1][c * NN + oi] = (double)o.Lt[c];
      op[2][c * NN + oi] = (double)o.gbx[c];
      op[2][(4 + c) * NN + oi] = (double)o.gby[c];
      op[3][c * NN + oi] = (double)o.gtx[c];
      op[3][(4 + c) * NN + oi] = (double)o.gty[c];
    }
    return;
  }
  // dual nodes on a no-slip wall: velocity set to zero (internal energy kept),
  // and, as U = V = 0 along the whole wall, the momentum gradients along it too
  const bool xwall = g == 1 && ((a.bc[0] == 3 && i == 0) || (a.bc[1] == 3 && i == nxg - 1));
  const bool ywall = g == 1 && ((a.bc[2] == 3 && j == 0) || (a.bc[3] == 3 && j == nyg - 1));
  const long P = L.plane;

  if constexpr (IsF32<R>::v) {
    // mixed path: state and accumulators are float-float pairs; increments are
    // formed in FP32 and added exactly (two_sum) to the pairs
    const float dtr = a.gas.dt_r;
    float Wh[4], Wl[4], Gh[8], Gl[8];
    const float* Snh = a.Sn_hi + (long)g * NFLD * P;
    const float* Snl = a.Sn_lo + (long)g * NFLD * P;
    float* Ah = a.Acc_hi + (long)g * 4 * P;
    float* Al = a.Acc_lo + (long)g * 4 * P;
    float* Bh = a.Gb_hi + (long)g * 8 * P;
    float* Bl = a.Gb_lo + (long)g * 8 * P;
    // every input pair is loaded before the first store, so that the loads
    // are issued together (the stores could alias them for the compiler)
    if (mode == UPD_STAGE1) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        Wh[c] = Snh[(long)c * P + c0];
        Wl[c] = Snl[(long)c * P + c0];
      }
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        Gh[f] = a.grad_base ? Snh[(long)(4 + f) * P + c0] : (f < 4 ? o.gbx[f] : o.gby[f - 4]);
        Gl[f] = a.grad_base ? Snl[(long)(4 + f) * P + c0] : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float wh = Wh[c], wl = Wl[c];
        ff_add(Wh[c], Wl[c], 0.5f * dtr * o.L[c] + 0.125f * dtr * dtr * o.Lt[c]);
        float ah = wh, al = wl;
        ff_add(ah, al, dtr * o.L[c] + dtr * dtr * (1.0f / 6.0f) * o.Lt[c]);
        Ah[(long)c * P + c0] = ah;
        Al[(long)c * P + c0] = al;
      }
      // the gradient base: re-evaluated gradients are FP32 values (low part 0,
      // not stored); a base taken from the state keeps its low part
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        Bh[(long)f * P + c0] = Gh[f];
        if (a.grad_base) Bl[(long)f * P + c0] = Gl[f];
        ff_add(Gh[f], Gl[f], 0.5f * dtr * (f < 4 ? o.gtx[f] : o.gty[f - 4]));
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        Wh[c] = Ah[(long)c * P + c0];
        Wl[c] = Al[(long)c * P + c0];
      }
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        Gh[f] = Bh[(long)f * P + c0];
        Gl[f] = a.grad_base ? Bl[(long)f * P + c0] : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) ff_add(Wh[c], Wl[c], dtr * dtr * (1.0f / 3.0f) * o.Lt[c]);
#pragma unroll
      for (int f = 0; f < 8; ++f) ff_add(Gh[f], Gl[f], dtr * (f < 4 ? o.gtx[f] : o.gty[f - 4]));
    }
    if (xwall || ywall) {
      float ke = 0.5f * (Wh[1] * Wh[1] + Wh[2] * Wh[2]) / Wh[0];
      Wh[1] = Wl[1] = Wh[2] = Wl[2] = 0.0f;
      ff_add(Wh[3], Wl[3], -ke);
    }
    if (xwall) { Gh[5] = Gl[5] = Gh[6] = Gl[6] = 0.0f; }   // y-gradients of rho U, rho V
    if (ywall) { Gh[1] = Gl[1] = Gh[2] = Gl[2] = 0.0f; }   // x-gradients of rho U, rho V
    float* Oh = a.Out_hi + (long)g * NFLD * P;
#pragma unroll
    for (int c = 0; c < 4; ++c) Oh[(long)c * P + c0] = Wh[c];
#pragma unroll
    for (int f = 0; f < 8; ++f) Oh[(long)(4 + f) * P + c0] = Gh[f];
    if (a.Out_lo) {
      float* Ol = a.Out_lo + (long)g * NFLD * P;
#pragma unroll
      for (int c = 0; c < 4; ++c) Ol[(long)c * P + c0] = Wl[c];
#pragma unroll
      for (int f = 0; f < 8; ++f) Ol[(long)(4 + f) * P + c0] = Gl[f];
    }
    float pr = Wh[3] - 0.5f * (Wh[1] * Wh[1] + Wh[2] * Wh[2]) / Wh[0];
    if (!(Wh[0] > 0.0f) || !(pr > 0.0f)) atomicOr(a.flag, 1);
  } else {
    // FP64 path
    const double dt = a.dt;
    const double* Sng = a.Sn + (long)g * NFLD * P;
    double* Og = a.Sout + (long)g * NFLD * P;
    double* Ag = a.Wacc + (long)g * 4 * P;
    double* Bg = a.gB + (long)g * 8 * P;
    double Wnew[4], Gnew[8];
    // inputs first, then the stores (see the mixed branch)
    if (mode == UPD_STAGE1) {
      double Wn[4], Gb[8];
#pragma unroll
      for (int c = 0; c < 4; ++c) Wn[c] = Sng[(long)c * P + c0];
#pragma unroll
      for (int f = 0; f < 8; ++f)
        Gb[f] = a.grad_base ? Sng[(long)(4 + f) * P + c0] : (double)(f < 4 ? o.gbx[f] : o.gby[f - 4]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double dL = (double)o.L[c], dLt = (double)o.Lt[c];
        Wnew[c] = Wn[c] + 0.5 * dt * dL + 0.125 * dt * dt * dLt;
        Ag[(long)c * P + c0] = Wn[c] + dt * dL + dt * dt / 6.0 * dLt;
      }
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        Bg[(long)f * P + c0] = Gb[f];
        Gnew[f] = Gb[f] + 0.5 * dt * (double)(f < 4 ? o.gtx[f] : o.gty[f - 4]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) Wnew[c] = Ag[(long)c * P + c0];
#pragma unroll
      for (int f = 0; f < 8; ++f) Gnew[f] = Bg[(long)f * P + c0];
#pragma unroll
      for (int c = 0; c < 4; ++c) Wnew[c] = Wnew[c] + dt * dt / 3.0 * (double)o.Lt[c];
#pragma unroll
      for (int f = 0; f < 8; ++f) Gnew[f] = Gnew[f] + dt * (double)(f < 4 ? o.gtx[f] : o.gty[f - 4]);
    }
    if (xwall || ywall) {
      double ke = 0.5 * (Wnew[1] * Wnew[1] + Wnew[2] * Wnew[2]) / Wnew[0];
      Wnew[1] = 0.0;
      Wnew[2] = 0.0;
      Wnew[3] -= ke;
    }
    if (xwall) { Gnew[5] = 0.0; Gnew[6] = 0.0; }   // y-gradients of rho U, rho V
    if (ywall) { Gnew[1] = 0.0; Gnew[2] = 0.0; }   // x-gradients of rho U, rho V
#pragma unroll
    for (int c = 0; c < 4; ++c) Og[(long)c * P + c0] = Wnew[c];
#pragma unroll
    for (int f = 0; f < 8; ++f) Og[(long)(4 + f) * P + c0] = Gnew[f];
    // positivity of density and pressure (no trap: a flag the host reads)
    double p = Wnew[3] - 0.5 * (Wnew[1] * Wnew[1] + Wnew[2] * Wnew[2]) / Wnew[0];
    if (!(Wnew[0] > 0.0) || !(p > 0.0)) atomicOr(a.flag, 1);
  }
}

template <class R>
__global__ void __launch_bounds__(128, PointTune<R>::update_minb) update_kernel(KArgs<R> a, int mode) {
  update_body(a, mode, blockIdx.z, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
inline dim3 grid2(int nxp, int nyp, dim3 b, int z) {
  return dim3((unsigned)((nxp + b.x - 1) / b.x), (unsigned)((nyp + b.y - 1) / b.y), (unsigned)z);
}

template <class R>
cudaError_t launch_nodal(const KArgs<R>& a, cudaStream_t s) {
  dim3 b(32, 4);
  int mx = (a.L.nx > a.L.nxd ? a.L.nx : a.L.nxd) + 2, my = (a.L.ny > a.L.nyd ? a.L.ny : a.L.nyd) + 2;
  nodal_kernel<R><<<grid2(mx, my, b, 2), b, 0, s>>>(a);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_points(const KArgs<R>& a, cudaStream_t s) {
  dim3 b(32, 4);
  if constexpr (PointTune<R>::pair) {
    const dim3 bp(16, 4);   // points per block; the block itself is (32, 4) threads
    const dim3 gA = grid2(a.L.nx + 3, a.L.nyd + 3, bp, 1), gB = grid2(a.L.nxd + 3, a.L.ny + 3, bp, 1);
    if (a.recon_vars) point_pair_kernel<R, 0, true><<<gA, b, 0, s>>>(a);
    else point_pair_kernel<R, 0, false><<<gA, b, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.recon_vars) point_pair_kernel<R, 1, true><<<gB, b, 0, s>>>(a);
    else point_pair_kernel<R, 1, false><<<gB, b, 0, s>>>(a);
    return cudaGetLastError();
  }
  const dim3 gA = grid2(a.L.nx + 3, a.L.nyd + 3, b, 1), gB = grid2(a.L.nxd + 3, a.L.ny + 3, b, 1);
  if (a.recon_vars) point_kernel<R, 0, true><<<gA, b, 0, s>>>(a);
  else point_kernel<R, 0, false><<<gA, b, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.recon_vars) point_kernel<R, 1, true><<<gB, b, 0, s>>>(a);
  else point_kernel<R, 1, false><<<gB, b, 0, s>>>(a);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_update(const KArgs<R>& a, int mode, cudaStream_t s) {
  dim3 b(32, 4);
  int mx = a.L.nx > a.L.nxd ? a.L.nx : a.L.nxd, my = a.L.ny > a.L.nyd ? a.L.ny : a.L.nyd;
  update_kernel<R><<<grid2(mx, my, b, 2), b, 0, s>>>(a, mode);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// component batches
// ---------------------------------------------------------------------------
template <class R>
__global__ void iface_batch_kernel(GasK<R> gas, int normal, int n, const double* in, double* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  R v[20];
  for (int k = 0; k < 20; ++k) v[k] = (R)in[(long)t * 20 + k];
  IfaceOut<R> o;
  iface_solve(gas, normal, v, v + 4, v + 8, v + 12, v + 16, true, o);
  double* q = out + (long)t * 24;
  for (int k = 0; k < 4; ++k) {
    q[k] = o.F[k]; q[4 + k] = o.Ft[k]; q[8 + k] = o.Wl[k];
    q[12 + k] = o.Wr[k]; q[16 + k] = o.Wlt[k]; q[20 + k] = o.Wrt[k];
  }
}

template <class R>
__global__ void nodal_batch_kernel(GasK<R> gas, int n, const double* in, double* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  R v[12];
  for (int k = 0; k < 12; ++k) v[k] = (R)in[(long)t * 12 + k];
  R F[4], G[4], Ft[4], Gt[4];
  nodal_flux(gas, v, v + 4, v + 8, F, G, Ft, Gt);
  double* q = out + (long)t * 16;
  for (int k = 0; k < 4; ++k) { q[k] = F[k]; q[4 + k] = G[k]; q[8 + k] = Ft[k]; q[12 + k] = Gt[k]; }
}

template <class R>
__global__ void recon_batch_kernel(GenoK<R> g, int kind, R h, R ih, int n, const double* in, double* out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  if (kind == 0) {
    R Q[4], Qx[4];
    for (int k = 0; k < 4; ++k) { Q[k] = (R)in[(long)t * 8 + k]; Qx[k] = (R)in[(long)t * 8 + 4 + k]; }
    R vl, dl, cl, vr, dr, cr;
    recon_interface(g, Q, Qx, h, ih, vl, dl, cl, vr, dr, cr);
    double* q = out + (long)t * 6;
    q[0] = vl; q[1] = dl; q[2] = cl; q[3] = vr; q[4] = dr; q[5] = cr;
  } else {
    R Q[3], Qx[3];
    for (int k = 0; k < 3; ++k) { Q[k] = (R)in[(long)t * 6 + k]; Qx[k] = (R)in[(long)t * 6 + 3 + k]; }
    out[(long)t * 6] = recon_node(g, Q, Qx, h, ih);
    for (int k = 1; k < 6; ++k) out[(long)t * 6 + k] = 0.0;
  }
}

template <class R>
cudaError_t launch_iface_batch(const GasK<R>& gas, int normal, int n, const double* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  iface_batch_kernel<R><<<(n + 63) / 64, 64, 0, s>>>(gas, normal, n, in, out);
  return cudaGetLastError();
}
template <class R>
cudaError_t launch_nodal_batch(const GasK<R>& gas, int n, const double* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  nodal_batch_kernel<R><<<(n + 63) / 64, 64, 0, s>>>(gas, n, in, out);
  return cudaGetLastError();
}
template <class R>
cudaError_t launch_recon_batch(const GenoK<R>& g, int kind, double h, int n, const double* in, double* out,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  recon_batch_kernel<R><<<(n + 127) / 128, 128, 0, s>>>(g, kind, (R)h, (R)(1.0 / h), n, in, out);
  return cudaGetLastError();
}

#define FDK_INSTANTIATE(R)                                                                                  \
  template cudaError_t launch_nodal<R>(const KArgs<R>&, cudaStream_t);                                     \
  template cudaError_t launch_points<R>(const KArgs<R>&, cudaStream_t);                                    \
  template cudaError_t launch_update<R>(const KArgs<R>&, int, cudaStream_t);                               \
  template cudaError_t launch_iface_batch<R>(const GasK<R>&, int, int, const double*, double*, cudaStream_t); \
  template cudaError_t launch_nodal_batch<R>(const GasK<R>&, int, const double*, double*, cudaStream_t);   \
  template cudaError_t launch_recon_batch<R>(const GenoK<R>&, int, double, int, const double*, double*,     \
                                             cudaStream_t);

}  // namespace fdk
