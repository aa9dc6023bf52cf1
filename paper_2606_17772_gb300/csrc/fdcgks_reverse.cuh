// Hand-written reverse mode (adjoints) of the FP64 point and node arithmetic
// of fdcgks_math.cuh: the GENO interface and node reconstructions (Sec. 3.1,
// Sec. 3.2, App. C), the kinetic interface solve (App. A1-A2, Eq. eq:W-model)
// and the nodal flux (Sec. 2.1).
//
// Each *_adj function recomputes its forward values, then runs the forward
// statements backwards, adding to the adjoints of its inputs the transposed
// partial derivatives times the adjoints of its outputs.  Readings of the
// non-smooth points: the branch the forward took (GENO saturation, chi == 1, the positivity safeguard); at an
// exact tie of min/max the mean of the two one-sided derivatives (what a
// central difference sees), and at |x| = 0 derivative 0; a vanishing
// derivative factor times an infinite one (the time coefficients at tau = 0)
// counts as 0.  __host__ __device__ so that the CPU test suite checks it
// against forward-mode dual numbers on the same arithmetic without a GPU.
#pragma once

#include "fdcgks_math.cuh"

namespace fdk {
namespace rev {

typedef double R;

// sign of x, 0 at x = 0 (the derivative of |x| there, as for the dual numbers)
FD_HD R sgn0(R x) { return x > 0.0 ? 1.0 : x < 0.0 ? -1.0 : 0.0; }

// y = max(a, b) / min(a, b) with the dual numbers' tie rule
FD_HD void max_adj(R a, R b, R yb, R& ab, R& bb) {
  if (b > a) bb += yb;
  else if (a > b) ab += yb;
  else { ab += 0.5 * yb; bb += 0.5 * yb; }
}
FD_HD void min_adj(R a, R b, R yb, R& ab, R& bb) {
  if (b < a) bb += yb;
  else if (a < b) ab += yb;
  else { ab += 0.5 * yb; bb += 0.5 * yb; }
}

// ---------------------------------------------------------------------------
// GENO (Sec. 3.2)
// ---------------------------------------------------------------------------
// adjoint of geno_chi (FP64 product form) with the floor fl added to eps_a:
// chib -> ISb[3], flb
FD_HD void geno_chi_adj(const GenoK<R>& g, const R IS[3], R fl, R chib, R ISb[3], R& flb) {
  if (g.linear || chib == 0.0) return;
  const R m_lo = s_min(IS[1], IS[2]), ISL = s_min(IS[0], m_lo);
  const R m_hi = s_max(IS[1], IS[2]), ISH = s_max(IS[0], m_hi);
  const R D = 0.5 * (IS[1] + IS[2]) - IS[0];
  const R tau = s_abs(D);
  R ea = g.eps_a;
  if (fl != 0.0) ea = ea + fl;
  const R H = ISH + ea, Lo = ISL + ea;
  const R hr = rpow(H, g.r), lr = rpow(Lo, g.r), tr = rpow(tau, g.r);
  const R A = (hr + tr) * lr, B = (lr + tr) * hr;
  const R num = 2.0 * A, den = A + B;
  if (g.C * num > R(TanhSat<R>::z) * den) return;   // saturated: chi constant
  const R alpha = num / den, z = g.C * alpha;
  if (z > R(TanhSat<R>::z)) return;
  const R th = s_tanh(z);
  const R alphab = chib * g.inv_tanhC * (1.0 - th * th) * g.C;
  // alpha = 2 A / (A + B)
  const R Ab = alphab * 2.0 * B / (den * den), Bb = -alphab * 2.0 * A / (den * den);
  const R hrb = Ab * lr + Bb * (lr + tr), lrb = Ab * (hr + tr) + Bb * hr, trb = (Ab * lr + Bb * hr);
  const R dpow = g.r == 3 ? 3.0 : 2.0;
  const R Hb = hrb * dpow * (g.r == 3 ? H * H : H), Lob = lrb * dpow * (g.r == 3 ? Lo * Lo : Lo);
  const R taub = trb * dpow * (g.r == 3 ? tau * tau : tau);
  const R Db = taub * sgn0(D);
  if (fl != 0.0) flb += Hb + Lob;
  ISb[0] -= Db;
  ISb[1] += 0.5 * Db;
  ISb[2] += 0.5 * Db;
  R mb = 0.0;
  max_adj(IS[0], m_hi, Hb, ISb[0], mb);
  max_adj(IS[1], IS[2], mb, ISb[1], ISb[2]);
  mb = 0.0;
  min_adj(IS[0], m_lo, Lob, ISb[0], mb);
  min_adj(IS[1], IS[2], mb, ISb[1], ISb[2]);
}

// adjoint of geno_weights (FP64 product form): wb[3] -> ISb[3]
FD_HD void geno_weights_adj(const GenoK<R>& g, const R d[3], const R IS[3], const R wb[3], R ISb[3]) {
  const R e0 = IS[0] + g.eps_w, e1 = IS[1] + g.eps_w, e2 = IS[2] + g.eps_w;
  const R s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
  const R t0 = d[0] * s1 * s2, t1 = d[1] * s0 * s2, t2 = d[2] * s0 * s1;
  const R S = t0 + t1 + t2, inv = 1.0 / S;
  const R w0 = t0 * inv, w1 = t1 * inv, w2 = t2 * inv;
  const R dot = wb[0] * w0 + wb[1] * w1 + wb[2] * w2;
  const R t0b = (wb[0] - dot) * inv, t1b = (wb[1] - dot) * inv, t2b = (wb[2] - dot) * inv;
  const R s0b = d[1] * s2 * t1b + d[2] * s1 * t2b;
  const R s1b = d[0] * s2 * t0b + d[2] * s0 * t2b;
  const R s2b = d[0] * s1 * t0b + d[1] * s0 * t1b;
  ISb[0] += 2.0 * e0 * s0b;
  ISb[1] += 2.0 * e1 * s1b;
  ISb[2] += 2.0 * e2 * s2b;
}

// The GENO blend of one side: value v = chi PH + (1 - chi) PL, derivative
// d = chi PHx + (1 - chi) PLx, PL = sum w_k q_k, PLx = w0 qx0 + (w1 + w2) dq12.
// Given vb, db and the adjoint of chi, returns the adjoints of PH, PHx, q[3],
// qx0, dq12, IS[3] and the floor fl of the path function.
FD_HD void geno_blend_adj(const GenoK<R>& g, const R dk[3], const R IS[3], R fl, R PH, R PHx, const R q[3], R qx0,
                          R dq12, R vb, R db, R chib, R& PHb, R& PHxb, R qb[3], R& qx0b, R& dq12b, R ISb[3],
                          R& flb) {
  const R chi = geno_chi(g, IS[0], IS[1], IS[2], fl);
  if (chi == 1.0) {
    // the forward skips the blend; chi's derivative is zero there
    PHb += vb;
    PHxb += db;
    return;
  }
  R w[3];
  geno_weights(g, dk, IS[0], IS[1], IS[2], w);
  const R PL = w[0] * q[0] + w[1] * q[1] + w[2] * q[2];
  const R PLx = w[0] * qx0 + (w[1] + w[2]) * dq12;
  const R chib_t = chib + vb * (PH - PL) + db * (PHx - PLx);
  PHb += chi * vb;
  PHxb += chi * db;
  const R PLb = (1.0 - chi) * vb, PLxb = (1.0 - chi) * db;
  R wb[3];
  wb[0] = PLb * q[0] + PLxb * qx0;
  wb[1] = PLb * q[1] + PLxb * dq12;
  wb[2] = PLb * q[2] + PLxb * dq12;
  qb[0] += PLb * w[0];
  qb[1] += PLb * w[1];
  qb[2] += PLb * w[2];
  qx0b += PLxb * w[0];
  dq12b += PLxb * (w[1] + w[2]);
  geno_weights_adj(g, dk, IS, wb, ISb);
  geno_chi_adj(g, IS, fl, chib_t, ISb, flb);
}

// floor of the path function from max |Q| (geno_floor_of with fscale): its
// adjoint flb goes to the entry of largest magnitude (ties: shared, as for
// the dual numbers' nested max)
FD_HD void floor_adj4(const R Q[4], R fscale, R flb, R Qb[4]) {
  if (flb == 0.0 || fscale == 0.0) return;
  const R a0 = s_abs(Q[0]), a1 = s_abs(Q[1]), a2 = s_abs(Q[2]), a3 = s_abs(Q[3]);
  const R m01 = s_max(a0, a1), m23 = s_max(a2, a3), qmax = s_max(m01, m23);
  const R qb = flb * 2.0 * fscale * fscale * qmax;
  R m01b = 0.0, m23b = 0.0, ab[4] = {0.0, 0.0, 0.0, 0.0};
  max_adj(m01, m23, qb, m01b, m23b);
  max_adj(a0, a1, m01b, ab[0], ab[1]);
  max_adj(a2, a3, m23b, ab[2], ab[3]);
  for (int k = 0; k < 4; ++k) Qb[k] += ab[k] * sgn0(Q[k]);
}
FD_HD void floor_adj3(const R Q[3], R fscale, R flb, R Qb[3]) {
  if (flb == 0.0 || fscale == 0.0) return;
  // qmax = max(|Q1|, max(|Q0|, |Q2|)) as in recon_node
  const R a0 = s_abs(Q[0]), a1 = s_abs(Q[1]), a2 = s_abs(Q[2]);
  const R m02 = s_max(a0, a2), qmax = s_max(a1, m02);
  const R qb = flb * 2.0 * fscale * fscale * qmax;
  R m02b = 0.0, ab[3] = {0.0, 0.0, 0.0};
  max_adj(a1, m02, qb, ab[1], m02b);
  max_adj(a0, a2, m02b, ab[0], ab[2]);
  for (int k = 0; k < 3; ++k) Qb[k] += ab[k] * sgn0(Q[k]);
}

// 13/3 t^2 + u^2 with t = a - b - x h, u = 2 (a - b) - x h (the sub-stencil
// with an averaged gradient, App. C): adds to ab, bb, xb
FD_HD void is_grad_adj(R a, R b, R x, R h, R ISb, R& ab, R& bb, R& xb) {
  const R t = a - b - x * h, u = 2.0 * (a - b) - x * h;
  const R tb = (26.0 / 3.0) * t * ISb, ub = 2.0 * u * ISb;
  ab += tb + 2.0 * ub;
  bb -= tb + 2.0 * ub;
  xb -= h * (tb + ub);
}
// 13/12 t^2 + u^2 / 4 for given t and u: returns (tb, ub)
FD_HD void is_three_adj(R t, R u, R ISb, R& tb, R& ub) {
  tb = (13.0 / 6.0) * t * ISb;
  ub = 0.5 * u * ISb;
}

// adjoint of recon_interface (FP64, path-function floor from fscale as in
// geno_floor_of): output adjoints vlb, dlb, chilb, vrb, drb, chirb -> Qb[4],
// Qxb[4] (added)
FD_HD void recon_interface_adj(const GenoK<R>& g, const R Q[4], const R Qx[4], R h, R ih, R vlb, R dlb, R chilb,
                               R vrb, R drb, R chirb, R Qb[4], R Qxb[4], R fscale = 0.0) {
  const R c64 = 1.0 / 64.0, c30 = 1.0 / 30.0;
  const R fl = geno_floor_of(s_max(s_max(s_abs(Q[0]), s_abs(Q[1])), s_max(s_abs(Q[2]), s_abs(Q[3]))), fscale);
  R flb = 0.0;
  const R PHx = -((Q[0] + 45.0 * Q[1] - 45.0 * Q[2] - Q[3]) * ih + 9.0 * (Qx[1] + Qx[2])) * c30;
  const R dq12 = (Q[2] - Q[1]) * ih;
  R PHxb = 0.0, dq12b = 0.0;
  // ---- left (App. C1) ----
  {
    const R PH = ((7.0 * Q[0] + 35.0 * Q[1] + 21.0 * Q[2] + Q[3]) + (Qx[0] + 22.0 * Qx[1] - 7.0 * Qx[2]) * h) * c64;
    const R q[3] = {(-5.0 * Q[0] + 9.0 * Q[1] - 3.0 * Qx[0] * h) * 0.25, (-Q[0] + 6.0 * Q[1] + 3.0 * Q[2]) * 0.125,
                    (3.0 * Q[1] + 6.0 * Q[2] - Q[3]) * 0.125};
    const R qx0 = (-3.0 * Q[0] + 3.0 * Q[1]) * ih - 2.0 * Qx[0];
    R t = Q[1] - Q[0] - Qx[0] * h, u = 2.0 * (Q[1] - Q[0]) - Qx[0] * h;
    R IS[3];
    IS[0] = (13.0 / 3.0) * t * t + u * u;
    const R t1 = Q[0] - 2.0 * Q[1] + Q[2], u1 = Q[2] - Q[0];
    IS[1] = (13.0 / 12.0) * t1 * t1 + 0.25 * u1 * u1;
    const R t2 = Q[1] - 2.0 * Q[2] + Q[3], u2 = 3.0 * Q[1] - 4.0 * Q[2] + Q[3];
    IS[2] = (13.0 / 12.0) * t2 * t2 + 0.25 * u2 * u2;
    R PHb = 0.0, qb[3] = {0.0, 0.0, 0.0}, qx0b = 0.0, ISb[3] = {0.0, 0.0, 0.0};
    geno_blend_adj(g, g.d_iface, IS, fl, PH, PHx, q, qx0, dq12, vlb, dlb, chilb, PHb, PHxb, qb, qx0b, dq12b, ISb,
                   flb);
    // PH
    Qb[0] += 7.0 * c64 * PHb; Qb[1] += 35.0 * c64 * PHb; Qb[2] += 21.0 * c64 * PHb; Qb[3] += c64 * PHb;
    Qxb[0] += h * c64 * PHb; Qxb[1] += 22.0 * h * c64 * PHb; Qxb[2] -= 7.0 * h * c64 * PHb;
    // q0..q2, qx0
    Qb[0] += -1.25 * qb[0] - 0.125 * qb[1] - 3.0 * ih * qx0b;
    Qb[1] += 2.25 * qb[0] + 0.75 * qb[1] + 0.375 * qb[2] + 3.0 * ih * qx0b;
    Qb[2] += 0.375 * qb[1] + 0.75 * qb[2];
    Qb[3] -= 0.125 * qb[2];
    Qxb[0] += -0.75 * h * qb[0] - 2.0 * qx0b;
    // IS
    is_grad_adj(Q[1], Q[0], Qx[0], h, ISb[0], Qb[1], Qb[0], Qxb[0]);
    R tb, ub;
    is_three_adj(t1, u1, ISb[1], tb, ub);
    Qb[0] += tb - ub; Qb[1] -= 2.0 * tb; Qb[2] += tb + ub;
    is_three_adj(t2, u2, ISb[2], tb, ub);
    Qb[1] += tb + 3.0 * ub; Qb[2] -= 2.0 * tb + 4.0 * ub; Qb[3] += tb + ub;
  }
  // ---- right (App. C2, formulas for interface j+1/2) ----
  {
    const R PH = ((Q[0] + 21.0 * Q[1] + 35.0 * Q[2] + 7.0 * Q[3]) + (7.0 * Qx[1] - 22.0 * Qx[2] - Qx[3]) * h) * c64;
    const R q[3] = {(-5.0 * Q[3] + 9.0 * Q[2] + 3.0 * Qx[3] * h) * 0.25, (-Q[3] + 6.0 * Q[2] + 3.0 * Q[1]) * 0.125,
                    (-Q[0] + 6.0 * Q[1] + 3.0 * Q[2]) * 0.125};
    const R qx0 = (-3.0 * Q[2] + 3.0 * Q[3]) * ih - 2.0 * Qx[3];
    R IS[3];
    const R t0 = Q[2] - Q[3] + Qx[3] * h, u0 = 2.0 * (Q[3] - Q[2]) - Qx[3] * h;
    IS[0] = (13.0 / 3.0) * t0 * t0 + u0 * u0;
    const R t1 = Q[1] - 2.0 * Q[2] + Q[3], u1 = Q[3] - Q[1];
    IS[1] = (13.0 / 12.0) * t1 * t1 + 0.25 * u1 * u1;
    const R t2 = Q[0] - 2.0 * Q[1] + Q[2], u2 = 3.0 * Q[2] - 4.0 * Q[1] + Q[0];
    IS[2] = (13.0 / 12.0) * t2 * t2 + 0.25 * u2 * u2;
    R PHb = 0.0, qb[3] = {0.0, 0.0, 0.0}, qx0b = 0.0, ISb[3] = {0.0, 0.0, 0.0};
    geno_blend_adj(g, g.d_iface, IS, fl, PH, PHx, q, qx0, dq12, vrb, drb, chirb, PHb, PHxb, qb, qx0b, dq12b, ISb,
                   flb);
    Qb[0] += c64 * PHb; Qb[1] += 21.0 * c64 * PHb; Qb[2] += 35.0 * c64 * PHb; Qb[3] += 7.0 * c64 * PHb;
    Qxb[1] += 7.0 * h * c64 * PHb; Qxb[2] -= 22.0 * h * c64 * PHb; Qxb[3] -= h * c64 * PHb;
    Qb[3] += -1.25 * qb[0] - 0.125 * qb[1] + 3.0 * ih * qx0b;
    Qb[2] += 2.25 * qb[0] + 0.75 * qb[1] + 0.375 * qb[2] - 3.0 * ih * qx0b;
    Qb[1] += 0.375 * qb[1] + 0.75 * qb[2];
    Qb[0] -= 0.125 * qb[2];
    Qxb[3] += 0.75 * h * qb[0] - 2.0 * qx0b;
    // IS0: t = Q2 - Q3 + Qx3 h = (Q2) - (Q3) - (-Qx3) h, u = 2 (Q3 - Q2) - Qx3 h
    {
      const R tb0 = (26.0 / 3.0) * t0 * ISb[0], ub0 = 2.0 * u0 * ISb[0];
      Qb[2] += tb0 - 2.0 * ub0;
      Qb[3] += -tb0 + 2.0 * ub0;
      Qxb[3] += h * tb0 - h * ub0;
    }
    R tb, ub;
    is_three_adj(t1, u1, ISb[1], tb, ub);
    Qb[1] += tb - ub; Qb[2] -= 2.0 * tb; Qb[3] += tb + ub;
    is_three_adj(t2, u2, ISb[2], tb, ub);
    Qb[0] += tb + ub; Qb[1] -= 2.0 * tb + 4.0 * ub; Qb[2] += tb + 3.0 * ub;
  }
  // shared PHx and dq12
  Qb[0] -= c30 * ih * PHxb; Qb[1] -= 45.0 * c30 * ih * PHxb; Qb[2] += 45.0 * c30 * ih * PHxb; Qb[3] += c30 * ih * PHxb;
  Qxb[1] -= 9.0 * c30 * PHxb; Qxb[2] -= 9.0 * c30 * PHxb;
  Qb[2] += ih * dq12b;
  Qb[1] -= ih * dq12b;
  floor_adj4(Q, fscale, flb, Qb);
}

// adjoint of recon_node (FP64, floor from fscale): rb -> Qb[3], Qxb[3] (added)
FD_HD void recon_node_adj(const GenoK<R>& g, const R Q[3], const R Qx[3], R h, R ih, R rb, R Qb[3], R Qxb[3],
                          R fscale = 0.0) {
  const R c30 = 1.0 / 30.0;
  const R PHx = (9.0 * (Q[0] - Q[2]) * ih + (Qx[0] + 46.0 * Qx[1] + Qx[2])) * c30;
  const R qx[3] = {(Q[2] - Q[0]) * 0.5 * ih, 2.0 * (Q[1] - Q[0]) * ih - Qx[0], 2.0 * (Q[2] - Q[1]) * ih - Qx[2]};
  const R t0 = Q[0] - 2.0 * Q[1] + Q[2], u0 = Q[2] - Q[0];
  R IS[3];
  IS[0] = (13.0 / 12.0) * t0 * t0 + 0.25 * u0 * u0;
  R t = Q[1] - Q[0] - Qx[0] * h, u = 2.0 * (Q[1] - Q[0]) - Qx[0] * h;
  IS[1] = (13.0 / 3.0) * t * t + u * u;
  t = Q[2] - Q[1] - Qx[2] * h;
  u = 2.0 * (Q[2] - Q[1]) - Qx[2] * h;
  IS[2] = (13.0 / 3.0) * t * t + u * u;
  R PHxb = 0.0, qxb[3] = {0.0, 0.0, 0.0}, ISb[3] = {0.0, 0.0, 0.0}, flb = 0.0;
  const R fl = geno_floor_of(s_max(s_abs(Q[1]), s_max(s_abs(Q[0]), s_abs(Q[2]))), fscale);
  const R chi = geno_chi(g, IS[0], IS[1], IS[2], fl);
  if (chi == 1.0) {
    PHxb = rb;
  } else {
    R w[3];
    geno_weights(g, g.d_node, IS[0], IS[1], IS[2], w);
    const R PLx = w[0] * qx[0] + w[1] * qx[1] + w[2] * qx[2];
    PHxb = chi * rb;
    const R PLxb = (1.0 - chi) * rb;
    const R wb[3] = {PLxb * qx[0], PLxb * qx[1], PLxb * qx[2]};
    for (int k = 0; k < 3; ++k) qxb[k] = PLxb * w[k];
    geno_weights_adj(g, g.d_node, IS, wb, ISb);
    geno_chi_adj(g, IS, fl, rb * (PHx - PLx), ISb, flb);
  }
  floor_adj3(Q, fscale, flb, Qb);
  Qb[0] += 9.0 * c30 * ih * PHxb;
  Qb[2] -= 9.0 * c30 * ih * PHxb;
  Qxb[0] += c30 * PHxb; Qxb[1] += 46.0 * c30 * PHxb; Qxb[2] += c30 * PHxb;
  Qb[2] += 0.5 * ih * qxb[0]; Qb[0] -= 0.5 * ih * qxb[0];
  Qb[1] += 2.0 * ih * qxb[1]; Qb[0] -= 2.0 * ih * qxb[1]; Qxb[0] -= qxb[1];
  Qb[2] += 2.0 * ih * qxb[2]; Qb[1] -= 2.0 * ih * qxb[2]; Qxb[2] -= qxb[2];
  R tb, ub;
  is_three_adj(t0, u0, ISb[0], tb, ub);
  Qb[0] += tb - ub; Qb[1] -= 2.0 * tb; Qb[2] += tb + ub;
  is_grad_adj(Q[1], Q[0], Qx[0], h, ISb[1], Qb[1], Qb[0], Qxb[0]);
  is_grad_adj(Q[2], Q[1], Qx[2], h, ISb[2], Qb[2], Qb[1], Qxb[2]);
}

// Adjoint of the reconstruction of one 4-point line in conservative
// components with the positivity safeguard (recon_line_ld): x[e * 8 + f] the
// line's inputs (entry e, field f: 0-3 W, 4-7 the averaged gradient along the
// line); vb[0..3][c] the adjoints of the left value, left derivative, right
// value and right derivative of component c; chib that of the line's chi
// (the smaller of the two sides' chi of rho, 0 where the safeguard acts).
// Adds to xb[32].  radj(Q, Qx, vlb, dlb, chilb, vrb, drb, chirb, Qb, Qxb)
// runs recon_interface_adj for one component (an out-of-line copy on the GPU)
// with the same fscale (the path-function floor, geno_floor_of).
// The forward of that line (recon_line_ld's arithmetic, with the floor):
// v[0..3][c] = left value, left derivative, right value, right derivative;
// chi of the flux; cl0, cr0 the two sides' chi of rho; fixl / fixr whether
// the safeguard replaced a side.
FD_HD void recon_line_fwd(const GenoK<R>& g, const R* x, R h, R ih, R fscale, R v[4][4], R& chi, R& cl0, R& cr0,
                          bool& fixl, bool& fixr) {
  for (int c = 0; c < 4; ++c) {
    const R Q[4] = {x[c], x[8 + c], x[16 + c], x[24 + c]};
    const R Qx[4] = {x[4 + c], x[12 + c], x[20 + c], x[28 + c]};
    R cl, cr;
    recon_interface(g, Q, Qx, h, ih, v[0][c], v[1][c], cl, v[2][c], v[3][c], cr, fscale);
    if (c == 0) { cl0 = cl; cr0 = cr; }
  }
  chi = s_min(cl0, cr0);
  fixl = !physical_state(v[0]);
  fixr = !physical_state(v[2]);
  for (int c = 0; c < 4; ++c) {
    if (fixl) { v[0][c] = x[8 + c]; v[1][c] = 0.0; }
    if (fixr) { v[2][c] = x[16 + c]; v[3][c] = 0.0; }
  }
  if (fixl || fixr) chi = 0.0;
}

template <class RADJ>
FD_HD void recon_line_adj(const GenoK<R>& g, const R* x, R h, R ih, const R vb[4][4], R chib, R* xb, RADJ radj,
                          R fscale = 0.0) {
  R v[4][4], chi, cl0, cr0;
  bool fixl, fixr;
  recon_line_fwd(g, x, h, ih, fscale, v, chi, cl0, cr0, fixl, fixr);
  R chilb = 0.0, chirb = 0.0;
  if (!fixl && !fixr) min_adj(cl0, cr0, chib, chilb, chirb);
  for (int c = 0; c < 4; ++c) {
    // a replaced side takes the value of its node (entry 1 left, 2 right) and a zero slope
    if (fixl) xb[8 + c] += vb[0][c];
    if (fixr) xb[16 + c] += vb[2][c];
    const R Q[4] = {x[c], x[8 + c], x[16 + c], x[24 + c]};
    const R Qx[4] = {x[4 + c], x[12 + c], x[20 + c], x[28 + c]};
    R Qb[4] = {0.0, 0.0, 0.0, 0.0}, Qxb[4] = {0.0, 0.0, 0.0, 0.0};
    radj(Q, Qx, fixl ? 0.0 : vb[0][c], fixl ? 0.0 : vb[1][c], c == 0 ? chilb : 0.0, fixr ? 0.0 : vb[2][c],
         fixr ? 0.0 : vb[3][c], c == 0 ? chirb : 0.0, Qb, Qxb);
    for (int e = 0; e < 4; ++e) {
      xb[e * 8 + c] += Qb[e];
      xb[e * 8 + 4 + c] += Qxb[e];
    }
  }
}

// ---------------------------------------------------------------------------
// Maxwellian moments (App. A1)
// ---------------------------------------------------------------------------
struct MaxwB {
  R rho, ir, U, V, p, i2l, lam;
};
FD_HD MaxwB maxw_zero() {
  MaxwB b;
  b.rho = b.ir = b.U = b.V = b.p = b.i2l = b.lam = 0.0;
  return b;
}

struct TabB {
  R u[NT], v[NT], xi[3];
};
FD_HD TabB tab_zero() {
  TabB b;
  for (int k = 0; k < NT; ++k) b.u[k] = b.v[k] = 0.0;
  b.xi[0] = b.xi[1] = b.xi[2] = 0.0;
  return b;
}

// W -> Maxwellian, given the adjoints gb of the Maxwellian's fields: Wb += ...
FD_HD void maxw_from_W_adj(const R W[4], R gm1, const Maxw<R>& g, MaxwB gb, R Wb[4]) {
  gb.i2l += -gb.lam * g.lam / g.i2l;                    // lam = 1/2 / i2l
  gb.p += gb.i2l * g.ir;                                // i2l = p ir
  gb.ir += gb.i2l * g.p;
  Wb[3] += gm1 * gb.p;                                  // p = gm1 (W3 - W0 (U^2 + V^2)/2)
  Wb[0] -= 0.5 * gm1 * (g.U * g.U + g.V * g.V) * gb.p;
  gb.U -= gm1 * W[0] * g.U * gb.p;
  gb.V -= gm1 * W[0] * g.V * gb.p;
  Wb[1] += gb.U * g.ir;                                 // U = W1 ir, V = W2 ir
  Wb[2] += gb.V * g.ir;
  gb.ir += gb.U * W[1] + gb.V * W[2];
  Wb[0] += gb.rho - gb.ir * g.ir * g.ir;                // rho = W0, ir = 1/W0
}

// t[n+2] = m t[n+1] + (n+1) i2l t[n], run backwards
FD_HD void recur_adj(R m, R i2l, const R* t, R* tb, R& mb, R& i2lb) {
  for (int n = NT - 3; n >= 0; --n) {
    const R b = tb[n + 2];
    tb[n + 1] += m * b;
    tb[n] += R(n + 1) * i2l * b;
    mb += t[n + 1] * b;
    i2lb += R(n + 1) * t[n] * b;
  }
}

FD_HD void tab_full_adj(const Maxw<R>& g, R K, const Tab<R>& T, TabB& Tb, MaxwB& gb) {
  recur_adj(g.U, g.i2l, T.u, Tb.u, gb.U, gb.i2l);
  recur_adj(g.V, g.i2l, T.v, Tb.v, gb.V, gb.i2l);
  gb.U += Tb.u[1];
  gb.V += Tb.v[1];
  gb.i2l += K * Tb.xi[1] + 2.0 * K * (K + 2.0) * g.i2l * Tb.xi[2];
}

FD_HD void tab_half_adj(const Maxw<R>& g, int sign, const Tab<R>& H, TabB& Hb, TabB& fullb, MaxwB& gb) {
  const R sl = s_sqrt(g.lam), isl = sl * (2.0 * g.i2l), e = s_exp(-g.lam * g.U * g.U);
  const R isqpi = 0.56418958354775628695;
  const R sg = R(sign);
  recur_adj(g.U, g.i2l, H.u, Hb.u, gb.U, gb.i2l);
  // H.u1 = U H.u0 + sign e isl / (2 sqrt(pi))
  const R b1 = Hb.u[1];
  gb.U += b1 * H.u[0];
  const R u0b = Hb.u[0] + b1 * g.U;
  const R eb = sg * 0.5 * isqpi * isl * b1;
  R islb = sg * 0.5 * e * isqpi * b1;
  // H.u0 = erfc(z)/2, z = -sign sl U, d erfc/dz = -2 e^{-z^2}/sqrt(pi), e^{-z^2} = e
  const R zb = -u0b * isqpi * e;
  R slb = -zb * sg * g.U;
  gb.U -= zb * sg * sl;
  // e = exp(-lam U^2)
  gb.lam -= eb * e * g.U * g.U;
  gb.U -= 2.0 * eb * e * g.lam * g.U;
  // isl = 2 sl i2l
  slb += islb * 2.0 * g.i2l;
  gb.i2l += islb * 2.0 * sl;
  gb.lam += slb * 0.5 / sl;   // sl = sqrt(lam)
  for (int n = 0; n < NT; ++n) fullb.v[n] += Hb.v[n];
  for (int n = 0; n < 3; ++n) fullb.xi[n] += Hb.xi[n];
}

template <int a, int b, int c>
FD_HD void mm_adj(const Tab<R>& T, R ob, TabB& Tb) {
  Tb.u[a] += ob * T.v[b] * T.xi[c];
  Tb.v[b] += ob * T.u[a] * T.xi[c];
  Tb.xi[c] += ob * T.u[a] * T.v[b];
}

template <int a, int b, int c>
FD_HD void mpsi_adj(const Tab<R>& T, const R ob[4], TabB& Tb) {
  mm_adj<a, b, c>(T, ob[0], Tb);
  mm_adj<a + 1, b, c>(T, ob[1], Tb);
  mm_adj<a, b + 1, c>(T, ob[2], Tb);
  mm_adj<a + 2, b, c>(T, 0.5 * ob[3], Tb);
  mm_adj<a, b + 2, c>(T, 0.5 * ob[3], Tb);
  mm_adj<a, b, c + 1>(T, 0.5 * ob[3], Tb);
}

// o = <s u^a v^b psi> (mslope, factored form): sb += ..., Tb += ...
// Forward, with h = s3/2, c0 = s0 + h xi[1]:
//   U(p) = c0 u[p] + s1 u[p+1] + h u[p+2],  V(q) = s2 v[q+1] + h v[q+2],
//   S(p,q) = v[q] U(p) + u[p] V(q),  U'(a) = s0 u[a] + s1 u[a+1] + h u[a+2],
//   Sx = xi[1] (v[b] U'(a) + u[a] V(b)) + h xi[2] u[a] v[b],
//   o = (S(a,b), S(a+1,b), S(a,b+1), (S(a+2,b) + S(a,b+2) + Sx)/2).
// Reverse: the weights of the S terms give the adjoints of U, V and the
// tables; those of U, U', V give the adjoints of the slope and the tables.
template <int a, int b>
FD_HD void mslope_adj(const Tab<R>& T, const R s[4], const R ob[4], TabB& Tb, R sb[4]) {
  const R h = 0.5 * s[3], x1 = T.xi[1], x2 = T.xi[2];
  const R c0 = s[0] + h * x1;
  R U[3], V[3];                                   // U(a + k), V(b + k)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U[k] = c0 * T.u[a + k] + s[1] * T.u[a + k + 1] + h * T.u[a + k + 2];
    V[k] = s[2] * T.v[b + k + 1] + h * T.v[b + k + 2];
  }
  const R Up = s[0] * T.u[a] + s[1] * T.u[a + 1] + h * T.u[a + 2];
  R Ub[3] = {0.0, 0.0, 0.0}, Vb[3] = {0.0, 0.0, 0.0}, c0b = 0.0, hb = 0.0, Upb = 0.0;
  // S(a + dp, b + dq) with weight w
  auto S_adj = [&](int dp, int dq, R w) {
    Ub[dp] += w * T.v[b + dq];
    Tb.v[b + dq] += w * U[dp];
    Tb.u[a + dp] += w * V[dq];
    Vb[dq] += w * T.u[a + dp];
  };
  const R w3 = 0.5 * ob[3];
  S_adj(0, 0, ob[0]);
  S_adj(1, 0, ob[1]);
  S_adj(0, 1, ob[2]);
  S_adj(2, 0, w3);
  S_adj(0, 2, w3);
  // Sx with weight w3
  {
    const R inner = T.v[b] * Up + T.u[a] * V[0];
    Tb.xi[1] += w3 * inner;
    const R wi = w3 * x1;
    Upb += wi * T.v[b];
    Tb.v[b] += wi * Up;
    Tb.u[a] += wi * V[0];
    Vb[0] += wi * T.u[a];
    const R uv = T.u[a] * T.v[b];
    hb += w3 * x2 * uv;
    Tb.xi[2] += w3 * h * uv;
    Tb.u[a] += w3 * h * x2 * T.v[b];
    Tb.v[b] += w3 * h * x2 * T.u[a];
  }
  // U(a + k), V(b + k), U'(a)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c0b += Ub[k] * T.u[a + k];
    sb[1] += Ub[k] * T.u[a + k + 1];
    hb += Ub[k] * T.u[a + k + 2];
    Tb.u[a + k] += Ub[k] * c0;
    Tb.u[a + k + 1] += Ub[k] * s[1];
    Tb.u[a + k + 2] += Ub[k] * h;
    sb[2] += Vb[k] * T.v[b + k + 1];
    hb += Vb[k] * T.v[b + k + 2];
    Tb.v[b + k + 1] += Vb[k] * s[2];
    Tb.v[b + k + 2] += Vb[k] * h;
  }
  sb[0] += Upb * T.u[a];
  sb[1] += Upb * T.u[a + 1];
  hb += Upb * T.u[a + 2];
  Tb.u[a] += Upb * s[0];
  Tb.u[a + 1] += Upb * s[1];
  Tb.u[a + 2] += Upb * h;
  // c0 = s0 + h xi[1], h = s3 / 2
  sb[0] += c0b;
  hb += c0b * x1;
  Tb.xi[1] += c0b * h;
  sb[3] += 0.5 * hb;
}

// s = slope_solve(g, r): sb -> rb, gb (added)
FD_HD void slope_solve_adj(const Maxw<R>& g, R K, R c4K, const R r[4], const R s[4], const R sb_in[4], MaxwB& gb,
                           R rb[4]) {
  const R q = g.U * g.U + g.V * g.V + (K + 2.0) * g.i2l;
  const R Ah = r[1] - g.U * r[0], Ch = r[2] - g.V * r[0], B = 2.0 * r[3] - q * r[0];
  const R X = B - 2.0 * g.U * Ah - 2.0 * g.V * Ch;
  R s1b = sb_in[1], s2b = sb_in[2], s3b = sb_in[3], qb = 0.0, Ahb = 0.0, Chb = 0.0;
  // s0 = r0 - U s1 - V s2 - s3 q / 2
  const R s0b = sb_in[0];
  rb[0] += s0b;
  gb.U -= s0b * s[1];
  gb.V -= s0b * s[2];
  s1b -= s0b * g.U;
  s2b -= s0b * g.V;
  s3b -= 0.5 * s0b * q;
  qb -= 0.5 * s0b * s[3];
  // s1 = 2 lam Ah - U s3, s2 = 2 lam Ch - V s3
  gb.lam += 2.0 * (Ah * s1b + Ch * s2b);
  Ahb += 2.0 * g.lam * s1b;
  Chb += 2.0 * g.lam * s2b;
  gb.U -= s[3] * s1b;
  gb.V -= s[3] * s2b;
  s3b -= g.U * s1b + g.V * s2b;
  // s3 = c4K lam^2 X
  gb.lam += 2.0 * c4K * g.lam * X * s3b;
  const R Xb = c4K * g.lam * g.lam * s3b;
  const R Bb = Xb;
  gb.U -= 2.0 * Ah * Xb;
  Ahb -= 2.0 * g.U * Xb;
  gb.V -= 2.0 * Ch * Xb;
  Chb -= 2.0 * g.V * Xb;
  // B = 2 r3 - q r0, Ch = r2 - V r0, Ah = r1 - U r0
  rb[3] += 2.0 * Bb;
  qb -= r[0] * Bb;
  rb[0] -= q * Bb;
  rb[2] += Chb;
  gb.V -= r[0] * Chb;
  rb[0] -= g.V * Chb;
  rb[1] += Ahb;
  gb.U -= r[0] * Ahb;
  rb[0] -= g.U * Ahb;
  // q = U^2 + V^2 + (K + 2) i2l
  gb.U += 2.0 * g.U * qb;
  gb.V += 2.0 * g.V * qb;
  gb.i2l += (K + 2.0) * qb;
}

// heat flux of the energy flux relative to (U0, V0), x-normal and y-normal:
// adds hb times its partial derivatives to Fb, Wb, U0b, V0b
FD_HD void heat_flux_x_adj(const R F[4], const R W[4], R U0, R V0, R hb, R Fb[4], R Wb[4], R& U0b, R& V0b) {
  Fb[3] += hb;
  Wb[3] -= U0 * hb;
  Fb[1] -= U0 * hb;
  Fb[2] -= V0 * hb;
  Wb[1] += (1.5 * U0 * U0 + 0.5 * V0 * V0) * hb;
  Wb[2] += U0 * V0 * hb;
  Wb[0] -= 0.5 * U0 * (U0 * U0 + V0 * V0) * hb;
  U0b += hb * (-W[3] - F[1] + 3.0 * U0 * W[1] + V0 * W[2] - 0.5 * (3.0 * U0 * U0 + V0 * V0) * W[0]);
  V0b += hb * (-F[2] + V0 * W[1] + U0 * W[2] - U0 * V0 * W[0]);
}
FD_HD void heat_flux_y_adj(const R G[4], const R W[4], R U0, R V0, R hb, R Gb[4], R Wb[4], R& U0b, R& V0b) {
  Gb[3] += hb;
  Wb[3] -= V0 * hb;
  Gb[2] -= V0 * hb;
  Gb[1] -= U0 * hb;
  Wb[2] += (1.5 * V0 * V0 + 0.5 * U0 * U0) * hb;
  Wb[1] += U0 * V0 * hb;
  Wb[0] -= 0.5 * V0 * (U0 * U0 + V0 * V0) * hb;
  V0b += hb * (-W[3] - G[2] + 3.0 * V0 * W[2] + U0 * W[1] - 0.5 * (3.0 * V0 * V0 + U0 * U0) * W[0]);
  U0b += hb * (-G[1] + U0 * W[2] + V0 * W[1] - U0 * V0 * W[0]);
}

// time coefficients of the interface distribution (time_coef): the adjoints
// of cn[6], ct[6], E, e1 -> d/dtau
FD_HD R time_coef_adj(R tau, R dt, R inv_dt, const R cnb_in[6], const R ctb_in[6], R Eb, R e1b) {
  const R em = s_expm1(-0.5 * dt / tau);
  const R Eh = 1.0 + em, e1h = -em, E = Eh * Eh, e1 = -em * (em + 2.0);
  R cnb[3], ctb[3], taub = 0.0;
  // cn3 = 1 - cn0, ct3 = -ct0, cn4 = -tau - cn1, ct4 = -ct1, cn5 = -tau - cn2, ct5 = 1 - ct2
  cnb[0] = cnb_in[0] - cnb_in[3];
  ctb[0] = ctb_in[0] - ctb_in[3];
  cnb[1] = cnb_in[1] - cnb_in[4];
  ctb[1] = ctb_in[1] - ctb_in[4];
  cnb[2] = cnb_in[2] - cnb_in[5];
  ctb[2] = ctb_in[2] - ctb_in[5];
  taub -= cnb_in[4] + cnb_in[5];
  R Ehb = 0.0, e1hb = 0.0;
  for (int half = 0; half < 2; ++half) {
    // Ch (d = dt/2, with Eh, e1h) and Cf (d = dt, with E, e1)
    const R d = half ? 0.5 * dt : dt;
    const R EE = half ? Eh : E, ee = half ? e1h : e1;
    R Cb[3];
    for (int k = 0; k < 3; ++k)
      Cb[k] = half ? 4.0 * inv_dt * cnb[k] - 8.0 * inv_dt * inv_dt * ctb[k]
                   : -inv_dt * cnb[k] + 4.0 * inv_dt * inv_dt * ctb[k];
    // C0 = d - tau ee, C1 = -tau d (1 + EE) + 2 tau^2 ee, C2 = d^2/2 - tau d + tau^2 ee
    taub += -ee * Cb[0] + (-d * (1.0 + EE) + 4.0 * tau * ee) * Cb[1] + (-d + 2.0 * tau * ee) * Cb[2];
    const R eeb = -tau * Cb[0] + 2.0 * tau * tau * Cb[1] + tau * tau * Cb[2];
    const R EEb = -tau * d * Cb[1];
    if (half) { Ehb += EEb; e1hb += eeb; }
    else { Eb += EEb; e1b += eeb; }
  }
  // E = Eh^2, e1 = -em (em + 2), Eh = 1 + em, e1h = -em
  Ehb += 2.0 * Eh * Eb;
  const R emb = Ehb - e1hb - (2.0 * em + 2.0) * e1b;
  // em = expm1(-dt / (2 tau)): d em / d tau = (em + 1) dt / (2 tau^2); zero when em + 1 is
  if (emb != 0.0 && em + 1.0 != 0.0) taub += emb * (em + 1.0) * 0.5 * dt / (tau * tau);
  return taub;
}

// ---------------------------------------------------------------------------
// kinetic interface solve, x-normal (iface_solve_x): output adjoints ob ->
// input adjoints (added)
// ---------------------------------------------------------------------------
FD_HD void iface_solve_x_adj(const GasK<R>& gas, const R Wl[4], const R Wr[4], const R Wln[4], const R Wrn[4],
                             const R Wt[4], bool want_n, const IfaceOut<R>& ob, R Wlb[4], R Wrb[4], R Wlnb[4],
                             R Wrnb[4], R Wtb[4]) {
  const R K = gas.K, c4K = gas.c4K, gm1 = gas.gm1;
  // ---- forward ----
  const Maxw<R> gl = maxw_from_W(Wl, gm1), gr = maxw_from_W(Wr, gm1);
  Tab<R> Tl, Tr, Tlp, Trn;
  tab_full(gl, K, Tl);
  tab_full(gr, K, Tr);
  tab_half(gl, +1, Tl, Tlp);
  tab_half(gr, -1, Tr, Trn);
  R W0[4], pl0[4], pr0[4];
  mpsi<0, 0, 0>(Tlp, pl0);
  mpsi<0, 0, 0>(Trn, pr0);
  for (int k = 0; k < 4; ++k) W0[k] = gl.rho * pl0[k] + gr.rho * pr0[k];
  const Maxw<R> g0 = maxw_from_W(W0, gm1);
  Tab<R> T0;
  tab_full(g0, K, T0);
  R ral[4], rbl[4], rar[4], rbr[4], ra0[4], rb0[4];
  for (int k = 0; k < 4; ++k) {
    ral[k] = Wln[k] * gl.ir;
    rbl[k] = Wt[k] * gl.ir;
    rar[k] = Wrn[k] * gr.ir;
    rbr[k] = Wt[k] * gr.ir;
    ra0[k] = 0.5 * (Wln[k] + Wrn[k]) * g0.ir;
    rb0[k] = Wt[k] * g0.ir;
  }
  R al[4], bl[4], ar[4], br[4], a0[4], b0[4];
  slope_solve(gl, K, c4K, ral, al);
  slope_solve(gl, K, c4K, rbl, bl);
  slope_solve(gr, K, c4K, rar, ar);
  slope_solve(gr, K, c4K, rbr, br);
  slope_solve(g0, K, c4K, ra0, a0);
  slope_solve(g0, K, c4K, rb0, b0);
  R rl[4], rr[4], r0[4], Al[4], Ar[4], A0[4], x1[4], x2[4];
  mslope<1, 0>(Tl, al, x1);
  mslope<0, 1>(Tl, bl, x2);
  for (int k = 0; k < 4; ++k) rl[k] = -(x1[k] + x2[k]);
  slope_solve(gl, K, c4K, rl, Al);
  mslope<1, 0>(Tr, ar, x1);
  mslope<0, 1>(Tr, br, x2);
  for (int k = 0; k < 4; ++k) rr[k] = -(x1[k] + x2[k]);
  slope_solve(gr, K, c4K, rr, Ar);
  mslope<1, 0>(T0, a0, x1);
  mslope<0, 1>(T0, b0, x2);
  for (int k = 0; k < 4; ++k) r0[k] = -(x1[k] + x2[k]);
  slope_solve(g0, K, c4K, r0, A0);
  const R ip0 = 2.0 * g0.lam * g0.ir;
  const R dp = gl.p - gr.p, sp = gl.p + gr.p;
  const R tau = gas.c1 * gas.dt + gas.mu * ip0 + gas.c2 * gas.dt * s_abs(dp) / sp;
  const TimeCoef<R> tc = time_coef(tau, gas.dt, gas.inv_dt);
  // the six basis terms' flux (mf) and W (mw) moment vectors
  R mf[6][4], mw[6][4], y1[4], y2[4];
  mpsi<1, 0, 0>(T0, mf[0]);
  mpsi<0, 0, 0>(T0, mw[0]);
  for (int k = 0; k < 4; ++k) { mf[0][k] *= g0.rho; mw[0][k] *= g0.rho; }
  mslope<2, 0>(T0, a0, x1);
  mslope<1, 1>(T0, b0, x2);
  for (int k = 0; k < 4; ++k) { mf[1][k] = g0.rho * (x1[k] + x2[k]); mw[1][k] = -g0.rho * r0[k]; }
  mslope<1, 0>(T0, A0, x1);
  for (int k = 0; k < 4; ++k) { mf[2][k] = g0.rho * x1[k]; mw[2][k] = g0.rho * r0[k]; }
  mpsi<1, 0, 0>(Tlp, x1);
  mpsi<1, 0, 0>(Trn, x2);
  for (int k = 0; k < 4; ++k) { mf[3][k] = gl.rho * x1[k] + gr.rho * x2[k]; mw[3][k] = W0[k]; }
  mslope<2, 0>(Tlp, al, x1);
  mslope<1, 1>(Tlp, bl, x2);
  mslope<2, 0>(Trn, ar, y1);
  mslope<1, 1>(Trn, br, y2);
  for (int k = 0; k < 4; ++k) mf[4][k] = gl.rho * (x1[k] + x2[k]) + gr.rho * (y1[k] + y2[k]);
  mslope<1, 0>(Tlp, al, x1);
  mslope<0, 1>(Tlp, bl, x2);
  mslope<1, 0>(Trn, ar, y1);
  mslope<0, 1>(Trn, br, y2);
  for (int k = 0; k < 4; ++k) mw[4][k] = gl.rho * (x1[k] + x2[k]) + gr.rho * (y1[k] + y2[k]);
  mslope<1, 0>(Tlp, Al, x1);
  mslope<1, 0>(Trn, Ar, y1);
  mslope<0, 0>(Tlp, Al, x2);
  mslope<0, 0>(Trn, Ar, y2);
  for (int k = 0; k < 4; ++k) { mf[5][k] = gl.rho * x1[k] + gr.rho * y1[k]; mw[5][k] = gl.rho * x2[k] + gr.rho * y2[k]; }
  R F[4], Ftt[4], We[4], Wet[4];
  for (int k = 0; k < 4; ++k) {
    F[k] = Ftt[k] = We[k] = Wet[k] = 0.0;
    for (int kk = 0; kk < 6; ++kk) {
      F[k] += tc.cn[kk] * mf[kk][k];
      Ftt[k] += tc.ct[kk] * mf[kk][k];
      We[k] += tc.cn[kk] * mw[kk][k];
      Wet[k] += tc.ct[kk] * mw[kk][k];
    }
  }
  const R E = tc.E, e1 = tc.e1;

  // ---- reverse ----
  MaxwB glb = maxw_zero(), grb = maxw_zero(), g0b = maxw_zero();
  TabB Tlb = tab_zero(), Trb = tab_zero(), Tlpb = tab_zero(), Trnb = tab_zero(), T0b = tab_zero();
  R Fb[4], Fttb[4], Web[4], Wetb[4], rlb[4], rrb[4], r0b[4], Eb = 0.0, e1b = 0.0;
  for (int k = 0; k < 4; ++k) {
    rlb[k] = rrb[k] = r0b[k] = 0.0;
    // o.Ft = Ftt; o.Wlt = e1 Wet + E rho_l rl; o.Wrt = e1 Wet + E rho_r rr
    Fttb[k] = ob.Ft[k];
    Wetb[k] = e1 * (ob.Wlt[k] + ob.Wrt[k]);
    e1b += Wet[k] * (ob.Wlt[k] + ob.Wrt[k]);
    Eb += gl.rho * rl[k] * ob.Wlt[k] + gr.rho * rr[k] * ob.Wrt[k];
    glb.rho += E * rl[k] * ob.Wlt[k];
    grb.rho += E * rr[k] * ob.Wrt[k];
    rlb[k] += E * gl.rho * ob.Wlt[k];
    rrb[k] += E * gr.rho * ob.Wrt[k];
    Fb[k] = Web[k] = 0.0;
    if (want_n) {
      // o.F = F; o.Wl = e1 We + E Wl; o.Wr = e1 We + E Wr
      Fb[k] = ob.F[k];
      Web[k] = e1 * (ob.Wl[k] + ob.Wr[k]);
      e1b += We[k] * (ob.Wl[k] + ob.Wr[k]);
      Eb += Wl[k] * ob.Wl[k] + Wr[k] * ob.Wr[k];
      Wlb[k] += E * ob.Wl[k];
      Wrb[k] += E * ob.Wr[k];
    }
  }
  // Prandtl correction F3 += prfix q(F, We), Ftt3 likewise (F, Ftt above are
  // the sums before the correction; only the energy components change)
  heat_flux_x_adj(F, We, g0.U, g0.V, gas.prfix * Fb[3], Fb, Web, g0b.U, g0b.V);
  heat_flux_x_adj(Ftt, Wet, g0.U, g0.V, gas.prfix * Fttb[3], Fttb, Wetb, g0b.U, g0b.V);
  // accumulation F = sum cn mf, ... -> adjoints of mf, mw and of the coefficients
  R cnb[6], ctb[6], mfb[6][4], mwb[6][4];
  for (int kk = 0; kk < 6; ++kk) {
    cnb[kk] = ctb[kk] = 0.0;
    for (int k = 0; k < 4; ++k) {
      mfb[kk][k] = tc.cn[kk] * Fb[k] + tc.ct[kk] * Fttb[k];
      mwb[kk][k] = tc.cn[kk] * Web[k] + tc.ct[kk] * Wetb[k];
      cnb[kk] += mf[kk][k] * Fb[k] + mw[kk][k] * Web[k];
      ctb[kk] += mf[kk][k] * Fttb[k] + mw[kk][k] * Wetb[k];
    }
  }
  R W0b[4] = {0.0, 0.0, 0.0, 0.0};
  R alb[4] = {0, 0, 0, 0}, blb[4] = {0, 0, 0, 0}, arb[4] = {0, 0, 0, 0}, brb[4] = {0, 0, 0, 0};
  R a0b[4] = {0, 0, 0, 0}, b0b[4] = {0, 0, 0, 0}, Alb[4] = {0, 0, 0, 0}, Arb[4] = {0, 0, 0, 0};
  R A0b[4] = {0, 0, 0, 0};
  R t[4];
  // term 0: rho0 <u psi>_0, rho0 <psi>_0
  mpsi<1, 0, 0>(T0, x1);
  mpsi<0, 0, 0>(T0, x2);
  for (int k = 0; k < 4; ++k) g0b.rho += x1[k] * mfb[0][k] + x2[k] * mwb[0][k];
  for (int k = 0; k < 4; ++k) t[k] = g0.rho * mfb[0][k];
  mpsi_adj<1, 0, 0>(T0, t, T0b);
  for (int k = 0; k < 4; ++k) t[k] = g0.rho * mwb[0][k];
  mpsi_adj<0, 0, 0>(T0, t, T0b);
  // term 1: rho0 (<a0 u u psi> + <b0 u v psi>), -rho0 r0
  mslope<2, 0>(T0, a0, x1);
  mslope<1, 1>(T0, b0, x2);
  for (int k = 0; k < 4; ++k) {
    g0b.rho += (x1[k] + x2[k]) * mfb[1][k] - r0[k] * mwb[1][k];
    r0b[k] -= g0.rho * mwb[1][k];
    t[k] = g0.rho * mfb[1][k];
  }
  mslope_adj<2, 0>(T0, a0, t, T0b, a0b);
  mslope_adj<1, 1>(T0, b0, t, T0b, b0b);
  // term 2: rho0 <A0 u psi>, rho0 r0
  mslope<1, 0>(T0, A0, x1);
  for (int k = 0; k < 4; ++k) {
    g0b.rho += x1[k] * mfb[2][k] + r0[k] * mwb[2][k];
    r0b[k] += g0.rho * mwb[2][k];
    t[k] = g0.rho * mfb[2][k];
  }
  mslope_adj<1, 0>(T0, A0, t, T0b, A0b);
  // term 3: rho_l <u psi>_{u>0} + rho_r <u psi>_{u<0}, W0
  mpsi<1, 0, 0>(Tlp, x1);
  mpsi<1, 0, 0>(Trn, x2);
  for (int k = 0; k < 4; ++k) {
    glb.rho += x1[k] * mfb[3][k];
    grb.rho += x2[k] * mfb[3][k];
    W0b[k] += mwb[3][k];
  }
  for (int k = 0; k < 4; ++k) t[k] = gl.rho * mfb[3][k];
  mpsi_adj<1, 0, 0>(Tlp, t, Tlpb);
  for (int k = 0; k < 4; ++k) t[k] = gr.rho * mfb[3][k];
  mpsi_adj<1, 0, 0>(Trn, t, Trnb);
  // term 4: the one-sided (a u + b v) terms
  {
    R f1[4], f2[4], f3[4], f4[4], w1[4], w2[4], w3[4], w4[4];
    mslope<2, 0>(Tlp, al, f1);
    mslope<1, 1>(Tlp, bl, f2);
    mslope<2, 0>(Trn, ar, f3);
    mslope<1, 1>(Trn, br, f4);
    mslope<1, 0>(Tlp, al, w1);
    mslope<0, 1>(Tlp, bl, w2);
    mslope<1, 0>(Trn, ar, w3);
    mslope<0, 1>(Trn, br, w4);
    for (int k = 0; k < 4; ++k) {
      glb.rho += (f1[k] + f2[k]) * mfb[4][k] + (w1[k] + w2[k]) * mwb[4][k];
      grb.rho += (f3[k] + f4[k]) * mfb[4][k] + (w3[k] + w4[k]) * mwb[4][k];
    }
    for (int k = 0; k < 4; ++k) t[k] = gl.rho * mfb[4][k];
    mslope_adj<2, 0>(Tlp, al, t, Tlpb, alb);
    mslope_adj<1, 1>(Tlp, bl, t, Tlpb, blb);
    for (int k = 0; k < 4; ++k) t[k] = gr.rho * mfb[4][k];
    mslope_adj<2, 0>(Trn, ar, t, Trnb, arb);
    mslope_adj<1, 1>(Trn, br, t, Trnb, brb);
    for (int k = 0; k < 4; ++k) t[k] = gl.rho * mwb[4][k];
    mslope_adj<1, 0>(Tlp, al, t, Tlpb, alb);
    mslope_adj<0, 1>(Tlp, bl, t, Tlpb, blb);
    for (int k = 0; k < 4; ++k) t[k] = gr.rho * mwb[4][k];
    mslope_adj<1, 0>(Trn, ar, t, Trnb, arb);
    mslope_adj<0, 1>(Trn, br, t, Trnb, brb);
  }
  // term 5: the one-sided A terms
  {
    R f1[4], f3[4], w1[4], w3[4];
    mslope<1, 0>(Tlp, Al, f1);
    mslope<1, 0>(Trn, Ar, f3);
    mslope<0, 0>(Tlp, Al, w1);
    mslope<0, 0>(Trn, Ar, w3);
    for (int k = 0; k < 4; ++k) {
      glb.rho += f1[k] * mfb[5][k] + w1[k] * mwb[5][k];
      grb.rho += f3[k] * mfb[5][k] + w3[k] * mwb[5][k];
    }
    for (int k = 0; k < 4; ++k) t[k] = gl.rho * mfb[5][k];
    mslope_adj<1, 0>(Tlp, Al, t, Tlpb, Alb);
    for (int k = 0; k < 4; ++k) t[k] = gr.rho * mfb[5][k];
    mslope_adj<1, 0>(Trn, Ar, t, Trnb, Arb);
    for (int k = 0; k < 4; ++k) t[k] = gl.rho * mwb[5][k];
    mslope_adj<0, 0>(Tlp, Al, t, Tlpb, Alb);
    for (int k = 0; k < 4; ++k) t[k] = gr.rho * mwb[5][k];
    mslope_adj<0, 0>(Trn, Ar, t, Trnb, Arb);
  }
  // time coefficients and the collision time
  {
    const R taub = time_coef_adj(tau, gas.dt, gas.inv_dt, cnb, ctb, Eb, e1b);
    const R ip0b = gas.mu * taub;
    g0b.lam += 2.0 * g0.ir * ip0b;
    g0b.ir += 2.0 * g0.lam * ip0b;
    // |dp| / sp with d|x|/dx = sign(x), 0 at x = 0
    const R s = sgn0(dp), adp = s_abs(dp);
    const R c = gas.c2 * gas.dt * taub / (sp * sp);
    glb.p += c * (s * sp - adp);
    grb.p += c * (-s * sp - adp);
  }
  // time slopes A = slope_solve(g, -<(a u + b v) psi>)
  slope_solve_adj(g0, K, c4K, r0, A0, A0b, g0b, r0b);
  for (int k = 0; k < 4; ++k) t[k] = -r0b[k];
  mslope_adj<1, 0>(T0, a0, t, T0b, a0b);
  mslope_adj<0, 1>(T0, b0, t, T0b, b0b);
  slope_solve_adj(gr, K, c4K, rr, Ar, Arb, grb, rrb);
  for (int k = 0; k < 4; ++k) t[k] = -rrb[k];
  mslope_adj<1, 0>(Tr, ar, t, Trb, arb);
  mslope_adj<0, 1>(Tr, br, t, Trb, brb);
  slope_solve_adj(gl, K, c4K, rl, Al, Alb, glb, rlb);
  for (int k = 0; k < 4; ++k) t[k] = -rlb[k];
  mslope_adj<1, 0>(Tl, al, t, Tlb, alb);
  mslope_adj<0, 1>(Tl, bl, t, Tlb, blb);
  // spatial slopes from r = dW / rho
  {
    R rb_[4];
    for (int k = 0; k < 4; ++k) rb_[k] = 0.0;
    slope_solve_adj(g0, K, c4K, rb0, b0, b0b, g0b, rb_);
    for (int k = 0; k < 4; ++k) { Wtb[k] += rb_[k] * g0.ir; g0b.ir += rb_[k] * Wt[k]; rb_[k] = 0.0; }
    slope_solve_adj(g0, K, c4K, ra0, a0, a0b, g0b, rb_);
    for (int k = 0; k < 4; ++k) {
      Wlnb[k] += 0.5 * rb_[k] * g0.ir;
      Wrnb[k] += 0.5 * rb_[k] * g0.ir;
      g0b.ir += rb_[k] * 0.5 * (Wln[k] + Wrn[k]);
      rb_[k] = 0.0;
    }
    slope_solve_adj(gr, K, c4K, rbr, br, brb, grb, rb_);
    for (int k = 0; k < 4; ++k) { Wtb[k] += rb_[k] * gr.ir; grb.ir += rb_[k] * Wt[k]; rb_[k] = 0.0; }
    slope_solve_adj(gr, K, c4K, rar, ar, arb, grb, rb_);
    for (int k = 0; k < 4; ++k) { Wrnb[k] += rb_[k] * gr.ir; grb.ir += rb_[k] * Wrn[k]; rb_[k] = 0.0; }
    slope_solve_adj(gl, K, c4K, rbl, bl, blb, glb, rb_);
    for (int k = 0; k < 4; ++k) { Wtb[k] += rb_[k] * gl.ir; glb.ir += rb_[k] * Wt[k]; rb_[k] = 0.0; }
    slope_solve_adj(gl, K, c4K, ral, al, alb, glb, rb_);
    for (int k = 0; k < 4; ++k) { Wlnb[k] += rb_[k] * gl.ir; glb.ir += rb_[k] * Wln[k]; }
  }
  // equilibrium state W0 = rho_l <psi>_{u>0} + rho_r <psi>_{u<0} and its Maxwellian
  tab_full_adj(g0, K, T0, T0b, g0b);
  maxw_from_W_adj(W0, gm1, g0, g0b, W0b);
  for (int k = 0; k < 4; ++k) {
    glb.rho += pl0[k] * W0b[k];
    grb.rho += pr0[k] * W0b[k];
    t[k] = gl.rho * W0b[k];
  }
  mpsi_adj<0, 0, 0>(Tlp, t, Tlpb);
  for (int k = 0; k < 4; ++k) t[k] = gr.rho * W0b[k];
  mpsi_adj<0, 0, 0>(Trn, t, Trnb);
  // one-sided tables and the Maxwellians of the two sides
  tab_half_adj(gl, +1, Tlp, Tlpb, Tlb, glb);
  tab_half_adj(gr, -1, Trn, Trnb, Trb, grb);
  tab_full_adj(gl, K, Tl, Tlb, glb);
  tab_full_adj(gr, K, Tr, Trb, grb);
  maxw_from_W_adj(Wl, gm1, gl, glb, Wlb);
  maxw_from_W_adj(Wr, gm1, gr, grb, Wrb);
}

// any normal: the x <-> y transposition of iface_solve, transposed
FD_HD void iface_solve_adj(const GasK<R>& gas, int normal, const R Wl[4], const R Wr[4], const R Wln[4], const R Wrn[4],
                           const R Wt[4], bool want_n, const IfaceOut<R>& ob, R Wlb[4], R Wrb[4], R Wlnb[4],
                           R Wrnb[4], R Wtb[4]) {
  const bool sw = normal != 0;
  R a[4], b[4], c[4], d[4], e[4];
  swap_uv(Wl, a, sw); swap_uv(Wr, b, sw); swap_uv(Wln, c, sw); swap_uv(Wrn, d, sw); swap_uv(Wt, e, sw);
  IfaceOut<R> obs;
  swap_uv(ob.Ft, obs.Ft, sw); swap_uv(ob.Wlt, obs.Wlt, sw); swap_uv(ob.Wrt, obs.Wrt, sw);
  if (want_n) { swap_uv(ob.F, obs.F, sw); swap_uv(ob.Wl, obs.Wl, sw); swap_uv(ob.Wr, obs.Wr, sw); }
  R ab[4] = {0, 0, 0, 0}, bb[4] = {0, 0, 0, 0}, cb[4] = {0, 0, 0, 0}, db[4] = {0, 0, 0, 0}, eb[4] = {0, 0, 0, 0};
  iface_solve_x_adj(gas, a, b, c, d, e, want_n, obs, ab, bb, cb, db, eb);
  R t[4];
  swap_uv(ab, t, sw); for (int k = 0; k < 4; ++k) Wlb[k] += t[k];
  swap_uv(bb, t, sw); for (int k = 0; k < 4; ++k) Wrb[k] += t[k];
  swap_uv(cb, t, sw); for (int k = 0; k < 4; ++k) Wlnb[k] += t[k];
  swap_uv(db, t, sw); for (int k = 0; k < 4; ++k) Wrnb[k] += t[k];
  swap_uv(eb, t, sw); for (int k = 0; k < 4; ++k) Wtb[k] += t[k];
}

// ---------------------------------------------------------------------------
// nodal flux (Sec. 2.1): adjoints of F, G, F_t, G_t -> of W, W_x, W_y (added)
// ---------------------------------------------------------------------------
FD_HD void nodal_flux_adj(const GasK<R>& gas, const R W[4], const R Wx[4], const R Wy[4], const R Fb_in[4],
                          const R Gb_in[4], const R Ftb_in[4], const R Gtb_in[4], R Wb[4], R Wxb[4], R Wyb[4]) {
  const R K = gas.K, c4K = gas.c4K;
  const Maxw<R> g = maxw_from_W(W, gas.gm1);
  Tab<R> T;
  tab_full(g, K, T);
  R rx[4], ry[4], a[4], b[4], r[4], A[4], x1[4], x2[4], Wt[4];
  for (int k = 0; k < 4; ++k) { rx[k] = Wx[k] * g.ir; ry[k] = Wy[k] * g.ir; }
  slope_solve(g, K, c4K, rx, a);
  slope_solve(g, K, c4K, ry, b);
  mslope<1, 0>(T, a, x1);
  mslope<0, 1>(T, b, x2);
  for (int k = 0; k < 4; ++k) r[k] = -(x1[k] + x2[k]);
  slope_solve(g, K, c4K, r, A);
  for (int k = 0; k < 4; ++k) Wt[k] = g.rho * r[k];
  const R tau = gas.c1_r * gas.dt_r + gas.mu_r * (2.0 * g.lam * g.ir);
  R e0x[4], eax[4], ebx[4], eAx[4], e0y[4], eay[4], eby[4], eAy[4];
  mpsi<1, 0, 0>(T, e0x);
  mslope<2, 0>(T, a, eax);
  mslope<1, 1>(T, b, ebx);
  mslope<1, 0>(T, A, eAx);
  mpsi<0, 1, 0>(T, e0y);
  mslope<1, 1>(T, a, eay);
  mslope<0, 2>(T, b, eby);
  mslope<0, 1>(T, A, eAy);
  R F[4], G[4], Ft[4], Gt[4];   // before the Prandtl correction
  for (int k = 0; k < 4; ++k) {
    F[k] = g.rho * (e0x[k] - tau * (eax[k] + ebx[k] + eAx[k]));
    Ft[k] = g.rho * eAx[k];
    G[k] = g.rho * (e0y[k] - tau * (eay[k] + eby[k] + eAy[k]));
    Gt[k] = g.rho * eAy[k];
  }
  // ---- reverse ----
  MaxwB gb = maxw_zero();
  TabB Tb = tab_zero();
  R Fb[4], Gb[4], Ftb[4], Gtb[4], Wtb[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) { Fb[k] = Fb_in[k]; Gb[k] = Gb_in[k]; Ftb[k] = Ftb_in[k]; Gtb[k] = Gtb_in[k]; }
  heat_flux_x_adj(F, W, g.U, g.V, gas.prfix * Fb[3], Fb, Wb, gb.U, gb.V);
  heat_flux_y_adj(G, W, g.U, g.V, gas.prfix * Gb[3], Gb, Wb, gb.U, gb.V);
  heat_flux_x_adj(Ft, Wt, g.U, g.V, gas.prfix * Ftb[3], Ftb, Wtb, gb.U, gb.V);
  heat_flux_y_adj(Gt, Wt, g.U, g.V, gas.prfix * Gtb[3], Gtb, Wtb, gb.U, gb.V);
  R e0b[4], sb[4], eAb[4], taub = 0.0, ab[4] = {0, 0, 0, 0}, bb[4] = {0, 0, 0, 0}, Ab[4] = {0, 0, 0, 0};
  // x-flux: F = rho (e0 - tau (ea + eb + eA)), Ft = rho eA
  for (int k = 0; k < 4; ++k) {
    gb.rho += (e0x[k] - tau * (eax[k] + ebx[k] + eAx[k])) * Fb[k] + eAx[k] * Ftb[k];
    taub -= g.rho * (eax[k] + ebx[k] + eAx[k]) * Fb[k];
    e0b[k] = g.rho * Fb[k];
    sb[k] = -g.rho * tau * Fb[k];
    eAb[k] = sb[k] + g.rho * Ftb[k];
  }
  mpsi_adj<1, 0, 0>(T, e0b, Tb);
  mslope_adj<2, 0>(T, a, sb, Tb, ab);
  mslope_adj<1, 1>(T, b, sb, Tb, bb);
  mslope_adj<1, 0>(T, A, eAb, Tb, Ab);
  for (int k = 0; k < 4; ++k) {
    gb.rho += (e0y[k] - tau * (eay[k] + eby[k] + eAy[k])) * Gb[k] + eAy[k] * Gtb[k];
    taub -= g.rho * (eay[k] + eby[k] + eAy[k]) * Gb[k];
    e0b[k] = g.rho * Gb[k];
    sb[k] = -g.rho * tau * Gb[k];
    eAb[k] = sb[k] + g.rho * Gtb[k];
  }
  mpsi_adj<0, 1, 0>(T, e0b, Tb);
  mslope_adj<1, 1>(T, a, sb, Tb, ab);
  mslope_adj<0, 2>(T, b, sb, Tb, bb);
  mslope_adj<0, 1>(T, A, eAb, Tb, Ab);
  // tau = c1 dt + mu (2 lam ir)
  gb.lam += gas.mu_r * 2.0 * g.ir * taub;
  gb.ir += gas.mu_r * 2.0 * g.lam * taub;
  // Wt = rho r, A = slope_solve(g, r), r = -(<a u psi> + <b v psi>)
  R rb[4];
  for (int k = 0; k < 4; ++k) {
    gb.rho += r[k] * Wtb[k];
    rb[k] = g.rho * Wtb[k];
  }
  slope_solve_adj(g, K, c4K, r, A, Ab, gb, rb);
  for (int k = 0; k < 4; ++k) rb[k] = -rb[k];
  mslope_adj<1, 0>(T, a, rb, Tb, ab);
  mslope_adj<0, 1>(T, b, rb, Tb, bb);
  R rxb[4] = {0, 0, 0, 0}, ryb[4] = {0, 0, 0, 0};
  slope_solve_adj(g, K, c4K, ry, b, bb, gb, ryb);
  slope_solve_adj(g, K, c4K, rx, a, ab, gb, rxb);
  for (int k = 0; k < 4; ++k) {
    Wxb[k] += rxb[k] * g.ir;
    Wyb[k] += ryb[k] * g.ir;
    gb.ir += rxb[k] * Wx[k] + ryb[k] * Wy[k];
  }
  tab_full_adj(g, K, T, Tb, gb);
  maxw_from_W_adj(W, gas.gm1, g, gb, Wb);
}

}  // namespace rev
}  // namespace fdk
