"""Velocity-space quadrature of Maxwellian moments (test reference, independent of the oracle).

Under g = rho (lam/pi)^{(K+2)/2} exp(-lam((u-U)^2 + (v-V)^2 + xi^2)) the particle
velocities u, v are normal with mean U, V and variance 1/(2 lam), and the
internal energy xi^2 (K degrees of freedom) is Gamma(K/2, scale 1/lam).  So
int phi(u, v, xi^2) g dXi = rho E[phi], evaluated here by tensor
Gauss-Hermite (u, v) x generalized Gauss-Laguerre (xi^2) quadrature; a
half space in u or v uses Gauss-Legendre on a truncated half line.
"""
import math

import numpy as np
from scipy.special import roots_genlaguerre


def _normal_nodes(m, lam, n):
    x, w = np.polynomial.hermite.hermgauss(n)
    return m + x / math.sqrt(lam), w / math.sqrt(math.pi)


def _half_nodes(m, lam, sign, n=400):
    sd = 1.0 / math.sqrt(2.0 * lam)
    if sign > 0:
        a, b = 0.0, max(0.0, m) + 40.0 * sd
    else:
        a, b = min(0.0, m) - 40.0 * sd, 0.0
    x, w = np.polynomial.legendre.leggauss(n)
    c = 0.5 * (a + b) + 0.5 * (b - a) * x
    wt = 0.5 * (b - a) * w * math.sqrt(lam / math.pi) * np.exp(-lam * (c - m) ** 2)
    return c, wt


def _xi2_nodes(lam, K, n):
    alpha = K / 2.0 - 1.0
    s, w = roots_genlaguerre(n, alpha)
    return s / lam, w / math.gamma(K / 2.0)


def expect(phi, rho, U, V, lam, K, half=None, n=30):
    """rho * E[phi(u, v, xi2)]; half = None, ('u', +1/-1) or ('v', +1/-1)."""
    if half is not None and half[0] == "u":
        u, wu = _half_nodes(U, lam, half[1])
    else:
        u, wu = _normal_nodes(U, lam, n)
    if half is not None and half[0] == "v":
        v, wv = _half_nodes(V, lam, half[1])
    else:
        v, wv = _normal_nodes(V, lam, n)
    s, ws = _xi2_nodes(lam, K, n)
    UU, VV, SS = np.meshgrid(u, v, s, indexing="ij")
    W = wu[:, None, None] * wv[None, :, None] * ws[None, None, :]
    return rho * float(np.sum(W * phi(UU, VV, SS)))


def psi(k, u, v, s):
    return [np.ones_like(u), u, v, 0.5 * (u * u + v * v + s)][k]


def state_of(W, K):
    rho = W[0]
    U, V = W[1] / rho, W[2] / rho
    lam = (K + 2.0) * rho / (4.0 * (W[3] - 0.5 * rho * (U * U + V * V)))
    return rho, U, V, lam
