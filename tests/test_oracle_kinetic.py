"""Pins of the oracle's kinetic layer (paper App. A) against quadrature and closed forms.

Every check here compares the oracle with something it does not share code
with: numerical quadrature in velocity space and in time, or textbook
Euler / Navier-Stokes constitutive relations.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from quadrature import expect, psi, state_of

GAMMA = 1.4
K2D = (4.0 - 2.0 * GAMMA) / (GAMMA - 1.0)   # internal DOF of the 2-D gas (= 3)


def _rand_state(rng):
    rho = rng.uniform(0.5, 2.0)
    U, V = rng.uniform(-1.5, 1.5, size=2)
    p = rng.uniform(0.3, 2.0)
    return np.array([rho, rho * U, rho * V, p / (GAMMA - 1) + 0.5 * rho * (U * U + V * V)])


@pytest.mark.parametrize("seed", range(4))
def test_full_space_moments_match_quadrature(seed):
    rng = np.random.default_rng(seed)
    rho, U, V, lam = rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.3, 3)
    for a in range(7):
        for b in range(0, 7, 2):
            for c in range(3):
                got = oracle.maxwell_moment(rho, U, V, lam, K2D, a, b, c)
                ref = expect(lambda u, v, s: u ** a * v ** b * s ** c, rho, U, V, lam, K2D)
                assert got == pytest.approx(ref, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1)])
def test_half_space_moments_match_quadrature(axis, sign):
    rng = np.random.default_rng(10 + 2 * axis + (sign > 0))
    for _ in range(3):
        rho, U, V, lam = rng.uniform(0.5, 2), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(0.2, 4)
        for a in range(7):
            for b in (0, 1, 3):
                got = oracle.maxwell_moment(rho, U, V, lam, K2D, a, b, 1, axis, sign)
                ref = expect(lambda u, v, s: u ** a * v ** b * s, rho, U, V, lam, K2D,
                             half=("u" if axis == 0 else "v", sign))
                assert got == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_half_spaces_sum_to_full_space():
    for a in range(7):
        full = oracle.maxwell_moment(1.3, 0.4, -0.2, 0.8, K2D, a, 2, 0)
        s = sum(oracle.maxwell_moment(1.3, 0.4, -0.2, 0.8, K2D, a, 2, 0, 0, sg) for sg in (1, -1))
        assert s == pytest.approx(full, rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_slope_reproduces_derivative_moments(seed):
    """a = sum a_l psi_l must satisfy int a psi_k g dXi = dW_k (App. A)."""
    rng = np.random.default_rng(100 + seed)
    W = _rand_state(rng)
    dW = rng.normal(size=4)
    a = oracle.slope(W, dW, GAMMA)
    rho, U, V, lam = state_of(W, K2D)

    def apoly(u, v, s):
        return a[0] + a[1] * u + a[2] * v + a[3] * 0.5 * (u * u + v * v + s)
    for k in range(4):
        got = expect(lambda u, v, s: apoly(u, v, s) * psi(k, u, v, s), rho, U, V, lam, K2D)
        assert got == pytest.approx(dW[k], rel=1e-10, abs=1e-11)


@pytest.mark.parametrize("seed", range(4))
def test_time_slope_satisfies_compatibility(seed):
    """int (a u + b v + A) psi g dXi = 0 (compatibility of the Chapman-Enskog expansion)."""
    rng = np.random.default_rng(200 + seed)
    W = _rand_state(rng)
    ax = oracle.slope(W, rng.normal(size=4), GAMMA)
    ay = oracle.slope(W, rng.normal(size=4), GAMMA)
    A = oracle.time_slope(W, ax, ay, GAMMA)
    rho, U, V, lam = state_of(W, K2D)

    def pol(c, u, v, s):
        return c[0] + c[1] * u + c[2] * v + c[3] * 0.5 * (u * u + v * v + s)
    for k in range(4):
        val = expect(lambda u, v, s: (pol(ax, u, v, s) * u + pol(ay, u, v, s) * v + pol(A, u, v, s))
                     * psi(k, u, v, s), rho, U, V, lam, K2D)
        scale = expect(lambda u, v, s: np.abs(pol(ax, u, v, s) * u * psi(k, u, v, s)), rho, U, V, lam, K2D)
        assert abs(val) < 1e-10 * max(1.0, scale)


@pytest.mark.parametrize("tau,t", [(0.3, 0.1), (0.05, 0.7), (2.0, 0.4), (0.01, 0.02)])
def test_distribution_coefficients_solve_integral_solution(tau, t):
    """Closed-form f(0,t) against direct time quadrature of Eq. (eq:integral_f).

    Scalar model: along the characteristic x' = -u(t - t') the equilibrium is
    g0 (1 - s0 (t - t') + A0 t') with s0 = a0 u + b0 v, and the initial
    distribution of the upwind side is gl (1 - sl t - tau (sl + Al)).
    """
    rng = np.random.default_rng(int(1000 * tau + 10 * t))
    s0, A0, sl, Al = rng.normal(size=4)
    g0, gl = 1.0, 1.3

    def integrand(tp):
        return g0 * (1.0 - s0 * (t - tp) + A0 * tp) * math.exp(-(t - tp) / tau) / tau
    first, _ = integrate.quad(integrand, 0.0, t, epsabs=1e-15, epsrel=1e-13)
    ref = first + math.exp(-t / tau) * gl * (1.0 - sl * t - tau * (sl + Al))
    c = oracle.fdist_coeffs(tau, t)
    got = c[0] * g0 + c[1] * s0 * g0 + c[2] * A0 * g0 + c[3] * gl + c[4] * sl * gl + c[5] * Al * gl
    assert got == pytest.approx(ref, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("tau,delta", [(0.3, 0.1), (0.05, 0.7), (5.0, 0.01), (1e-3, 0.5)])
def test_time_integrals_match_quadrature(tau, delta):
    C = oracle.time_integrals(tau, delta)
    for k in range(6):
        ref, _ = integrate.quad(lambda t: oracle.fdist_coeffs(tau, t)[k] if t > 0 else
                                [0.0, 0.0, 0.0, 1.0, -tau, -tau][k], 0.0, delta, epsabs=1e-15, epsrel=1e-12,
                                limit=200)
        assert C[k] == pytest.approx(ref, rel=1e-9, abs=1e-15)


def test_time_integrals_collisionless_limit():
    """tau = 0: f = g0 (1 + A0 t), so C = (delta, 0, delta^2/2, 0, 0, 0)."""
    C = oracle.time_integrals(0.0, 0.3)
    assert np.allclose(C, [0.3, 0.0, 0.045, 0.0, 0.0, 0.0], rtol=0, atol=1e-16)


def _euler_flux(W, normal):
    rho, mu_, mv_, E = W
    U, V = mu_ / rho, mv_ / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * (U * U + V * V))
    un = U if normal == 0 else V
    F = np.array([rho * un, mu_ * un, mv_ * un, (E + p) * un])
    F[1 + normal] += p
    return F


@pytest.mark.parametrize("normal", [0, 1])
@pytest.mark.parametrize("c1", [0.0, 0.05])
def test_uniform_state_gives_euler_flux(normal, c1):
    """W^l = W^r, zero slopes: the interface flux is the Euler flux, steady, W^ = W."""
    W = np.array([1.2, 0.5, -0.3, 2.9])
    p = oracle.make_params(8, 8, tau_c1=c1, tau_c2=1.0)
    z = np.zeros(4)
    o = oracle.iface_solve(p, normal, 0.01, W, W, z, z, z)
    np.testing.assert_allclose(o["Fh"], _euler_flux(W, normal), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(o["Fht"], 0.0, atol=1e-12)
    for k in ("Whl", "Whr"):
        np.testing.assert_allclose(o[k], W, rtol=1e-13)
    for k in ("Whlt", "Whrt"):
        np.testing.assert_allclose(o[k], 0.0, atol=1e-12)


@pytest.mark.parametrize("normal", [0, 1])
@pytest.mark.parametrize("mu,Pr,c1", [(0.0, 1.0, 0.05), (0.02, 0.73, 0.0), (0.01, 1.0, 0.02)])
def test_smooth_interface_reduces_to_nodal_flux(normal, mu, Pr, c1):
    """Equal left/right states and slopes: the discontinuous solution becomes
    g0 (1 - tau(a u + b v + A) + t A), i.e. the nodal formula of Sec. 2.1."""
    rng = np.random.default_rng(7 + normal)
    W = _rand_state(rng)
    Wx, Wy = 0.1 * rng.normal(size=4), 0.1 * rng.normal(size=4)
    p = oracle.make_params(8, 8, mu=mu, Pr=Pr, tau_c1=c1, tau_c2=1.0)
    dt = 0.01
    Wn, Wt = (Wx, Wy) if normal == 0 else (Wy, Wx)
    o = oracle.iface_solve(p, normal, dt, W, W, Wn, Wn, Wt)
    nd = oracle.nodal_flux(p, dt, W, Wx, Wy)
    F, Ft = (nd["F"], nd["Ft"]) if normal == 0 else (nd["G"], nd["Gt"])
    np.testing.assert_allclose(o["Fh"], F, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(o["Fht"], Ft, rtol=1e-8, atol=1e-10)


def test_nodal_flux_shear_stress():
    """Navier-Stokes limit: with tau = mu/p, a pure shear dV/dx = s at rest
    gives the viscous flux -mu s in the y-momentum and -mu s V in the energy."""
    rho, p, V0, s, mu = 1.1, 0.9, 0.4, 0.3, 0.02
    W = np.array([rho, 0.0, rho * V0, p / (GAMMA - 1) + 0.5 * rho * V0 * V0])
    Wx = np.array([0.0, 0.0, rho * s, rho * V0 * s])
    prm = oracle.make_params(8, 8, mu=mu, Pr=0.73)
    o = oracle.nodal_flux(prm, 0.01, W, Wx, np.zeros(4))
    np.testing.assert_allclose(o["F"], [0.0, p, -mu * s, -mu * s * V0], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("Pr", [1.0, 0.72])
def test_nodal_flux_fourier_heat_flux(Pr):
    """Navier-Stokes limit: gas at rest with uniform pressure and a density
    gradient conducts heat q = -(mu/Pr) c_p dT/dx, T = p/rho, c_p = gamma/(gamma-1)."""
    rho, p, drho, mu = 1.3, 0.8, 0.25, 0.03
    W = np.array([rho, 0.0, 0.0, p / (GAMMA - 1)])
    Wx = np.array([drho, 0.0, 0.0, 0.0])
    prm = oracle.make_params(8, 8, mu=mu, Pr=Pr)
    o = oracle.nodal_flux(prm, 0.01, W, Wx, np.zeros(4))
    dT = -p * drho / rho ** 2
    q = -(mu / Pr) * GAMMA / (GAMMA - 1) * dT
    np.testing.assert_allclose(o["F"], [0.0, p, 0.0, q], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(o["G"], [0.0, 0.0, p, 0.0], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("Ux,Vy", [(0.3, 0.0), (0.3, 0.3), (0.25, -0.4)])
def test_nodal_flux_normal_stresses(Ux, Vy):
    """Navier-Stokes limit of the BGK gas with N = K + 2 degrees of freedom
    (Chapman-Enskog): with tau = mu/p, uniform density and pressure and a
    velocity field (U0 + Ux x, V0 + Vy y), the viscous stresses are
    sigma_xx = mu (2 Ux - (2/N) div U), sigma_yy = mu (2 Vy - (2/N) div U),
    sigma_xy = 0; the energy fluxes carry the work U0 sigma_xx, V0 sigma_yy
    and no heat flux (the temperature is uniform), whatever Pr."""
    rho, p, U0, V0, mu = 1.2, 0.85, 0.4, -0.3, 0.025
    N = K2D + 2.0
    E = p / (GAMMA - 1) + 0.5 * rho * (U0 * U0 + V0 * V0)
    W = np.array([rho, rho * U0, rho * V0, E])
    Wx = np.array([0.0, rho * Ux, 0.0, rho * U0 * Ux])
    Wy = np.array([0.0, 0.0, rho * Vy, rho * V0 * Vy])
    prm = oracle.make_params(8, 8, mu=mu, Pr=0.73)
    o = oracle.nodal_flux(prm, 0.01, W, Wx, Wy)
    div = Ux + Vy
    sxx = mu * (2.0 * Ux - 2.0 / N * div)
    syy = mu * (2.0 * Vy - 2.0 / N * div)
    F = [rho * U0, rho * U0 * U0 + p - sxx, rho * U0 * V0, U0 * (E + p) - U0 * sxx]
    G = [rho * V0, rho * U0 * V0, rho * V0 * V0 + p - syy, V0 * (E + p) - V0 * syy]
    np.testing.assert_allclose(o["F"], F, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(o["G"], G, rtol=1e-12, atol=1e-14)
