"""Pins of the oracle's compact reconstruction, GENO weights and compact flux
(paper Sec. 2.1-2.2, Sec. 3, App. C, App. D).

Exactness is checked on polynomial data built here from point values and
exact interval-averaged derivatives; the compact-flux error constant is the
paper's printed 1/8960 (tests/golden/compact_flux_error_constant.txt).
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _poly_data(coef, h, offsets):
    """Point values at node offsets (node k at (k - 1/2) h from the interface at 0)
    and averaged derivatives over [x_k - h/2, x_k + h/2]."""
    P = np.polynomial.Polynomial(coef)
    xs = np.array([(k - 0.5) * h for k in offsets])
    Q = P(xs)
    Qx = (P(xs + h / 2) - P(xs - h / 2)) / h
    return P, Q, Qx


@pytest.mark.parametrize("deg", range(7))
@pytest.mark.parametrize("h", [0.5, 0.1])
def test_interface_reconstruction_exact_to_degree_6(deg, h):
    rng = np.random.default_rng(deg)
    coef = rng.normal(size=deg + 1)
    P, Q, Qx = _poly_data(coef, h, (-1, 0, 1, 2))
    l = oracle.recon_left(2, Q, Qx[:3], h)
    r = oracle.recon_right(2, Q, Qx[1:], h)
    scale = np.abs(coef).sum()
    for out in (l, r):
        assert out[0] == pytest.approx(P(0.0), abs=1e-12 * scale)
        assert out[1] == pytest.approx(P.deriv()(0.0), abs=1e-11 * scale / h)
        assert out[2] == 1.0


def test_interface_reconstruction_not_exact_at_degree_7():
    h = 0.5
    P, Q, Qx = _poly_data([0, 0, 0, 0, 0, 0, 0, 1.0], h, (-1, 0, 1, 2))
    l = oracle.recon_left(2, Q, Qx[:3], h)
    assert abs(l[0] - P(0.0)) > 1e-8


@pytest.mark.parametrize("deg", range(7))
def test_node_derivative_exact_to_degree_6(deg):
    h = 0.3
    rng = np.random.default_rng(50 + deg)
    coef = rng.normal(size=deg + 1)
    P, Q, Qx = _poly_data(coef, h, (-1, 0, 1))
    out = oracle.recon_node(2, Q, Qx, h)
    # node j sits at -h/2 in these coordinates
    assert out[0] == pytest.approx(P.deriv()(-0.5 * h), abs=1e-11 * np.abs(coef).sum() / h)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_geno_is_linear_on_quadratics(variant, seed):
    """For quadratic data every sub-stencil reproduces the same quadratic, so
    all IS_k are equal, IS^tau = 0 and chi = 1: GENO returns the linear P^H."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.05, 0.5)
    coef = rng.normal(size=3)
    P, Q, Qx = _poly_data(coef, h, (-1, 0, 1, 2))
    for fn, gx in ((oracle.recon_left, Qx[:3]), (oracle.recon_right, Qx[1:])):
        g = fn(variant, Q, gx, h)
        lin = fn(2, Q, gx, h)
        assert g[2] == 1.0
        assert g[0] == pytest.approx(lin[0], rel=1e-14, abs=1e-14)
        assert g[0] == pytest.approx(P(0.0), rel=1e-13, abs=1e-13)
    _, Qn, Qxn = _poly_data(coef, h, (-1, 0, 1))
    n = oracle.recon_node(variant, Qn, Qxn, h)
    assert n[1] == 1.0
    assert n[0] == pytest.approx(P.deriv()(-0.5 * h), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("jump_at", [0, 1, 2])
def test_geno_does_not_create_extrema_at_a_step(variant, jump_at):
    """Step data: chi -> 0 and the reconstructed interface states stay within
    the data range (essentially non-oscillatory)."""
    h = 0.1
    Q = np.array([0.0, 0.0, 0.0, 0.0])
    Q[jump_at + 1:] = 1.0
    Qx = np.zeros(4)
    Qx[jump_at] = 1.0 / h      # averaged derivative of the cell holding the jump
    for fn, gx in ((oracle.recon_left, Qx[:3]), (oracle.recon_right, Qx[1:])):
        v, d, chi = fn(variant, Q, gx, h)
        assert chi < 1e-6
        assert -1e-6 <= v <= 1.0 + 1e-6


@pytest.mark.parametrize("variant,expect_weights", [(0, (8.0, 1.0, 1.0)), (1, (1.0, 8.0, 1.0))])
def test_geno_ideal_weights_placement(variant, expect_weights):
    """With equal IS_k and chi forced to 0 by IS^tau, P^L = sum d_k q_k / sum d_k:
    variant 0 (Sec. 3.2 text) puts d = 8 on the first interface sub-stencil,
    variant 1 (App. D) on the central one."""
    q = np.array([1.0, 2.0, 4.0])
    # IS = (1, 0, 0) gives IS^tau = 1 >> IS^L + eps: chi ~ 0; the weights then
    # favour the two zero-IS stencils equally, and the d ratio decides between them.
    IS = np.array([1.0, 0.0, 0.0])
    v, d, chi = oracle.geno_blend(variant, 0, IS, q, q, 0.0, 0.0)
    assert chi < 1e-10
    w = np.array(expect_weights) / np.array([1.0 + 1e-6, 1e-6, 1e-6]) ** 2
    assert v == pytest.approx(float(np.dot(w, q) / w.sum()), rel=1e-9)


def _sliding_averages(P, h):
    """Nodal fluxes (averages over [x_k - h/2, x_k + h/2]) at nodes j, j+1 and
    interface fluxes (averages over [x_i - h, x_i]... between adjacent nodes)
    at j-1/2, j+1/2, j+3/2, for the interface j+1/2 at 0 (Eq. fd-conservative-flux-recons)."""
    I = P.integ()

    def avg(a, b):
        return (I(b) - I(a)) / (b - a)
    nodes = [-0.5 * h, 0.5 * h]
    Fn = np.array([avg(x - h / 2, x + h / 2) for x in nodes])
    ifs = [-h, 0.0, h]
    Fi = np.array([avg(x - h / 2, x + h / 2) for x in ifs])
    return Fi, Fn


@pytest.mark.parametrize("deg", range(6))
def test_compact_flux_exact_to_degree_5(deg):
    h = 0.4
    coef = np.random.default_rng(deg).normal(size=deg + 1)
    P = np.polynomial.Polynomial(coef)
    Fi, Fn = _sliding_averages(P, h)
    assert oracle.compact_flux(64, 1.0, Fi, Fn) == pytest.approx(P(0.0), abs=1e-13 * np.abs(coef).sum())


def test_compact_flux_error_constant_is_paper_value():
    const = float(open(os.path.join(GOLD, "compact_flux_error_constant.txt")).read().split()[-1])
    h = 0.25
    P = np.polynomial.Polynomial([0, 0, 0, 0, 0, 0, 1.0])     # x^6, sixth derivative 720
    Fi, Fn = _sliding_averages(P, h)
    err = oracle.compact_flux(64, 1.0, Fi, Fn) - P(0.0)
    assert err == pytest.approx(h ** 6 * 720.0 / const, rel=1e-10)


@pytest.mark.parametrize("deg", range(4))
def test_fourth_order_fallback_flux_exact_to_degree_3(deg):
    """FD-CGKS(6-4) low-order flux (8 F_{j+1/2} - F_j - F_{j+1}) / 6 (with 1/6)."""
    h = 0.4
    coef = np.random.default_rng(20 + deg).normal(size=deg + 1)
    P = np.polynomial.Polynomial(coef)
    Fi, Fn = _sliding_averages(P, h)
    assert oracle.compact_flux(64, 0.0, Fi, Fn) == pytest.approx(P(0.0), abs=1e-13 * np.abs(coef).sum())


def test_second_order_fallback_is_interface_flux():
    Fi, Fn = np.array([1.0, 2.5, 7.0]), np.array([3.0, 4.0])
    assert oracle.compact_flux(62, 0.0, Fi, Fn) == 2.5


# ---------------------------------------------------------------------------
# characteristic components (recon_vars = 1)
# ---------------------------------------------------------------------------
def _euler_flux(W, normal, gamma=1.4):
    """Textbook Euler flux along x (normal 0) or y (normal 1) of W = (rho, rho U, rho V, rho E)."""
    rho, mx, my, E = W
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    un = u if normal == 0 else v
    return np.array([rho * un, mx * un + (p if normal == 0 else 0.0), my * un + (p if normal == 1 else 0.0),
                      (E + p) * un])


@pytest.mark.parametrize("normal", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_characteristic_basis_diagonalises_the_flux_jacobian(normal, seed):
    """L R = I and R diag(u_n - c, u_n, u_n, u_n + c) L = dF_n/dW at the mean state,
    with the Jacobian taken by central differences of the Euler flux."""
    rng = np.random.default_rng(seed)
    g = 1.4

    def state():
        rho, u, v, p = rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.3, 2)
        return np.array([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)])
    Wa, Wb = state(), state()
    L, R = oracle.char_basis(g, normal, Wa, Wb)
    W = 0.5 * (Wa + Wb)
    perm = [0, 1, 2, 3] if normal == 0 else [0, 2, 1, 3]       # (rho, m_n, m_t, E) order
    P = np.eye(4)[perm]                                          # W_perm = P W
    assert np.allclose(L @ R, np.eye(4), atol=1e-13)
    A = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = 1e-6 * max(1.0, abs(W[k]))
        A[:, k] = (_euler_flux(W + e, normal) - _euler_flux(W - e, normal)) / (2 * e[k])
    rho, u, v = W[0], W[1] / W[0], W[2] / W[0]
    p = (g - 1) * (W[3] - 0.5 * rho * (u * u + v * v))
    c, un = np.sqrt(g * p / rho), (u if normal == 0 else v)
    lam = np.diag([un - c, un, un, un + c])
    assert np.allclose(P.T @ R @ lam @ L @ P, A, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("normal", [0, 1])
def test_characteristic_reconstruction_equals_conservative_when_linear(normal):
    """With the linear reconstruction (GENO variant 2) both are linear maps and the
    projection is fixed per line, so characteristic and conservative
    reconstruction agree to rounding on any data."""
    rng = np.random.default_rng(5)
    g = 1.4
    for _ in range(20):
        rho = rng.uniform(0.5, 2, 4)
        u, v, p = rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4), rng.uniform(0.3, 2, 4)
        Q = np.stack([rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)], 1)   # [entry][field]
        Qx = rng.normal(size=(4, 4))
        a = oracle.recon_line(2, 1, g, normal, Q, Qx, 0.1)
        b = oracle.recon_line(2, 0, g, normal, Q, Qx, 0.1)
        for x, y in zip(a[:4], b[:4]):
            assert np.allclose(x, y, rtol=1e-12, atol=1e-12)


def test_characteristic_reconstruction_exact_to_degree_6():
    """Polynomial data of degree 6 in every conservative variable, smooth enough that
    GENO keeps the high-order stencil: the characteristic reconstruction is exact."""
    g, h = 1.4, 0.05
    x = np.array([-1.5, -0.5, 0.5, 1.5]) * h                     # entries around the interface at 0
    base = np.array([1.0, 0.3, -0.2, 2.5])
    cf = np.array([0.02, -0.01, 0.015, 0.03])

    def f(t):
        return base + cf * (t + t ** 2 + t ** 3 + t ** 4 + t ** 5 + t ** 6)

    Q = np.array([f(t) for t in x])
    Qx = np.array([(f(t + h / 2) - f(t - h / 2)) / h for t in x])     # exact averaged gradients
    Wl, Wr, Wlx, Wrx, chi = oracle.recon_line(0, 1, g, 0, Q, Qx, h)
    assert chi == pytest.approx(1.0)
    assert np.allclose(Wl, f(0.0), atol=1e-12) and np.allclose(Wr, f(0.0), atol=1e-12)
