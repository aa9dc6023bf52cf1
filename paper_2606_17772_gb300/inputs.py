"""Seeded synthetic inputs for FD-CGKS runs (initial data only).

This module holds no arithmetic of the scheme.  It evaluates analytic initial
conditions at the node positions of the primary and dual grids and forms the
initial averaged gradients as the exact mean derivative over each node's
interval, (W(x + h/2) - W(x - h/2)) / h (the definition of the averaged
gradient, Sec. 2.3 of the paper, applied to the exact initial field).  The
CUDA path and the CPU oracle both take their inputs from here.

Workloads (paper Sec. 5 and the throughput workloads):
  * density wave (Sec. 5.1): rho = 1 + 0.2 sin(pi (x + y)), U = V = 1, p = 1 on
    [0, 2]^2 periodic; its 1-D form on a y-periodic strip;
  * Sod and Lax tubes (Sec. 5.2) on a y-periodic strip with transmissive x ends;
  * isentropic vortex on [0, 10]^2 periodic (standard closed form, strength 5);
  * viscous shock tube (Sec. 5.8) on [0, 1] x [0, 0.5] with walls/symmetry;
  * Woodward-Colella blast waves (Sec. 5.3) between reflecting walls;
  * double Mach reflection (Sec. 5.5) on [0, 4] x [0, 1] with inflow, outflow,
    a wall from x = 1/6 and a top boundary following the exact Mach 10 shock;
  * a seeded random smooth perturbation used by the parity tests.

Node placement: primary nodes at cell centres x0 + (i + 1/2) h, dual nodes at
x0 + i h; a bounded direction carries n + 1 dual nodes (on both boundaries).
"""
import math
from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC, BC_TRANSMISSIVE, BC_SYMMETRY, BC_NOSLIP, BC_FIXED = 0, 1, 2, 3, 4


@dataclass
class Case:
    """A workload: grid, gas constants, boundary conditions and initial data."""
    name: str
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    bc: tuple
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 1.0
    tau_c1: float = 0.0
    tau_c2: float = 0.0
    flux_variant: int = 64
    geno_variant: int = 0
    grad_base: int = 0
    recon_vars: int = 0          # 0 conservative, 1 characteristic components
    prim: object = None          # callable (x, y) -> (rho, U, V, p) arrays
    sides: object = None         # None, or 4 split-side dicts (kind, split0, split_speed, prim)
    extra: dict = field(default_factory=dict)

    @property
    def nxd(self):
        return self.nx + (0 if self.bc[0] == BC_PERIODIC else 1)

    @property
    def nyd(self):
        return self.ny + (0 if self.bc[2] == BC_PERIODIC else 1)

    @property
    def hx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self):
        return (self.y1 - self.y0) / self.ny

    def node_xy(self, dual):
        """Node coordinates (X, Y) arrays of shape (ny, nx) for one grid."""
        if dual:
            i = np.arange(self.nxd, dtype=np.float64)
            j = np.arange(self.nyd, dtype=np.float64)
            xs = self.x0 + (self.x1 - self.x0) * i / self.nx
            ys = self.y0 + (self.y1 - self.y0) * j / self.ny
        else:
            i = np.arange(self.nx, dtype=np.float64)
            j = np.arange(self.ny, dtype=np.float64)
            xs = self.x0 + (self.x1 - self.x0) * (2 * i + 1) / (2 * self.nx)
            ys = self.y0 + (self.y1 - self.y0) * (2 * j + 1) / (2 * self.ny)
        return np.meshgrid(xs, ys)

    def conservative(self, x, y):
        rho, U, V, p = self.prim(x, y)
        rho = np.broadcast_to(rho, np.shape(x)).astype(np.float64)
        U = np.broadcast_to(U, np.shape(x)).astype(np.float64)
        V = np.broadcast_to(V, np.shape(x)).astype(np.float64)
        p = np.broadcast_to(p, np.shape(x)).astype(np.float64)
        return np.stack([rho, rho * U, rho * V, p / (self.gamma - 1.0) + 0.5 * rho * (U * U + V * V)])

    def initial_state(self):
        """(Wp [4,ny,nx], Gp [2,4,ny,nx], Wd [4,nyd,nxd], Gd [2,4,nyd,nxd]) float64."""
        out = []
        for dual in (False, True):
            X, Y = self.node_xy(dual)
            W = self.conservative(X, Y)
            gx = (self.conservative(X + 0.5 * self.hx, Y) - self.conservative(X - 0.5 * self.hx, Y)) / self.hx
            gy = (self.conservative(X, Y + 0.5 * self.hy) - self.conservative(X, Y - 0.5 * self.hy)) / self.hy
            out += [np.ascontiguousarray(W), np.ascontiguousarray(np.stack([gx, gy]))]
        return tuple(out)

    def oracle_kwargs(self):
        return dict(nx=self.nx, ny=self.ny, x0=self.x0, x1=self.x1, y0=self.y0, y1=self.y1,
                    gamma=self.gamma, mu=self.mu, Pr=self.Pr, bc=tuple(self.bc),
                    flux_variant=self.flux_variant, geno_variant=self.geno_variant,
                    grad_base=self.grad_base, tau_c1=self.tau_c1, tau_c2=self.tau_c2,
                    recon_vars=self.recon_vars, sides=self.sides)


def line_state(case):
    """Initial data of the one-dimensional scheme (Sec. 2) from a strip case:
    (W [3][n], Wx [3][n]), the first primary row's (rho, rho U, rho E) and
    their averaged x-gradients."""
    Wp, Gp, _, _ = case.initial_state()
    idx = [0, 1, 3]
    return np.ascontiguousarray(Wp[idx, 0, :]), np.ascontiguousarray(Gp[0][idx][:, 0, :])


# ---------------------------------------------------------------------------
# analytic initial conditions
# ---------------------------------------------------------------------------

def density_wave_2d(n, t=0.0, **kw):
    """Sec. 5.1, 2-D: rho = 1 + 0.2 sin(pi(x + y - 2t)), U = V = 1, p = 1 on [0,2]^2."""
    def prim(x, y):
        return 1.0 + 0.2 * np.sin(np.pi * (x + y - 2.0 * t)), 1.0, 1.0, 1.0
    kw.setdefault("flux_variant", 62)
    return Case("density_wave_2d", n, n, 0.0, 2.0, 0.0, 2.0, (0, 0, 0, 0), prim=prim, **kw)


def density_wave_1d(n, ny=1, t=0.0, **kw):
    """Sec. 5.1, 1-D on a y-periodic strip: rho = 1 + 0.2 sin(pi(x - t)), U = 1, V = 0, p = 1."""
    h = 2.0 / n

    def prim(x, y):
        return 1.0 + 0.2 * np.sin(np.pi * (x - t)), 1.0, 0.0, 1.0
    kw.setdefault("flux_variant", 62)
    return Case("density_wave_1d", n, ny, 0.0, 2.0, 0.0, ny * h, (0, 0, 0, 0), prim=prim, **kw)


def vortex(n, strength=5.0, xc=5.0, yc=5.0, t=0.0, L=10.0, gamma=1.4, images=0, **kw):
    """Isentropic vortex on [0, L]^2 periodic, free stream (1, 1, 1, 1), advected to time t.

    Standard closed form: with (xb, yb) the minimum-image offset from the
    centre (xc + t, yc + t), r^2 = xb^2 + yb^2,
      dU = -(eps/2pi) e^{(1-r^2)/2} yb,  dV = (eps/2pi) e^{(1-r^2)/2} xb,
      T = 1 - (gamma-1) eps^2 / (8 gamma pi^2) e^{1-r^2},  rho = T^{1/(gamma-1)},  p = rho T.

    The minimum-image field is continuous across the box edges but its
    derivative jumps there by the vortex's tail (about 1e-6 at strength 5 on
    [0, 10]^2), which puts a floor under the error of a long run.  images = k
    instead sums the perturbations dU, dV and the temperature deficit of the
    vortices centred at the (2k + 1)^2 periodic images (offsets -k..k boxes in
    each direction), a smooth periodic field; images = 1 already drops every
    neglected image below e^{-80}.  Superposing vortices is exact only up to
    products of their perturbations, about 1e-10 where two tails meet.

    GENO constants default to App. D's (variant 1): with the Sec. 3.2 text's
    constants the vortex's error stays near 5e-4 from 128^2 to 1024^2 (t = 10),
    with App. D's it converges (1.1e-8 at 512^2), and both reproduce the
    paper's Tables 1 and 2.  Long runs need CFL 0.2 (per-direction
    definition): at 0.4 the scheme's grid-scale diagonal modes grow.
    """
    eps = strength

    def prim(x, y):
        x0 = np.mod(x - (xc + t) + 0.5 * L, L) - 0.5 * L
        y0 = np.mod(y - (yc + t) + 0.5 * L, L) - 0.5 * L
        du = dv = dT = 0.0
        for kx in range(-images, images + 1):
            for ky in range(-images, images + 1):
                xb, yb = x0 - kx * L, y0 - ky * L
                r2 = xb * xb + yb * yb
                e = np.exp(0.5 * (1.0 - r2))
                du = du - eps / (2 * math.pi) * e * yb
                dv = dv + eps / (2 * math.pi) * e * xb
                dT = dT + (gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
        T = 1.0 - dT
        rho = T ** (1.0 / (gamma - 1.0))
        return rho, 1.0 + du, 1.0 + dv, rho * T
    kw.setdefault("tau_c2", 1.0)
    kw.setdefault("geno_variant", 1)
    return Case("vortex", n, n, 0.0, L, 0.0, L, (0, 0, 0, 0), gamma=gamma, prim=prim,
                extra=dict(strength=strength, xc=xc, yc=yc, images=images), **kw)


def sod_strip(nx=200, ny=4, **kw):
    """Sec. 5.2 Sod tube on [0,1], y-periodic strip of ny rows, transmissive x ends.

    (rho, U, p) = (1, 0, 1) for x < 0.5 and (0.125, 0, 0.1) for x >= 0.5.
    """
    h = 1.0 / nx

    def prim(x, y):
        right = x >= 0.5
        return np.where(right, 0.125, 1.0), 0.0, 0.0, np.where(right, 0.1, 1.0)
    kw.setdefault("tau_c1", 0.05)
    kw.setdefault("tau_c2", 1.0)
    return Case("sod_strip", nx, ny, 0.0, 1.0, 0.0, ny * h, (1, 1, 0, 0), prim=prim, **kw)


def lax_strip(nx=100, ny=1, **kw):
    """Sec. 5.2 Lax tube on [0,1], y-periodic strip of ny rows, transmissive x ends:
    (rho, U, p) = (0.445, 0.698, 3.528) for x < 0.5 and (0.5, 0, 0.571) for x >= 0.5;
    final time 0.16."""
    h = 1.0 / nx

    def prim(x, y):
        right = x >= 0.5
        return (np.where(right, 0.5, 0.445), np.where(right, 0.0, 0.698), 0.0,
                np.where(right, 0.571, 3.528))
    kw.setdefault("tau_c1", 0.05)
    kw.setdefault("tau_c2", 1.0)
    return Case("lax_strip", nx, ny, 0.0, 1.0, 0.0, ny * h, (1, 1, 0, 0), prim=prim, **kw)


def strong_shock_strip(nx=200, ny=1, gamma=1.4, **kw):
    """1-D Riemann problem with the viscous shock tube's states (Sec. 5.8), inviscid, on a
    y-periodic strip with transmissive x ends: (rho, U, p) = (120, 0, 120/gamma) for x < 0.5
    and (1.2, 0, 1.2/gamma) for x >= 0.5 (density and pressure ratio 100)."""
    h = 1.0 / nx

    def prim(x, y):
        right = x >= 0.5
        rho = np.where(right, 1.2, 120.0)
        return rho, 0.0, 0.0, rho / gamma
    kw.setdefault("tau_c2", 1.0)
    return Case("strong_shock_strip", nx, ny, 0.0, 1.0, 0.0, ny * h, (1, 1, 0, 0), gamma=gamma, prim=prim, **kw)


def woodward_colella(nx=400, ny=1, gamma=1.4, **kw):
    """Sec. 5.3 interacting blast waves on [0, 1] between reflecting (symmetry) walls,
    a y-periodic strip of ny rows: (rho, U, p) = (1, 0, 1000) for x < 0.1, (1, 0, 0.01)
    for 0.1 <= x < 0.9, (1, 0, 100) for x >= 0.9; final time 0.038."""
    h = 1.0 / nx

    def prim(x, y):
        p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
        return 1.0, 0.0, 0.0, p
    kw.setdefault("tau_c1", 0.05)
    kw.setdefault("tau_c2", 1.0)
    return Case("woodward_colella", nx, ny, 0.0, 1.0, 0.0, ny * h, (BC_SYMMETRY, BC_SYMMETRY, 0, 0),
                gamma=gamma, prim=prim, **kw)


DMR_POST = (8.0, 4.125 * math.sqrt(3.0), -4.125, 116.5)
DMR_PRE = (1.4, 0.0, 0.0, 1.0)


def double_mach(nx=960, ny=240, **kw):
    """Sec. 5.5 double Mach reflection on [0, 4] x [0, 1], gamma 1.4, final time 0.2.

    A Mach 10 shock through (1/6, 0) at 60 degrees to the x-axis, post-shock
    (8, 4.125 sqrt 3, -4.125, 116.5) to its left, pre-shock (1.4, 0, 0, 1) to its
    right; the shock line x = 1/6 + (y + 20 t)/sqrt 3.  Sides: inflow (post-shock
    state) at x = 0, outflow (transmissive) at x = 4, outflow below x = 1/6 and a
    reflecting wall from x = 1/6 on at y = 0, and at y = 1 the exact shock's
    states, split where the shock meets y = 1 (speed 20/sqrt 3 along x).

    Collision-time constants (the paper gives none): c1 = 0.05, c2 = 25.  With
    FD-CGKS(6-2) and characteristic reconstruction these carry both of the
    paper's grids to t = 0.2 in FP64 and in mixed precision; c2 = 15 or 20
    lose positivity next to the start of the wall before t = 0.2 and c2 = 30
    in the first steps."""
    r3 = math.sqrt(3.0)

    def prim(x, y):
        post = x < 1.0 / 6.0 + y / r3
        return tuple(np.where(post, a, b) for a, b in zip(DMR_POST, DMR_PRE))
    fixed_post = dict(kind=(BC_FIXED, BC_FIXED), prim=(DMR_POST, DMR_POST))
    sides = (fixed_post,
             dict(kind=(BC_TRANSMISSIVE, BC_TRANSMISSIVE)),
             dict(kind=(BC_TRANSMISSIVE, BC_SYMMETRY), split0=1.0 / 6.0),
             dict(kind=(BC_FIXED, BC_FIXED), split0=1.0 / 6.0 + 1.0 / r3, split_speed=20.0 / r3,
                  prim=(DMR_POST, DMR_PRE)))
    kw.setdefault("tau_c1", 0.05)
    kw.setdefault("tau_c2", 25.0)
    return Case("double_mach", nx, ny, 0.0, 4.0, 0.0, 1.0,
                (BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_SYMMETRY, BC_TRANSMISSIVE), prim=prim, sides=sides, **kw)


def viscous_shock_tube(nx=1000, ny=500, gamma=1.4, mu=0.005, Pr=0.73, **kw):
    """Sec. 5.8: [0,1] x [0,0.5], diaphragm x = 0.5, (120,0,0,120/gamma) | (1.2,0,0,1.2/gamma).

    No-slip adiabatic walls left, right and bottom; symmetry at y = 0.5.
    Defaults: the Sec. 3.2 GENO constants and tau c2 = 1.  On 1000 x 500 runs
    are marginal in either precision with every constant set tried: whether
    they leave the physical states near the shock's foot (t = 0.0015 to 0.009)
    depends on rounding-level details.  geno_variant=1, tau_c2=25.0 carried
    most runs to t = 1 but leave the physical states on coarse grids (40 x 20)
    within a few steps, so they are a run option, not the default.
    """
    def prim(x, y):
        right = x >= 0.5
        rho = np.where(right, 1.2, 120.0)
        return rho, 0.0, 0.0, rho / gamma
    kw.setdefault("tau_c2", 1.0)
    return Case("viscous_shock_tube", nx, ny, 0.0, 1.0, 0.0, 0.5,
                (BC_NOSLIP, BC_NOSLIP, BC_NOSLIP, BC_SYMMETRY), gamma=gamma, mu=mu, Pr=Pr,
                prim=prim, **kw)


def random_smooth(nx, ny, seed, amp=0.05, modes=4, bc=(0, 0, 0, 0), **kw):
    """Seeded random smooth field: a free stream plus `modes` random Fourier modes per variable.

    Used by the parity tests to exercise every term with non-trivial data.
    On bounded directions the field is still smooth (the modes need not match
    the boundaries: the ghost treatment then creates weak discontinuities,
    which exercise the nonlinear weights too).
    """
    rng = np.random.default_rng(seed)
    Lx, Ly = 1.0, ny / nx
    k = rng.integers(1, 4, size=(4, modes, 2))
    ph = rng.uniform(0, 2 * math.pi, size=(4, modes))
    a = rng.uniform(-amp, amp, size=(4, modes))
    base = np.array([1.0, 0.6, -0.4, 1.0])

    def prim(x, y):
        out = []
        for v in range(4):
            f = np.full(np.shape(x), base[v])
            for m in range(modes):
                f = f + a[v, m] * np.sin(2 * math.pi * (k[v, m, 0] * x / Lx + k[v, m, 1] * y / Ly) + ph[v, m])
            out.append(f)
        return tuple(out)
    return Case("random_smooth", nx, ny, 0.0, Lx, 0.0, Ly, tuple(bc), prim=prim, extra=dict(seed=seed), **kw)


def ensemble_members(count=256, seed=0, nmin=32, nmax=512, L=10.0):
    """Seeded ensemble of periodic isentropic vortices on uneven grids.

    Grid sizes log-uniform in [nmin, nmax] (rounded), strength uniform in
    [1, 5], centre uniform in the domain.  Returns a list of Case objects.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        eps = rng.uniform(1.0, 5.0)
        xc, yc = rng.uniform(0.0, L, size=2)
        out.append(vortex(n, strength=eps, xc=xc, yc=yc, L=L))
    return out
