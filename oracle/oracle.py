"""ctypes wrapper around the C++ FD-CGKS oracle (test infrastructure only).

Array layouts (all float64, C order):
  W     [4][ny][nx]      conservative (rho, rho U, rho V, rho E) at the nodes
  grad  [2][4][ny][nx]   averaged gradients (x first, then y)
Dual-grid arrays use (nyd, nxd) from :func:`dual_dims`.
"""
import ctypes
import numpy as np

from .build import build_oracle

BC_PERIODIC, BC_TRANSMISSIVE, BC_SYMMETRY, BC_NOSLIP, BC_FIXED = 0, 1, 2, 3, 4


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("flux_variant", ctypes.c_int),
        ("geno_variant", ctypes.c_int),
        ("grad_base", ctypes.c_int),
        ("tau_c1", ctypes.c_double), ("tau_c2", ctypes.c_double),
        ("recon_vars", ctypes.c_int),
        ("has_sides", ctypes.c_int),
        ("side_kind", (ctypes.c_int * 2) * 4),
        ("side_split0", ctypes.c_double * 4), ("side_speed", ctypes.c_double * 4),
        ("side_prim", ((ctypes.c_double * 4) * 2) * 4),
        ("t0", ctypes.c_double),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        _lib.oracle_cfl_dt.restype = ctypes.c_double
        _lib.oracle_maxwell_moment.restype = ctypes.c_double
        _lib.oracle_compact_flux.restype = ctypes.c_double
        _lib.oracle_cfl_dt_1d.restype = ctypes.c_double
        _lib.oracle_cfl_dt_sum.restype = ctypes.c_double
    return _lib


def make_params(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, mu=0.0, Pr=1.0,
                bc=(0, 0, 0, 0), flux_variant=64, geno_variant=0, grad_base=0,
                tau_c1=0.0, tau_c2=0.0, recon_vars=0, sides=None, t0=0.0):
    """sides: None, or 4 dicts (x-low, x-high, y-low, y-high) with keys kind
    (2 boundary kinds), split0, split_speed and prim (2 x (rho, U, V, p)); t0:
    the time of the first step (moving split points)."""
    p = OracleParams()
    p.nx, p.ny = nx, ny
    p.x0, p.x1, p.y0, p.y1 = x0, x1, y0, y1
    p.gamma, p.mu, p.Pr = gamma, mu, Pr
    for k in range(4):
        p.bc[k] = bc[k]
    p.flux_variant, p.geno_variant, p.grad_base = flux_variant, geno_variant, grad_base
    p.tau_c1, p.tau_c2 = tau_c1, tau_c2
    p.recon_vars = recon_vars
    p.has_sides = int(sides is not None)
    for k, sd in enumerate(sides or ()):
        p.side_kind[k][0], p.side_kind[k][1] = sd["kind"]
        p.side_split0[k] = sd.get("split0", 0.0)
        p.side_speed[k] = sd.get("split_speed", 0.0)
        for q, prim in enumerate(sd.get("prim", ((0.0,) * 4,) * 2)):
            for j in range(4):
                p.side_prim[k][q][j] = prim[j]
    p.t0 = t0
    return p


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


def dual_dims(p):
    nxd, nyd = ctypes.c_int(), ctypes.c_int()
    if lib().oracle_dims(ctypes.byref(p), ctypes.byref(nxd), ctypes.byref(nyd)) != 0:
        raise ValueError("invalid oracle parameters")
    return nxd.value, nyd.value


def steps(p, dt, nsteps, Wp, Gp, Wd, Gd):
    """Advance ``nsteps`` S2O4 steps; returns new (Wp, Gp, Wd, Gd) arrays."""
    nxd, nyd = dual_dims(p)
    Wp = _arr(Wp, 4 * p.nx * p.ny).copy().reshape(4, p.ny, p.nx)
    Gp = _arr(Gp, 8 * p.nx * p.ny).copy().reshape(2, 4, p.ny, p.nx)
    Wd = _arr(Wd, 4 * nxd * nyd).copy().reshape(4, nyd, nxd)
    Gd = _arr(Gd, 8 * nxd * nyd).copy().reshape(2, 4, nyd, nxd)
    rc = lib().oracle_steps(ctypes.byref(p), ctypes.c_double(dt), ctypes.c_int(nsteps),
                            _ptr(Wp), _ptr(Gp), _ptr(Wd), _ptr(Gd))
    if rc != 0:
        raise ValueError("oracle_steps failed")
    return Wp, Gp, Wd, Gd


def steps_1d(p, dt, nsteps, W, Gx):
    """The one-dimensional scheme (Sec. 2): ``nsteps`` S2O4 steps of the line of
    p.nx nodes (bc[0], bc[1] at its ends); W, Gx: [3][n] (rho, rho U, rho E) and
    their averaged gradients.  Returns new arrays."""
    n = p.nx
    W = _arr(W, 3 * n).copy().reshape(3, n)
    Gx = _arr(Gx, 3 * n).copy().reshape(3, n)
    if lib().oracle_steps_1d(ctypes.byref(p), ctypes.c_double(dt), ctypes.c_int(nsteps), _ptr(W), _ptr(Gx)) != 0:
        raise ValueError("oracle_steps_1d failed")
    return W, Gx


def stage_1d(p, dt, W, Gx):
    """One stage's operator of the line: dict L, Lt, gb, gt ([3][n] each)."""
    n = p.nx
    out = {k: np.zeros((3, n)) for k in ("L", "Lt", "gb", "gt")}
    rc = lib().oracle_stage_1d(ctypes.byref(p), ctypes.c_double(dt), _ptr(_arr(W, 3 * n)), _ptr(_arr(Gx, 3 * n)),
                               *(_ptr(out[k]) for k in ("L", "Lt", "gb", "gt")))
    if rc != 0:
        raise ValueError("oracle_stage_1d failed")
    return out


def cfl_dt_sum(p, cfl, Wp, Wd):
    """The two-dimensional form of the CFL bound (rates of the directions added)."""
    return lib().oracle_cfl_dt_sum(ctypes.byref(p), ctypes.c_double(cfl), _ptr(_arr(Wp)), _ptr(_arr(Wd)))


def cfl_dt_1d(p, cfl, W):
    return lib().oracle_cfl_dt_1d(ctypes.byref(p), ctypes.c_double(cfl), _ptr(_arr(W, 3 * p.nx)))


def stage(p, dt, Wp, Gp, Wd, Gd):
    """One stage's operator: dict of L, Lt, gb (re-evaluated gradient), gt per grid."""
    nxd, nyd = dual_dims(p)
    Wp, Gp, Wd, Gd = (_arr(a) for a in (Wp, Gp, Wd, Gd))
    n, nd = p.nx * p.ny, nxd * nyd
    out = {k: np.zeros(s) for k, s in [("Lp", 4 * n), ("Ltp", 4 * n), ("gbp", 8 * n), ("gtp", 8 * n),
                                       ("Ld", 4 * nd), ("Ltd", 4 * nd), ("gbd", 8 * nd), ("gtd", 8 * nd)]}
    rc = lib().oracle_stage(ctypes.byref(p), ctypes.c_double(dt), _ptr(Wp), _ptr(Gp), _ptr(Wd), _ptr(Gd),
                            *(_ptr(out[k]) for k in ("Lp", "Ltp", "gbp", "gtp", "Ld", "Ltd", "gbd", "gtd")))
    if rc != 0:
        raise ValueError("oracle_stage failed")
    shp = {"p": (p.ny, p.nx), "d": (nyd, nxd)}
    for k in list(out):
        g = k[-1]
        lead = (4,) if k[:-1] in ("L", "Lt") else (2, 4)
        out[k] = out[k].reshape(lead + shp[g])
    return out


def cfl_dt(p, cfl, Wp, Wd):
    return lib().oracle_cfl_dt(ctypes.byref(p), ctypes.c_double(cfl), _ptr(_arr(Wp)), _ptr(_arr(Wd)))


# ---- component-level functions (pins) ----

def maxwell_moment(rho, U, V, lam, K, a, b, c, half_axis=-1, half_sign=0):
    return lib().oracle_maxwell_moment(ctypes.c_double(rho), ctypes.c_double(U), ctypes.c_double(V),
                                       ctypes.c_double(lam), ctypes.c_double(K), a, b, c,
                                       half_axis, half_sign)


def slope(W, dW, gamma=1.4):
    out = np.zeros(4)
    lib().oracle_slope(_ptr(_arr(W, 4)), _ptr(_arr(dW, 4)), ctypes.c_double(gamma), _ptr(out))
    return out


def time_slope(W, ax, ay, gamma=1.4):
    out = np.zeros(4)
    lib().oracle_time_slope(_ptr(_arr(W, 4)), _ptr(_arr(ax, 4)), _ptr(_arr(ay, 4)),
                            ctypes.c_double(gamma), _ptr(out))
    return out


def fdist_coeffs(tau, t):
    out = np.zeros(6)
    lib().oracle_fdist_coeffs(ctypes.c_double(tau), ctypes.c_double(t), _ptr(out))
    return out


def time_integrals(tau, delta):
    out = np.zeros(6)
    lib().oracle_time_integrals(ctypes.c_double(tau), ctypes.c_double(delta), _ptr(out))
    return out


def recon_left(variant, Q, Qx, h):
    out = np.zeros(3)
    lib().oracle_recon_left(variant, _ptr(_arr(Q, 4)), _ptr(_arr(Qx, 3)), ctypes.c_double(h), _ptr(out))
    return out


def recon_right(variant, Q, Qx, h):
    out = np.zeros(3)
    lib().oracle_recon_right(variant, _ptr(_arr(Q, 4)), _ptr(_arr(Qx, 3)), ctypes.c_double(h), _ptr(out))
    return out


def recon_node(variant, Q, Qx, h):
    out = np.zeros(2)
    lib().oracle_recon_node(variant, _ptr(_arr(Q, 3)), _ptr(_arr(Qx, 3)), ctypes.c_double(h), _ptr(out))
    return out


def geno_blend(variant, node, IS, q, qx, PH, PHx):
    out = np.zeros(3)
    lib().oracle_geno_blend(variant, node, _ptr(_arr(IS, 3)), _ptr(_arr(q, 3)), _ptr(_arr(qx, 3)),
                            ctypes.c_double(PH), ctypes.c_double(PHx), _ptr(out))
    return out


def compact_flux(variant, chi, Fi, Fn):
    return lib().oracle_compact_flux(variant, ctypes.c_double(chi), _ptr(_arr(Fi, 3)), _ptr(_arr(Fn, 2)))


def iface_solve(p, normal, dt, Wl, Wr, Wln, Wrn, Wt):
    """Returns dict Fh, Fht, Whl, Whr, Whlt, Whrt (4 each) and tau."""
    out = np.zeros(25)
    lib().oracle_iface_solve(ctypes.byref(p), normal, ctypes.c_double(dt), *(_ptr(_arr(a, 4)) for a in
                             (Wl, Wr, Wln, Wrn, Wt)), _ptr(out))
    keys = ["Fh", "Fht", "Whl", "Whr", "Whlt", "Whrt"]
    d = {k: out[4 * i:4 * i + 4].copy() for i, k in enumerate(keys)}
    d["tau"] = out[24]
    return d


def nodal_flux(p, dt, W, Wx, Wy):
    """Returns dict F, G, Ft, Gt (4 each)."""
    out = np.zeros(16)
    lib().oracle_nodal_flux(ctypes.byref(p), ctypes.c_double(dt), _ptr(_arr(W, 4)), _ptr(_arr(Wx, 4)),
                            _ptr(_arr(Wy, 4)), _ptr(out))
    return {k: out[4 * i:4 * i + 4].copy() for i, k in enumerate(["F", "G", "Ft", "Gt"])}


def char_basis(gamma, normal, Wa, Wb):
    """(L, R) 4x4 characteristic basis of a line (None if the mean state is not physical)."""
    L = np.zeros(16)
    R = np.zeros(16)
    rc = lib().oracle_char_basis(ctypes.c_double(gamma), int(normal), _ptr(_arr(Wa, 4)), _ptr(_arr(Wb, 4)),
                                 _ptr(L), _ptr(R))
    return None if rc else (L.reshape(4, 4), R.reshape(4, 4))


def recon_line(variant, recon_vars, gamma, normal, Q, Qx, h):
    """Line reconstruction from Q[4 entries][4 fields], Qx[4][4]: (Wl, Wr, Wlx, Wrx, chi)."""
    out = np.zeros(17)
    lib().oracle_recon_line(int(variant), int(recon_vars), ctypes.c_double(gamma), int(normal),
                            _ptr(_arr(Q, 16)), _ptr(_arr(Qx, 16)), ctypes.c_double(h), _ptr(out))
    return out[0:4], out[4:8], out[8:12], out[12:16], out[16]
