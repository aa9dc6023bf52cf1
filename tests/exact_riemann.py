"""Exact solution of the 1-D Euler Riemann problem for an ideal gas.

Textbook construction: the star-region pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0,
with f_K the shock (Rankine-Hugoniot) or rarefaction (isentropic) relation of
side K, found by Newton iteration; the solution is then sampled on x/t.
Used only as a closed-form reference for the Sod tube (paper Sec. 5.2).
"""
import numpy as np


def _fk(p, rho, pk, g):
    a = np.sqrt(g * pk / rho)
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = p / pk
    f = 2.0 * a / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * a) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(L, R, g=1.4):
    rl, ul, pl = L
    rr, ur, pr = R
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, g)
        fr, dr = _fk(p, rr, pr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, g)
    fr, _ = _fk(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(L, R, x, t, x0=0.5, g=1.4):
    """(rho, u, p) arrays at positions x and time t > 0 for the diaphragm at x0."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, g)
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    out = np.zeros((3, len(x)))
    for n, xx in enumerate(x):
        s = (xx - x0) / t
        if s <= us:   # left of contact
            if ps > pl:   # left shock
                sl = ul - al * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    st = (rl, ul, pl)
                else:
                    r = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                    st = (r, us, ps)
            else:         # left rarefaction
                shl = ul - al
                asl = al * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - asl
                if s <= shl:
                    st = (rl, ul, pl)
                elif s >= stl:
                    st = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (al + (g - 1) / 2 * (ul - s))
                    r = rl * (c / al) ** (2 / (g - 1))
                    st = (r, u, pl * (c / al) ** (2 * g / (g - 1)))
        else:         # right of contact
            if ps > pr:   # right shock
                sr = ur + ar * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    st = (rr, ur, pr)
                else:
                    r = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                    st = (r, us, ps)
            else:         # right rarefaction
                shr = ur + ar
                asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + asr
                if s >= shr:
                    st = (rr, ur, pr)
                elif s <= str_:
                    st = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (ar - (g - 1) / 2 * (ur - s))
                    r = rr * (c / ar) ** (2 / (g - 1))
                    st = (r, u, pr * (c / ar) ** (2 * g / (g - 1)))
        out[:, n] = st
    return out
