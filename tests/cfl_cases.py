"""Cases for the CFL time-step tests: a Mach-250 strip, planted maxima,
near-ties, a viscous limit (the GPU parity test and its host-side checks)."""
import math

import numpy as np

from paper_2606_17772_gb300 import inputs

GAMMA = 1.4


def hypersonic_strip():
    """Mach ~250 flow (p/E ~ 1e-5): FP32 estimates of the sound speed are
    unreliable at every node."""
    def prim(x, y):
        return (1.0 + 0.1 * np.sin(2 * math.pi * x), 30.0 + np.sin(2 * math.pi * y), 0.5 + 0 * x,
                0.01 * (1.0 + 0.5 * np.cos(2 * math.pi * x)))
    return inputs.Case("hypersonic", 24, 8, 0.0, 1.0, 0.0, 1.0 / 3.0, (0, 0, 0, 0), prim=prim, tau_c1=0.05)


def _cons(rho, u, v, p):
    return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


def planted(kind):
    """A smooth state with one dual-grid node carrying the largest rate:
    'unreliable': a fast, cold node (p/E ~ 1e-7, FP32 estimate unreliable);
    'near_tie': a node 1e-7 (relative) above the largest rate of a second
    planted node."""
    case = inputs.random_smooth(40, 24, seed=7, amp=0.1)
    S = [a.copy() for a in case.initial_state()]
    Wd = S[2]
    if kind == "unreliable":
        Wd[:, 5, 7] = _cons(1.0, 40.0, 0.0, 1e-4)
    else:
        Wd[:, 5, 7] = _cons(1.0, 6.0, 0.0, 1.0)
        Wd[:, 17, 30] = _cons(1.0, 6.0 * (1 + 1e-7), 0.0, 1.0)
    return case, S


def cases():
    out = []
    for c in (inputs.vortex(32), inputs.viscous_shock_tube(40, 20), hypersonic_strip(), inputs.sod_strip(64, 3),
              inputs.random_smooth(33, 17, seed=3, amp=1e-9),
              inputs.random_smooth(30, 20, seed=4, amp=0.05, mu=0.5, Pr=0.73)):
        out.append((c.name, c, c.initial_state()))
    for kind in ("unreliable", "near_tie"):
        c, S = planted(kind)
        out.append((kind, c, S))
    return out

