"""Pins of the oracle's split boundary sides (Sec. 5.5 double Mach reflection:
inflow, outflow, a reflecting wall that starts part way along the bottom,
and a top boundary that follows the exact moving shock).

* a side split into two parts of the same kind, or split beyond either end
  of the side, is exactly the unsplit boundary of that kind;
* fixed-state sides holding the state of a uniform moving flow keep it
  exactly (the fixed ghosts equal the interior, zero gradients);
* an oblique Mach 10 shock with the exact moving states imposed on the top
  and bottom sides stays where the Rankine-Hugoniot shock speed puts it, on
  the rows next to both tracked sides, and leaves the pre-shock gas ahead of
  it untouched; a split point moving 20 % too fast or too slow fails this;
* the double Mach reflection itself stays physical over its first steps.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_17772_gb300 import inputs

R3 = math.sqrt(3.0)
F = inputs.BC_FIXED


def _run(case, dt, nsteps, state=None, t0=0.0):
    p = oracle.make_params(**case.oracle_kwargs(), t0=t0)
    S = case.initial_state() if state is None else state
    return oracle.steps(p, dt, nsteps, *S)


def _pres(W, gamma=1.4):
    return (gamma - 1.0) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])


def _walls_case(sides=None):
    c = inputs.random_smooth(10, 9, seed=5, amp=0.08, bc=(1, 2, 2, 1), tau_c1=0.05, tau_c2=1.0)
    c.sides = sides
    return c


@pytest.mark.parametrize("split0", [0.3, -5.0, 5.0])
def test_sides_of_one_kind_are_the_unsplit_boundary(split0):
    base = _walls_case()
    ref = _run(base, 0.004, 2)
    sides = tuple(dict(kind=(b, b), split0=split0, split_speed=1.7) for b in base.bc)
    out = _run(_walls_case(sides), 0.004, 2)
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)


def test_split_beyond_the_ends_takes_one_part():
    base = _walls_case()
    ref = _run(base, 0.004, 2)
    # the other kinds would change the result (checked below); a split point
    # below every ghost node's coordinate selects part 1, above all of them part 0
    other = {1: 2, 2: 1}
    lo = tuple(dict(kind=(other[b], b), split0=-10.0) for b in base.bc)
    hi = tuple(dict(kind=(b, other[b]), split0=10.0) for b in base.bc)
    for sides in (lo, hi):
        out = _run(_walls_case(sides), 0.004, 2)
        for a, b in zip(out, ref):
            assert np.array_equal(a, b)
    swapped = tuple(dict(kind=(other[b], other[b])) for b in base.bc)
    out = _run(_walls_case(swapped), 0.004, 2)
    assert max(np.abs(a - b).max() for a, b in zip(out, ref)) > 1e-6


def test_fixed_sides_keep_a_uniform_moving_flow():
    state = (1.3, 0.45, -0.25, 0.9)
    c = inputs.random_smooth(9, 8, seed=6, bc=(1, 1, 1, 1), tau_c1=0.05, tau_c2=1.0)
    c.prim = lambda x, y: state
    c.sides = tuple(dict(kind=(F, F), split0=0.4, split_speed=3.0, prim=(state, state)) for _ in range(4))
    S = c.initial_state()
    out = _run(c, 0.01, 3)
    for a, b in zip(out, S):
        assert np.array_equal(a, b)


def _oblique(nx, ny, x0s, speed_factor=1.0):
    """Oblique Mach 10 shock through (x0s, 0) at 60 degrees on [0, 2] x [0, 1],
    the double Mach reflection's states, post-shock inflow at x = 0, outflow at
    x = 2 and the exact moving states on both y sides."""
    post, pre = inputs.DMR_POST, inputs.DMR_PRE

    def prim(x, y):
        behind = x < x0s + y / R3
        return tuple(np.where(behind, a, b) for a, b in zip(post, pre))
    speed = 20.0 / R3 * speed_factor
    sides = (dict(kind=(F, F), prim=(post, post)), dict(kind=(1, 1)),
             dict(kind=(F, F), split0=x0s, split_speed=20.0 / R3, prim=(post, pre)),
             dict(kind=(F, F), split0=x0s + 1.0 / R3, split_speed=speed, prim=(post, pre)))
    return inputs.Case("oblique_shock", nx, ny, 0.0, 2.0, 0.0, 1.0, (1, 1, 1, 1), prim=prim, sides=sides,
                       flux_variant=62, recon_vars=1, tau_c1=0.05, tau_c2=1.0)


def _advance(c, nsteps, cfl=0.4):
    p = oracle.make_params(**c.oracle_kwargs())
    S = c.initial_state()
    t = 0.0
    for _ in range(nsteps):
        dt = oracle.cfl_dt(p, cfl, S[0], S[2])
        p.t0 = t
        S = oracle.steps(p, dt, 1, *S)
        t += dt
    return S, t


def _shock_offsets(c, S, t, x0s):
    """Offset, in cells, of the rho = 4.7 crossing from the exact shock on the
    first and last rows of both grids (next to the tracked sides)."""
    out = []
    for dual, W in ((False, S[0]), (True, S[2])):
        X, Y = c.node_xy(dual)
        for row in (0, W.shape[1] - 1):
            rho, xs = W[0, row], X[row]
            i = np.where((rho[:-1] > 4.7) & (rho[1:] <= 4.7))[0]
            assert len(i) == 1, (dual, row, i)
            j = i[0]
            xc = xs[j] + (xs[j + 1] - xs[j]) * (rho[j] - 4.7) / (rho[j] - rho[j + 1])
            out.append((xc - (x0s + (Y[row, 0] + 20.0 * t) / R3)) / c.hx)
    return np.array(out)


def test_tracked_oblique_shock_moves_at_the_exact_speed():
    x0s = 0.25
    c = _oblique(36, 18, x0s)
    S, t = _advance(c, 30)
    assert t * 20.0 / R3 > 10 * c.hx                     # the shock crossed > 10 cells
    off = _shock_offsets(c, S, t, x0s)
    assert np.abs(off).max() < 1.0, off
    # the pre-shock gas more than 6 cells ahead of the exact shock is untouched
    # (up to the GENO weights' exponentially small reach across the shock)
    Wpre = c.conservative(np.array([3.0]), np.array([0.0]))[:, 0]
    for dual, W in ((False, S[0]), (True, S[2])):
        X, Y = c.node_xy(dual)
        ahead = (X - (x0s + (Y + 20.0 * t) / R3)) * (R3 / 2) > 6 * c.hx
        assert ahead.sum() > 100
        assert np.abs(W[:, ahead] - Wpre[:, None]).max() < 1e-4 * np.abs(Wpre).max()


@pytest.mark.parametrize("factor", [0.8, 1.2])
def test_tracked_oblique_shock_detects_a_wrong_split_speed(factor):
    x0s = 0.25
    c = _oblique(36, 18, x0s, speed_factor=factor)
    S, t = _advance(c, 30)
    off = _shock_offsets(c, S, t, x0s)
    assert np.abs(off).max() > 1.2, off


def test_double_mach_reflection_stays_physical():
    c = inputs.double_mach(48, 12, flux_variant=62, recon_vars=1)
    S, t = _advance(c, 20)
    for W in (S[0], S[2]):
        assert np.isfinite(W).all()
        assert W[0].min() > 1.0 and _pres(W).min() > 0.5
        assert W[0].max() < 30.0
    assert t > 0.03
