"""Time loops over the C ABI: advance a run to a final time with CFL steps.

Host-side driving only (time-step choice, final-step clipping, periodic
positivity checks); every step runs in the library's kernels.  The module
entry point runs the viscous shock tube (Sec. 5.8) to its final time and
prints a JSON summary with the density along the bottom wall and along
y = 0.075, the two profiles the paper plots.

    python -m paper_2606_17772_gb300.runs --nx 1000 --ny 500 --precision mixed --t-end 1.0
"""
import argparse
import json
import time

import numpy as np

from . import fdcgks, inputs


def advance(solver, t_end, cfl, check_every=200, t0=0.0):
    """Advance `solver` from time t0 to t_end with dt = fdcgks_cfl_dt(cfl) each
    step (the last step clipped to land on t_end).  Raises FdcgksError-style
    RuntimeError if a step produces a non-physical state.  Returns (t, steps)."""
    t, n = t0, 0
    while t < t_end * (1.0 - 1e-14):
        dt = min(solver.cfl_dt(cfl), t_end - t)
        solver.step(dt)
        t += dt
        n += 1
        if n % check_every == 0 and solver.check():
            raise RuntimeError("non-physical state at t = %.6g after %d steps" % (t, n))
    if solver.check():
        raise RuntimeError("non-physical state at t = %.6g after %d steps" % (t, n))
    return t, n


def viscous_shock_tube(nx=1000, ny=500, precision=fdcgks.MIXED, t_end=1.0, cfl=0.4):
    """Run Sec. 5.8's viscous shock tube; returns a summary dict."""
    case = inputs.viscous_shock_tube(nx, ny)
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*case.initial_state())
        w0 = time.perf_counter()
        t, n = advance(s, t_end, cfl)
        Wp, Gp, Wd, Gd = s.get_state(device=False)
        wall = time.perf_counter() - w0
    xd, yd = case.node_xy(True)
    xp, yp = case.node_xy(False)
    # density along y = 0 (dual nodes on the wall) and along y = 0.075 (primary rows
    # nearest to it, linearly interpolated in y)
    rho_wall = Wd[0, 0]
    yrow = yp[:, 0]
    k = int(np.searchsorted(yrow, 0.075)) - 1
    k = min(max(k, 0), len(yrow) - 2)
    w = (0.075 - yrow[k]) / (yrow[k + 1] - yrow[k])
    rho_line = (1 - w) * Wp[0, k] + w * Wp[0, k + 1]
    return {
        "case": "viscous shock tube, Re 200 (mu 0.005), Pr %.2f, %d x %d, %s, CFL %.2f" % (
            case.Pr, nx, ny, "mixed" if precision == fdcgks.MIXED else "fp64", cfl),
        "t": t, "steps": n, "wall_seconds": wall,
        "node_updates_per_s": n * (nx * ny + case.nxd * case.nyd) / wall,
        "rho_min": float(min(Wp[0].min(), Wd[0].min())), "rho_max": float(max(Wp[0].max(), Wd[0].max())),
        "x_wall": xd[0].tolist(), "rho_wall": rho_wall.tolist(),
        "x_line": xp[0].tolist(), "rho_y0075": rho_line.tolist(),
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--nx", type=int, default=1000)
    ap.add_argument("--ny", type=int, default=500)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--out", default=None, help="write the JSON summary here (default: stdout)")
    a = ap.parse_args()
    from . import build
    build.build()
    res = viscous_shock_tube(a.nx, a.ny, fdcgks.MIXED if a.precision == "mixed" else fdcgks.FP64, a.t_end, a.cfl)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
        print(json.dumps({k: v for k, v in res.items() if not isinstance(v, list)}))
    else:
        print(text)


if __name__ == "__main__":
    main()
