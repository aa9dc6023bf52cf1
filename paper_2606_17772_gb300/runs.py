"""Time loops over the C ABI: advance a run to a final time with CFL steps.

Host-side driving only (time-step choice, final-step clipping, periodic
positivity checks); every step runs in the library's kernels.  The module
entry point runs one of the paper's long runs to its final time and prints a
JSON summary:

  * viscous shock tube (Sec. 5.8): density along the bottom wall and along
    y = 0.075, the two profiles the paper plots;
  * double Mach reflection (Sec. 5.5) to t = 0.2: density extrema and the
    density on the wall and along y = 0.5 (the figure is a contour plot);
  * Woodward-Colella blast waves (Sec. 5.3) to t = 0.038 with the
    one-dimensional scheme: density and pressure along the tube;
  * the isentropic vortex once around the periodic box on 128^2 ... 1024^2:
    errors against the exact solution and the observed order (initial data and
    exact solution the sum of the vortex's periodic images, images = 1);
  * the adjoint workload: the gradient of a density misfit through 500 steps
    of the 256^2 vortex, checked along 16 directions by central differences.

    python -m paper_2606_17772_gb300.runs --case viscous_tube --nx 1000 --ny 500 --precision mixed
    python -m paper_2606_17772_gb300.runs --case double_mach --nx 960 --ny 240 --precision fp64
    python -m paper_2606_17772_gb300.runs --case vortex_convergence
    python -m paper_2606_17772_gb300.runs --case adjoint --precision fp64
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


def viscous_shock_tube(nx=1000, ny=500, precision=fdcgks.MIXED, t_end=1.0, cfl=0.4, **kw):
    """Run Sec. 5.8's viscous shock tube; returns a summary dict.  kw: scheme
    options of inputs.viscous_shock_tube (tau_c1, tau_c2, recon_vars, ...)."""
    case = inputs.viscous_shock_tube(nx, ny, **kw)
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
        "case": "viscous shock tube, Re 200 (mu 0.005), Pr %.2f, %d x %d, %s, CFL %.2f, tau c1 %g c2 %g, GENO %d" % (
            case.Pr, nx, ny, "mixed" if precision == fdcgks.MIXED else "fp64", cfl, case.tau_c1, case.tau_c2,
            case.geno_variant),
        "t": t, "steps": n, "wall_seconds": wall,
        "node_updates_per_s": n * (nx * ny + case.nxd * case.nyd) / wall,
        "rho_min": float(min(Wp[0].min(), Wd[0].min())), "rho_max": float(max(Wp[0].max(), Wd[0].max())),
        "x_wall": xd[0].tolist(), "rho_wall": rho_wall.tolist(),
        "x_line": xp[0].tolist(), "rho_y0075": rho_line.tolist(),
    }


def vortex_convergence(ns=(128, 256, 512, 1024), precisions=(fdcgks.FP64, fdcgks.MIXED), t_end=10.0, cfl=0.2,
                       dt_h2=False, **kw):
    """The isentropic vortex (strength 5, free stream (1, 1, 1, 1)) advected once
    around the periodic [0, 10]^2 box (t = 10: the exact solution is the
    initial state) on each grid: L1 error of the density against the exact
    solution (mean absolute error over the primary nodes, and the same
    integral over the domain), the observed order between successive grids,
    and for the mixed path the L1 difference from the FP64 run.  dt_h2: the
    CFL number halves with every doubling of the grid from the first one, so
    that dt ~ h^2 (the paper's accuracy runs) and the time error falls as fast
    as the spatial error of a sixth-order scheme."""
    out = {"case": "isentropic vortex, [0,10]^2 periodic, strength 5, to t = %g, CFL %.2f%s, %s" % (
        t_end, cfl, " x (n0/n) (dt ~ h^2)" if dt_h2 else "", json.dumps(kw)), "grids": []}
    prev = {}
    for n in ns:
        case = inputs.vortex(n, **kw)
        S0 = case.initial_state()
        exact = S0[0][0]
        row = {"n": n}
        rho = {}
        for prec in precisions:
            name = "mixed" if prec == fdcgks.MIXED else "fp64"
            with fdcgks.Solver.from_case(case, prec) as s:
                s.set_state(*S0)
                w0 = time.perf_counter()
                t, k = advance(s, t_end, cfl * ns[0] / n if dt_h2 else cfl)
                wall = time.perf_counter() - w0
                rho[name] = s.get_state(device=False)[0][0]
            err = np.abs(rho[name] - exact)
            row[name] = {"steps": k, "wall_seconds": wall, "L1_mean": float(err.mean()),
                         "L1_integral": float(err.sum() * case.hx * case.hy), "Linf": float(err.max())}
            if name in prev:
                row[name]["order_L1"] = float(np.log2(prev[name] / err.mean()))
            prev[name] = err.mean()
        if "fp64" in rho and "mixed" in rho:
            row["mixed_vs_fp64_L1_mean"] = float(np.abs(rho["mixed"] - rho["fp64"]).mean())
        out["grids"].append(row)
    return out


def _timed_run(case, precision, t_end, cfl):
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*case.initial_state())
        w0 = time.perf_counter()
        t, n = advance(s, t_end, cfl)
        state = s.get_state(device=False)
        wall = time.perf_counter() - w0
        t_ctx = s.get_time()
    return state, t, n, wall, t_ctx


def double_mach(nx=960, ny=240, precision=fdcgks.FP64, t_end=0.2, cfl=0.4, flux_variant=62, recon_vars=1, **kw):
    """Run Sec. 5.5's double Mach reflection; returns a summary dict."""
    case = inputs.double_mach(nx, ny, flux_variant=flux_variant, recon_vars=recon_vars, **kw)
    (Wp, Gp, Wd, Gd), t, n, wall, t_ctx = _timed_run(case, precision, t_end, cfl)
    xp, yp = case.node_xy(False)
    xd, _ = case.node_xy(True)
    k = min(max(int(np.searchsorted(yp[:, 0], 0.5)) - 1, 0), ny - 2)
    return {
        "case": "double Mach reflection, %d x %d, FD-CGKS(6-%d), %s reconstruction, %s, CFL %.2f" % (
            nx, ny, 2 if flux_variant == 62 else 4, "characteristic" if recon_vars else "conservative",
            "mixed" if precision == fdcgks.MIXED else "fp64", cfl),
        "t": t, "t_context": t_ctx, "steps": n, "wall_seconds": wall,
        "node_updates_per_s": n * (nx * ny + case.nxd * case.nyd) / wall,
        "rho_min": float(min(Wp[0].min(), Wd[0].min())), "rho_max": float(max(Wp[0].max(), Wd[0].max())),
        "x_wall": xd[0].tolist(), "rho_wall": Wd[0, 0].tolist(),
        "x_line": xp[0].tolist(), "rho_y05": Wp[0, k].tolist(),
    }


def woodward_colella(nx=400, t_end=0.038, cfl=0.4, flux_variant=62, recon_vars=0, geno_variant=1, **kw):
    """Run Sec. 5.3's interacting blast waves with the one-dimensional scheme
    (one launch: the line's own CFL steps run inside the kernel); returns a
    summary dict.  FP64.  Defaults: FD-CGKS(6-2) with App. D's GENO constants
    (with the Sec. 3.2 constants and tau_c2 = 1 the line loses positivity at
    t = 0.027)."""
    case = inputs.woodward_colella(nx, flux_variant=flux_variant, recon_vars=recon_vars, geno_variant=geno_variant,
                                   **kw)
    W, G = inputs.line_state(case)
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        w0 = time.perf_counter()
        tt, kk = L.run(t_end, cfl)
        wall = time.perf_counter() - w0
        flags, _ = L.check()
        Wf, _ = L.get_state(device=False)
    if flags[0]:
        raise RuntimeError("non-physical state at t = %.6g after %d steps" % (tt[0], kk[0]))
    xp, _ = case.node_xy(False)
    rho = Wf[0, 0]
    p = (case.gamma - 1.0) * (Wf[0, 2] - 0.5 * Wf[0, 1] ** 2 / rho)
    return {
        "case": "Woodward-Colella blast waves, N = %d, one-dimensional FD-CGKS(6-%d), GENO variant %d, %s, "
                "CFL %.2f, fp64" % (nx, 2 if flux_variant == 62 else 4, geno_variant,
                                    "characteristic" if recon_vars else "conservative", cfl),
        "t": float(tt[0]), "steps": int(kk[0]), "wall_seconds": wall,
        "rho_min": float(rho.min()), "rho_max": float(rho.max()), "p_min": float(p.min()),
        "x": xp[0].tolist(), "rho": rho.tolist(), "p": p.tolist(),
    }


def adjoint_window(n=256, nsteps=500, ndir=16, checkpoint_every=50, variant="linear", precision=fdcgks.FP64,
                   cfl=0.2, strength=5.0):
    """Gradient of a density misfit through nsteps steps of the n^2 isentropic
    vortex: J = 1/2 sum (rho - rho_target)^2 h^2 on the primary grid, the
    target a run from rho plus 8 seeded Gaussian bumps (sigma 0.5, amplitude
    1e-3), differentiated with respect to the primary W^0 by fdcgks_vjp_steps
    (checkpoints every checkpoint_every steps), and checked along ndir seeded
    random unit directions against central differences of J (Richardson
    extrapolated from steps 1e-5 n and 5e-6 n).  variant
    "linear": linear reconstruction with tau = 0.05 dt, where the differences
    are in their linear regime; "geno": the App. D GENO constants, where the
    vortex's far field puts them out of it (the errors are reported, not a
    check).  Along the first direction the difference step is swept from 1e-2
    to 1e-9 (times n), which shows whether the map is smooth at that scale.
    On a mixed-precision solver the trajectory is the mixed run."""
    import torch
    kw = dict(geno_variant=2, tau_c1=0.05, tau_c2=0.0) if variant == "linear" else dict(geno_variant=1)
    case = inputs.vortex(n, strength=strength, **kw)
    S0 = [torch.from_numpy(a).cuda() for a in case.initial_state()]
    rng = np.random.default_rng(1)
    X, Y = case.node_xy(False)
    bump = np.zeros_like(X)
    for _ in range(8):
        cx, cy = rng.uniform(0, 10, 2)
        bump += np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * 0.5 ** 2))
    h2 = case.hx * case.hy
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*S0)
        dt = s.cfl_dt(cfl)
        Wt = S0[0].clone()
        Wt[0] += torch.from_numpy(1e-3 * bump).cuda()
        s.set_state(Wt, *S0[1:])
        s.steps(dt, nsteps)
        target = s.get_state()[0][0].clone()

        def J(Wp0):
            s.set_state(Wp0, *S0[1:])
            s.steps(dt, nsteps)
            return 0.5 * float(((s.get_state()[0][0] - target) ** 2).sum()) * h2

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J0 = J(S0[0])
        torch.cuda.synchronize()
        t_forward = time.perf_counter() - t0
        fin = s.get_state()
        seed = [torch.zeros_like(t) for t in S0]
        seed[0][0] = (fin[0][0] - target) * h2
        t0 = time.perf_counter()
        g = s.vjp_steps(dt, nsteps, S0, seed, checkpoint_every=checkpoint_every)
        torch.cuda.synchronize()
        t_adjoint = time.perf_counter() - t0
        drng = np.random.default_rng(2)
        rel, sweep = [], []
        for k in range(ndir):
            d = torch.from_numpy(drng.standard_normal(S0[0].shape)).cuda()
            d /= d.norm()
            # central differences at steps e and e/2 combined by Richardson
            # extrapolation, (4 D(e/2) - D(e)) / 3: the O(e^2) term cancels, so a
            # step far above rounding (1e-5 n) still gives an O(e^4) error
            eps = 1e-5 * n
            d1 = (J(S0[0] + eps * d) - J(S0[0] - eps * d)) / (2 * eps)
            d2 = (J(S0[0] + 0.5 * eps * d) - J(S0[0] - 0.5 * eps * d)) / eps
            fd = (4.0 * d2 - d1) / 3.0
            ad = float((g[0] * d).sum())
            rel.append(abs(ad - fd) / abs(fd))
            if k == 0:
                # step-size sweep along the first direction: in the linear regime the
                # difference error falls as eps^2 until rounding takes over; where the
                # map is not smooth at the scale of eps it does not settle
                for e in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9):
                    ee = e * n
                    fde = (J(S0[0] + ee * d) - J(S0[0] - ee * d)) / (2 * ee)
                    sweep.append([e, abs(ad - fde) / abs(ad)])
    return {"case": "adjoint", "n": n, "steps": nsteps, "checkpoint_every": checkpoint_every, "variant": variant,
            "precision": "mixed" if precision == fdcgks.MIXED else "fp64", "dt": dt, "J": J0,
            "forward_s": t_forward, "adjoint_s": t_adjoint, "gradient_norm": float(g[0].norm()),
            "fd_rel_err": rel, "fd_rel_err_max": max(rel) if rel else None,
            "step_sweep_rel_err": sweep}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--case", choices=["viscous_tube", "double_mach", "woodward_colella", "vortex_convergence",
                                       "adjoint"], default="viscous_tube")
    ap.add_argument("--steps", type=int, default=500, help="adjoint: steps through which J is differentiated")
    ap.add_argument("--dirs", type=int, default=16, help="adjoint: directions checked by central differences")
    ap.add_argument("--variant", choices=["linear", "geno"], default="linear", help="adjoint: reconstruction")
    ap.add_argument("--nx", type=int, default=None)
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--t-end", type=float, default=None)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--flux", type=int, choices=[62, 64], default=None)
    ap.add_argument("--recon-vars", type=int, choices=[0, 1], default=None)
    ap.add_argument("--geno", type=int, choices=[0, 1, 2], default=None,
                    help="GENO constants: 0 Sec. 3.2 text, 1 App. D, 2 linear (default: the case's)")
    ap.add_argument("--tau-c1", type=float, default=None, help="collision time constant c1 (default: the case's)")
    ap.add_argument("--tau-c2", type=float, default=None, help="collision time constant c2 (default: the case's)")
    ap.add_argument("--images", type=int, default=None,
                    help="vortex_convergence: periodic images summed in the initial data (default 1)")
    ap.add_argument("--grids", default=None, help="vortex_convergence: comma-separated grid sizes")
    ap.add_argument("--precisions", default="fp64,mixed", help="vortex_convergence: fp64 and/or mixed")
    ap.add_argument("--dt-h2", action="store_true", help="vortex_convergence: dt ~ h^2 (CFL halved per doubling)")
    ap.add_argument("--out", default=None, help="write the JSON summary here (default: stdout)")
    a = ap.parse_args()
    from . import build
    build.build()
    prec = fdcgks.MIXED if a.precision == "mixed" else fdcgks.FP64
    opt = {k: v for k, v in (("flux_variant", a.flux), ("recon_vars", a.recon_vars), ("tau_c1", a.tau_c1),
                             ("tau_c2", a.tau_c2), ("geno_variant", a.geno)) if v is not None}
    if a.case == "adjoint":
        res = adjoint_window(a.nx or 256, a.steps, a.dirs, variant=a.variant, precision=prec,
                             cfl=a.cfl if a.cfl != 0.4 else 0.2)
    elif a.case == "vortex_convergence":
        ns = tuple(int(x) for x in a.grids.split(",")) if a.grids else (128, 256, 512, 1024)
        precs = tuple(fdcgks.MIXED if x == "mixed" else fdcgks.FP64 for x in a.precisions.split(","))
        res = vortex_convergence(ns=ns, precisions=precs, t_end=a.t_end or 10.0, cfl=a.cfl if a.cfl != 0.4 else 0.2,
                                 dt_h2=a.dt_h2, images=1 if a.images is None else a.images, **opt)
    elif a.case == "viscous_tube":
        res = viscous_shock_tube(a.nx or 1000, a.ny or 500, prec, a.t_end or 1.0, a.cfl, **opt)
    elif a.case == "double_mach":
        res = double_mach(a.nx or 960, a.ny or 240, prec, a.t_end or 0.2, a.cfl, **opt)
    else:
        res = woodward_colella(a.nx or 400, a.t_end or 0.038, a.cfl, **opt)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
        print(json.dumps({k: v for k, v in res.items() if not isinstance(v, list)}))
    else:
        print(text)


if __name__ == "__main__":
    main()
