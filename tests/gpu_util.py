"""Helpers shared by the GPU parity tests (comparison against the oracle)."""
import numpy as np

import oracle
from paper_2606_17772_gb300 import fdcgks


def gpu_run(case, dt, nsteps, precision=fdcgks.FP64, state=None):
    import torch
    S = case.initial_state() if state is None else state
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in S])
        if nsteps:
            s.steps(dt, nsteps)
        out = s.get_state()
        torch.cuda.synchronize()
        return tuple(t.cpu().numpy() for t in out)


def oracle_run(case, dt, nsteps, state=None):
    p = oracle.make_params(**case.oracle_kwargs())
    S = case.initial_state() if state is None else state
    return oracle.steps(p, dt, nsteps, *S)


def rel_err(a, b):
    """max |a - b| / max |b| (norm-wise relative error of one array)."""
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max())


def field_errors(gpu, ref):
    """Relative errors of each conservative component and gradient group on
    both grids, scaled by the magnitude of that grid's whole state vector
    (W: max over the four components; gradients: max over all gradient
    components), so that components that vanish in exact arithmetic (e.g.
    rho V in a 1-D problem) are measured against the state, not against
    rounding noise."""
    errs = {}
    for gname, (W, G), (Wr, Gr) in (("p", gpu[0:2], ref[0:2]), ("d", gpu[2:4], ref[2:4])):
        sW, sG = np.abs(Wr).max(), max(np.abs(Gr).max(), 1e-300)
        for c in range(4):
            errs["W%s%d" % (gname, c)] = float(np.abs(W[c] - Wr[c]).max() / sW)
            errs["G%s%d" % (gname, c)] = float(np.abs(G[:, c] - Gr[:, c]).max() / sG)
    return errs
