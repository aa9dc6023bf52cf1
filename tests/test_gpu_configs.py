"""GPU parity on the benchmark's own workloads, beyond one step.

* The resolved isentropic vortex (48^2 on [0,10]^2, App. D's GENO constants,
  CFL 0.2: the settings of the throughput benchmark) over 100 steps.  With
  GENO the scheme amplifies rounding on this case: the oracle itself turns a
  1e-15 relative perturbation of the initial data into a few 1e-9 after 100
  steps (the path function of Sec. 3.2 reacts to far-field variations of
  1e-6 and below), so the bound is 1e-10 or 100 times that spread, measured
  here on this exact case, whichever is larger.  With the linear
  reconstruction nothing switches and the bound is 1e-10 itself.
* Both paths against the FP64 oracle on the viscous shock tube (Sec. 5.8
  constants, no-slip walls; bounded by the oracle's own perturbation spread,
  as the case amplifies rounding) and the mixed path on a member of the
  ensemble workload (through the ensemble path), with stated bounds.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import field_errors, gpu_run, oracle_run
from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _cfl02_dt(case):
    S = case.initial_state()
    return oracle.cfl_dt(oracle.make_params(**case.oracle_kwargs()), 0.2, S[0], S[2])


def test_hundred_steps_resolved_vortex_linear():
    case = inputs.vortex(48, geno_variant=2)
    dt = _cfl02_dt(case)
    errs = field_errors(gpu_run(case, dt, 100), oracle_run(case, dt, 100))
    worst = max(errs, key=errs.get)
    assert errs[worst] < 1e-10, (worst, errs[worst])


def test_hundred_steps_resolved_vortex_geno_within_oracle_spread():
    case = inputs.vortex(48)
    assert case.geno_variant == 1
    dt = _cfl02_dt(case)
    p = oracle.make_params(**case.oracle_kwargs())
    S = case.initial_state()
    rng = np.random.default_rng(0)
    Sp = tuple(a * (1 + 1e-15 * rng.standard_normal(a.shape)) for a in S)
    ref = oracle.steps(p, dt, 100, *S)
    spread = max(field_errors(oracle.steps(p, dt, 100, *Sp), ref).values())
    errs = field_errors(gpu_run(case, dt, 100), ref)
    worst = max(errs, key=errs.get)
    assert errs[worst] < max(1e-10, 100 * spread), (worst, errs[worst], spread)


def _split(errs):
    w = max(v for k, v in errs.items() if k.startswith("W"))
    g = max(v for k, v in errs.items() if k.startswith("G"))
    return w, g


@pytest.mark.parametrize("nx,ny,t_end", [(40, 20, None), (120, 60, 0.006)])
def test_viscous_tube_within_oracle_spread(nx, ny, t_end):
    """The viscous tube (Sec. 5.8 constants), the oracle's CFL-0.4 steps
    replayed: 40 x 20 over 20 steps, and 120 x 60 to t = 0.006, past the
    time (t ~ 0.002-0.005) at which the 1000 x 500 runs leave the physical
    states with these constants.  Where the diaphragm
    meets the no-slip wall the scheme amplifies any perturbation strongly
    (about 1e10 in 20 steps on the 40 x 20 tube), so neither path can agree
    pointwise with the oracle to its rounding.  The bound is the oracle's own
    spread under a perturbation of the size of each path's rounding: FP64
    within max(1e-10, 100 x the spread at 1e-15); the mixed path (FP32
    arithmetic, rounding ~6e-8) within 10 x the spread at 1e-7, or its
    one-step bounds (1e-6 values, 2e-5 gradients) where that is larger."""
    case = inputs.viscous_shock_tube(nx, ny)
    p = oracle.make_params(**case.oracle_kwargs())
    S0 = case.initial_state()
    S = S0
    dts, t = [], 0.0
    while (t_end is None and len(dts) < 20) or (t_end is not None and t < t_end):
        dts.append(oracle.cfl_dt(p, 0.4, S[0], S[2]))
        S = oracle.steps(p, dts[-1], 1, *S)
        t += dts[-1]

    def spread(rel):
        rng = np.random.default_rng(1)
        Sp = tuple(a * (1 + rel * rng.standard_normal(a.shape)) for a in S0)
        for dt in dts:
            Sp = oracle.steps(p, dt, 1, *Sp)
        return _split(field_errors(Sp, S))

    got = {}
    for prec in (fdcgks.FP64, fdcgks.MIXED):
        with fdcgks.Solver.from_case(case, prec) as s:
            s.set_state(*S0)
            for dt in dts:
                s.step(dt)
            got[prec] = _split(field_errors(s.get_state(device=False), S))
            assert not s.check()
    sw, sg = spread(1e-15)
    assert got[fdcgks.FP64][0] < max(1e-10, 100 * sw) and got[fdcgks.FP64][1] < max(1e-10, 100 * sg), \
        (got[fdcgks.FP64], sw, sg)
    sw, sg = spread(1e-7)
    assert got[fdcgks.MIXED][0] < max(1e-6, 10 * sw) and got[fdcgks.MIXED][1] < max(2e-5, 10 * sg), \
        (got[fdcgks.MIXED], sw, sg)


def test_mixed_ensemble_member_within_stated_error():
    """The smallest member of the benchmark's ensemble (mixed precision,
    ensemble path), 20 fixed CFL-0.2 steps: within 1e-5 (values) and 2e-4
    (gradients) of the FP64 oracle, the bounds of the single-run mixed path."""
    cases = inputs.ensemble_members(count=256, seed=0, nmax=512)
    m = min(cases, key=lambda c: c.nx)
    dt = _cfl02_dt(m)
    ref = oracle_run(m, dt, 20)
    with fdcgks.Ensemble.from_cases([m], fdcgks.MIXED) as ens:
        ens.set_state(0, *m.initial_state())
        ens.run(20, dt=[dt])
        ens.synchronize()
        got = ens.get_state(0, device=False)
        _, _, st = ens.status()
        assert st[0] == 0
    w, g = _split(field_errors(got, ref))
    assert w < 1e-5 and g < 2e-4, (w, g)


def test_mixed_full_size_tube_passes_the_shock_wall_corner():
    """The 1000 x 500 viscous tube in mixed precision with App. D's GENO
    constants and tau c2 = 25, CFL-0.4 steps to t = 0.006: past the time
    (t = 0.0047) at which this run left the physical states while the FP32
    erfc was an absolute-error approximation (half-space moments off by up to
    1e-3 relative where erfc is small).  This grid is marginal with every
    constant set (whether a run leaves the physical states later depends on
    rounding-level details), so only this stretch is asserted."""
    from paper_2606_17772_gb300 import runs
    case = inputs.viscous_shock_tube(1000, 500, geno_variant=1, tau_c2=25.0)
    with fdcgks.Solver.from_case(case, fdcgks.MIXED) as s:
        s.set_state(*case.initial_state())
        t, n = runs.advance(s, 0.006, 0.4, check_every=25)
        assert t == pytest.approx(0.006) and n > 400
        W = s.get_state(device=False)
        assert np.all(np.isfinite(W[0])) and W[0][0].min() > 0.5
