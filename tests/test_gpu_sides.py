"""GPU parity of split boundary sides (fdcgks_set_sides) and the context
time that moves their split points, through the C ABI, against the oracle.

The double Mach reflection (Sec. 5.5) exercises every part: a fixed inflow
side, a transmissive outflow side, a bottom side split into outflow and a
reflecting wall at x = 1/6 (a node lies exactly on the split point), and a
top side whose fixed states switch at the exact shock's moving position.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import field_errors
from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

F = inputs.BC_FIXED


def _oracle_dts(case, nsteps, t0=0.0, spread=False):
    """Replay CFL-0.4 steps on the oracle; returns (final state, dts, spread)
    where spread is the oracle's own response to a 1e-15 relative
    perturbation of the initial data (the amplification of rounding by the
    shock)."""
    p = oracle.make_params(**case.oracle_kwargs(), t0=t0)
    S = case.initial_state()
    Sp = None
    if spread:
        rng = np.random.default_rng(0)
        Sp = tuple(a * (1 + 1e-15 * rng.standard_normal(a.shape)) for a in S)
    dts = []
    t = t0
    for _ in range(nsteps):
        dts.append(oracle.cfl_dt(p, 0.4, S[0], S[2]))
        p.t0 = t
        S = oracle.steps(p, dts[-1], 1, *S)
        if Sp is not None:
            Sp = oracle.steps(p, dts[-1], 1, *Sp)
        t += dts[-1]
    return S, dts, (max(field_errors(Sp, S).values()) if Sp is not None else 0.0)


def _gpu(case, dts, precision=fdcgks.FP64, t0=None):
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*case.initial_state())
        if t0 is not None:
            s.set_time(t0)
        for dt in dts:
            s.step(dt)
        got = s.get_state(device=False)
        t = s.get_time()
        bad = s.check()
    return got, t, bad


@pytest.mark.parametrize("recon_vars", [0, 1])
def test_double_mach_one_step_matches_oracle(recon_vars):
    case = inputs.double_mach(64, 16, flux_variant=62, recon_vars=recon_vars)
    ref, dts, _ = _oracle_dts(case, 1)
    got, t, bad = _gpu(case, dts)
    assert not bad
    assert t == dts[0]
    errs = field_errors(got, ref)
    worst = max(errs, key=errs.get)
    assert errs[worst] < 1e-12, (worst, errs[worst])


def test_double_mach_steps_match_oracle():
    """12 CFL-0.4 steps: the top split point crosses several columns; the
    bound is 1e-10 or 100 times the oracle's own spread under a 1e-15
    perturbation, whichever is larger (as for the other strong shocks)."""
    case = inputs.double_mach(64, 16, flux_variant=62, recon_vars=1)
    ref, dts, spread = _oracle_dts(case, 12, spread=True)
    assert sum(dts) * 20.0 / math.sqrt(3.0) > 3 * case.hx
    got, t, bad = _gpu(case, dts)
    assert not bad
    assert abs(t - sum(dts)) <= 1e-15 * sum(dts) * len(dts)
    errs = field_errors(got, ref)
    worst = max(errs, key=errs.get)
    assert errs[worst] < max(1e-10, 100 * spread), (worst, errs[worst], spread)


def test_context_time_starts_where_set():
    """set_time moves the split points' clock: steps from t0 match the oracle
    started at t0 (and differ from a start at 0)."""
    case = inputs.double_mach(64, 16, flux_variant=62, recon_vars=1)
    t0 = 0.01
    ref, dts, _ = _oracle_dts(case, 2, t0=t0)
    got, t, bad = _gpu(case, dts, t0=t0)
    assert abs(t - (t0 + sum(dts))) < 1e-15
    errs = field_errors(got, ref)
    assert max(errs.values()) < 1e-11
    got0, _, _ = _gpu(case, dts)
    assert max(field_errors(got0, ref).values()) > 1e-6


def test_double_mach_mixed_precision_stays_close():
    case = inputs.double_mach(64, 16, flux_variant=62, recon_vars=0)
    ref, dts, _ = _oracle_dts(case, 4)
    got, _, bad = _gpu(case, dts, fdcgks.MIXED)
    assert not bad
    errs = field_errors(got, ref)
    assert max(v for k, v in errs.items() if k.startswith("W")) < 1e-5, errs


def test_sides_of_one_kind_reproduce_the_unsplit_run():
    case = inputs.random_smooth(20, 17, seed=9, amp=0.08, bc=(1, 2, 3, 2), tau_c1=0.05, tau_c2=1.0)
    S = case.initial_state()
    outs = []
    for sides in (None, tuple(dict(kind=(b, b), split0=0.37, split_speed=2.0) for b in case.bc)):
        with fdcgks.Solver.from_case(case) as s:
            s.set_state(*S)
            if sides is not None:
                s.set_sides(sides)
            s.steps(0.003, 3)
            outs.append(s.get_state(device=False))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_set_sides_validation():
    case = inputs.random_smooth(12, 10, seed=3, bc=(1, 1, 0, 0))
    good = [dict(kind=(F, 1), split0=0.5, prim=((1.0, 0.0, 0.0, 1.0),) * 2), dict(kind=(1, 2)),
            dict(kind=(0, 0)), dict(kind=(0, 0))]
    with fdcgks.Solver.from_case(case) as s:
        s.set_sides(good)
        s.set_sides(None)
        bad_cases = [
            [good[0], good[1], dict(kind=(0, 1)), good[3]],                 # periodic direction made bounded
            [dict(kind=(0, 0)), good[1], good[2], good[3]],                  # bounded side made periodic
            [dict(kind=(3, 1)), good[1], good[2], good[3]],                  # split no-slip wall
            [dict(kind=(F, F), prim=((0.0, 0, 0, 1.0),) * 2), good[1], good[2], good[3]],   # rho = 0
            [dict(kind=(F, F), prim=((1.0, 0, 0, -1.0),) * 2), good[1], good[2], good[3]],  # p < 0
            [dict(kind=(7, 7)), good[1], good[2], good[3]],                  # unknown kind
        ]
        for sides in bad_cases:
            with pytest.raises(fdcgks.FdcgksError) as e:
                s.set_sides(sides)
            assert e.value.status == 1
        with pytest.raises(fdcgks.FdcgksError):
            s.set_time(float("nan"))


def test_adjoint_refuses_split_sides():
    case = inputs.random_smooth(12, 10, seed=3, bc=(1, 1, 2, 2))
    S = tuple(torch.from_numpy(a).cuda() for a in case.initial_state())
    with fdcgks.Solver.from_case(case) as s:
        s.set_sides([dict(kind=(1, 2), split0=0.5)] + [dict(kind=(b, b)) for b in case.bc[1:]])
        with pytest.raises(fdcgks.FdcgksError) as e:
            s.vjp_steps(0.001, 1, S, S)
        assert e.value.status == 1


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
def test_double_mach_runs_to_final_time(precision):
    """The double Mach reflection with its run settings (FD-CGKS(6-2),
    characteristic reconstruction, tau c1 = 0.05, c2 = 25) at 240 x 60 runs to
    t = 0.2 with CFL-0.4 steps and stays physical; the split top boundary's
    clock ends at the final time; the reflected shock compresses the gas well
    beyond the post-shock density 8."""
    from paper_2606_17772_gb300 import runs
    case = inputs.double_mach(240, 60, flux_variant=62, recon_vars=1)
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*case.initial_state())
        t, n = runs.advance(s, 0.2, 0.4)
        assert abs(s.get_time() - t) <= 1e-12
        Wp, _, Wd, _ = s.get_state(device=False)
    assert t == pytest.approx(0.2) and n > 100
    for W in (Wp, Wd):
        p = 0.4 * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])
        assert np.isfinite(W).all() and W[0].min() > 1.0 and p.min() > 0.5
    assert 12.0 < Wp[0].max() < 30.0
