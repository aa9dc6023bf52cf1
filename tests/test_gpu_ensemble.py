"""GPU tests of the batched ensemble (fdcgks_ens_*), called through the C ABI.

An ensemble member runs the same per-node device functions and the same
time-step formula as a single context.  The ensemble's kernels are separate
builds of those functions, and the compiler may fuse multiply-adds
differently in them, so a member agrees with a single-context run to
rounding (a few ulps per step; tolerances below), not bit for bit.  Within
one dispatch mode the ensemble runs one kernel build per phase whatever the
tile shapes, and each node's arithmetic does not depend on the tiling, so
tile shapes change nothing, bit for bit.  One member is also checked against
the oracle directly.
"""
import numpy as np
import pytest

import oracle
from gpu_util import field_errors, oracle_run
from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def members():
    """Uneven grids, every boundary kind, viscous and inviscid, both flux and GENO variants."""
    return [
        inputs.vortex(24, strength=3.0, xc=4.0, yc=6.5),
        inputs.density_wave_2d(16),
        inputs.sod_strip(40, 4),
        inputs.random_smooth(18, 13, seed=31, amp=0.08, bc=(3, 3, 3, 2), mu=0.01, Pr=0.73, tau_c2=1.0),
        inputs.random_smooth(7, 5, seed=32, amp=0.05, flux_variant=62, geno_variant=1, grad_base=1,
                             tau_c1=0.05),
        inputs.vortex(37, strength=1.5, xc=8.0, yc=2.0),
        inputs.random_smooth(21, 9, seed=33, amp=0.08, bc=(1, 2, 2, 1), geno_variant=2, tau_c1=0.05),
    ]


def single_run(case, precision, nsteps, dt=None, cfl=None):
    """Single-context run: fixed dt, or the CFL step recomputed before every step."""
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*[torch.from_numpy(a).cuda() for a in case.initial_state()])
        dts = []
        for _ in range(nsteps):
            d = dt if dt is not None else s.cfl_dt(cfl)
            s.step(d)
            dts.append(d)
        out = s.get_state()
        torch.cuda.synchronize()
        return tuple(t.cpu().numpy() for t in out), dts


def make_ensemble(cases, precision):
    ens = fdcgks.Ensemble.from_cases(cases, precision)
    for m, c in enumerate(cases):
        ens.set_state(m, *c.initial_state())
    return ens


def member_state(ens, m):
    return ens.get_state(m, device=False)


def fixed_dts(cases):
    out = []
    for c in cases:
        with fdcgks.Solver.from_case(c) as s:
            s.set_state(*c.initial_state())
            out.append(s.cfl_dt(0.3))
    return out


def assert_same(a, b, what):
    for k, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y), (what, k, float(np.abs(x - y).max()))


# member vs single context after a few steps, relative to each grid's state
# (W) and gradient (G) scale: FP64 to rounding; mixed to the FP32 rounding of
# the interface values, which the gradients re-evaluated from them as
# differences over h amplify (the mixed path's own bounds against FP64 are
# of the same size)
TOL = {fdcgks.FP64: (1e-13, 1e-13), fdcgks.MIXED: (2e-6, 1e-4)}


def assert_close(a, b, precision, what):
    errs = field_errors(a, b)
    for k, v in errs.items():
        assert v < TOL[precision][0 if k[0] == "W" else 1], (what, k, v)


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
def test_members_equal_single_runs_fixed_dt(precision):
    cases = members()
    dts = fixed_dts(cases)
    with make_ensemble(cases, precision) as ens:
        ens.run(3, dt=dts)
        t, last, st = ens.status()
        assert not st.any()
        for m, c in enumerate(cases):
            ref, _ = single_run(c, precision, 3, dt=dts[m])
            assert_close(member_state(ens, m), ref, precision, m)
            assert t[m] == (dts[m] + dts[m]) + dts[m] and last[m] == dts[m]


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
def test_members_equal_single_runs_cfl(precision):
    """Per-member CFL steps computed on the device agree with fdcgks_cfl_dt:
    the first (same state, same formula) to the last bit or two, later ones
    to the rounding of the states they are computed from."""
    cases = members()
    with make_ensemble(cases, precision) as ens:
        ens.run(1, cfl=0.4)
        t, last, st = ens.status()
        ens.run(3, cfl=0.4)
        t4, last4, st4 = ens.status()
        assert not st.any() and not st4.any()
        for m, c in enumerate(cases):
            ref, dts = single_run(c, precision, 4, cfl=0.4)
            assert last[m] == pytest.approx(dts[0], rel=1e-15) and t[m] == last[m], m
            assert last4[m] == pytest.approx(dts[-1], rel=1e-9), m
            assert t4[m] == pytest.approx(sum(dts), rel=1e-9), m
            assert_close(member_state(ens, m), ref, precision, m)


def hypersonic_strip():
    """Mach ~250 flow (p/E ~ 1e-5): FP32 estimates of the sound speed are
    unreliable here, so the mixed CFL screening must evaluate these nodes."""
    import math

    def prim(x, y):
        return (1.0 + 0.1 * np.sin(2 * math.pi * x), 30.0 + np.sin(2 * math.pi * y), 0.5 + 0 * x,
                0.01 * (1.0 + 0.5 * np.cos(2 * math.pi * x)))
    return inputs.Case("hypersonic", 24, 8, 0.0, 1.0, 0.0, 1.0 / 3.0, (0, 0, 0, 0), prim=prim, tau_c1=0.05)


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
def test_device_cfl_step_equals_host_formula(precision):
    """The first CFL step of every member equals fdcgks_cfl_dt on the same
    state and the oracle's all-node FP64 value (the mixed ensemble and the
    single contexts screen nodes in FP32 and evaluate the candidates in FP64:
    the maxima, hence dt, must still be those over all nodes)."""
    cases = members() + [hypersonic_strip(), inputs.viscous_shock_tube(40, 20), inputs.sod_strip(64, 3)]
    with make_ensemble(cases, precision) as ens:
        states = [member_state(ens, m) for m in range(len(cases))]
        ens.run(1, cfl=0.37)
        _, last, st = ens.status()
    for m, c in enumerate(cases):
        with fdcgks.Solver.from_case(c, precision) as s:
            s.set_state(*c.initial_state())
            ref = s.cfl_dt(0.37)
        assert last[m] == pytest.approx(ref, rel=1e-15), (m, last[m], ref)
        # and the all-node FP64 value of the oracle on the member's own state
        St = states[m]
        full = oracle.cfl_dt(oracle.make_params(**c.oracle_kwargs()), 0.37, St[0], St[2])
        assert last[m] == pytest.approx(full, rel=1e-14), (m, last[m], full)


def test_member_matches_oracle():
    cases = members()
    dts = fixed_dts(cases)
    with make_ensemble(cases, fdcgks.FP64) as ens:
        ens.run(2, dt=dts)
        for m in (0, 3, 4):
            errs = field_errors(member_state(ens, m), oracle_run(cases[m], dts[m], 2))
            worst = max(errs, key=errs.get)
            assert errs[worst] < 1e-12, (m, worst, errs[worst])


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
def test_tile_configurations_do_not_change_results(precision):
    cases = members()
    results = {}
    for cfg in ([5, 5, 5, 0], [3, 4, 7, 0], [0, 1, 2, 0], [5, 5, 5, 1], [7, 3, 6, 1], [4, 7, 3, 1]):
        with make_ensemble(cases, precision) as ens:
            ens.set_tiles(cfg)
            assert ens.get_tiles() == cfg
            ens.run(2, cfl=0.4)
            results[tuple(cfg)] = [member_state(ens, m) for m in range(len(cases))]
    ref = {0: results[(5, 5, 5, 0)], 1: results[(5, 5, 5, 1)]}
    for cfg, r in results.items():
        for m in range(len(cases)):
            assert_same(r[m], ref[cfg[3]][m], (cfg, m))          # same kernels: bit for bit
            assert_close(r[m], ref[0][m], precision, (cfg, m))   # other dispatch build: to rounding


def test_tuner_restores_state_and_picks_valid_config():
    cases = inputs.ensemble_members(count=12, seed=5, nmin=16, nmax=96)
    with make_ensemble(cases, fdcgks.MIXED) as ens:
        ens.run(1, cfl=0.4)
        before = [member_state(ens, m) for m in range(len(cases))]
        t0, d0, s0 = ens.status()
        cfg, ms = ens.tune(cfl=0.4, trial_steps=2)
        assert ms > 0 and all(3 <= c <= 7 for c in cfg[:3]) and cfg[3] in (0, 1)
        assert ens.get_tiles() == cfg
        t1, d1, s1 = ens.status()
        assert np.array_equal(t0, t1) and np.array_equal(d0, d1) and np.array_equal(s0, s1)
        for m in range(len(cases)):
            assert_same(member_state(ens, m), before[m], m)


def test_profile_advances_like_run():
    cases = members()[:4]
    with make_ensemble(cases, fdcgks.FP64) as a, make_ensemble(cases, fdcgks.FP64) as b:
        ms = a.profile(2, cfl=0.4)
        assert all(v > 0 for v in ms.values()), ms
        b.run(2, cfl=0.4)
        for m in range(len(cases)):
            assert_same(member_state(a, m), member_state(b, m), m)


@pytest.mark.parametrize("precision,cfl_kernels", [(fdcgks.FP64, 1), (fdcgks.MIXED, 2)])
def test_launch_count(precision, cfl_kernels):
    """Per step: CFL pass(es), the time-step kernel, then 5 phases per stage."""
    cases = members()[:3]
    with make_ensemble(cases, precision) as ens:
        n0 = ens.launches()
        ens.run(3, cfl=0.4)
        ens.run(2, dt=[1e-3] * 3)
        ens.synchronize()
        assert ens.launches() - n0 == 3 * (cfl_kernels + 11) + 2 * 11


def test_blown_up_member_is_frozen_and_others_continue():
    """A member driven unstable by a far too large dt is flagged and frozen;
    the others are unaffected (no fault: the flag is a device-side bit)."""
    cases = members()[:4]
    dts = fixed_dts(cases)
    bad = list(dts)
    bad[0] = 40.0 * dts[0]
    with make_ensemble(cases, fdcgks.FP64) as ens:
        ens.run(6, dt=bad)
        t, last, st = ens.status()
        assert st[0] & fdcgks.ENS_NONPHYSICAL and st[0] & fdcgks.ENS_FROZEN, st
        assert last[0] == 0.0 and t[0] < 6 * bad[0]
        assert not st[1:].any()
        for m in range(1, 4):
            ref, _ = single_run(cases[m], fdcgks.FP64, 6, dt=dts[m])
            assert_close(member_state(ens, m), ref, fdcgks.FP64, m)
        # set_state clears the member's status and time
        ens.set_state(0, *cases[0].initial_state())
        t, last, st = ens.status()
        assert st[0] == 0 and t[0] == 0.0


def test_ensemble_errors():
    cases = members()[:2]
    with pytest.raises(fdcgks.FdcgksError) as e:
        fdcgks.Ensemble([fdcgks.params_for_case(cases[0], fdcgks.FP64),
                         fdcgks.params_for_case(cases[1], fdcgks.MIXED)])
    assert e.value.status == 1
    with pytest.raises(fdcgks.FdcgksError) as e:
        fdcgks.Ensemble([fdcgks.make_params(2, 8, bc=(1, 1, 0, 0))])
    assert e.value.status == 1
    with fdcgks.Ensemble.from_cases(cases) as ens:
        with pytest.raises(fdcgks.FdcgksError) as e:
            ens.run(1, cfl=0.4)
        assert e.value.status == 4                                    # member without state
        ens.set_state(0, *cases[0].initial_state())
        ens.set_state(1, *cases[1].initial_state())
        for bad in (lambda: ens.run(1, cfl=-1.0), lambda: ens.run(1, dt=[1e-3, 0.0]),
                    lambda: ens.set_tiles([5, 5, 8, 0]), lambda: ens.set_tiles([5, 5, 5, 2]),
                    lambda: ens.get_state(2), lambda: ens.run(-1)):
            with pytest.raises((fdcgks.FdcgksError, IndexError)) as e:
                bad()
            if isinstance(e.value, fdcgks.FdcgksError):
                assert e.value.status == 1
        S = [a.copy() for a in cases[0].initial_state()]
        S[0][0, 2, 3] = -1.0
        with pytest.raises(fdcgks.FdcgksError) as e:
            ens.set_state(0, *S)
        assert e.value.status == 3
        with pytest.raises(fdcgks.FdcgksError) as e:
            ens.run(1, cfl=0.4)                                       # member 0 no longer loaded
        assert e.value.status == 4
