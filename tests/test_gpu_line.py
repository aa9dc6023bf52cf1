"""GPU parity of the one-dimensional scheme (fdcgks_line_*, Sec. 2) against
the oracle's one-dimensional scheme, through the C ABI.

Tolerances as for the 2-D path: 1e-12 (relative, norm-wise per component
group) for one stage operator and one step, 1e-10 after 100 steps; for
shock tubes, whose early steps amplify rounding, 1e-10 or 100 times the
oracle's own response to a 1e-15 relative perturbation.
"""
import math

import numpy as np
import pytest

import exact_riemann
import oracle
from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a - b).max())


def errs(gpu, ref):
    """errors of W and of W_x, each scaled by the whole group's magnitude"""
    return rel(gpu[0], ref[0]), rel(gpu[1], ref[1])


def random_line(n, seed, bc, **kw):
    kw.setdefault("tau_c1", 0.05)
    kw.setdefault("tau_c2", 1.0)
    return inputs.random_smooth(n, 1, seed=seed, amp=0.1, bc=(bc, bc, 0, 0), **kw)


CASES = {
    "periodic_64": lambda: random_line(37, 1, 0),
    "periodic_62_appD": lambda: random_line(29, 2, 0, flux_variant=62, geno_variant=1),
    "transmissive_viscous": lambda: random_line(41, 3, 1, mu=0.01, Pr=0.72),
    "reflecting_char": lambda: random_line(33, 4, 2, recon_vars=1),
    "reflecting_linear_A": lambda: random_line(30, 5, 2, geno_variant=2, grad_base=1),
}


def gpu_steps(case, dts, state=None, batch=1):
    W, G = inputs.line_state(case) if state is None else state
    with fdcgks.Lines.from_case(case, batch) as L:
        L.set_state(np.ascontiguousarray(np.broadcast_to(W, (batch,) + W.shape)),
                    np.ascontiguousarray(np.broadcast_to(G, (batch,) + G.shape)))
        for dt in dts:
            L.steps(dt, 1)
        out = L.get_state(device=False)
        flags, _ = L.check()
    return out, flags


@pytest.mark.parametrize("name", sorted(CASES))
def test_stage_operator_matches_oracle(name):
    case = CASES[name]()
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    ref = oracle.stage_1d(p, 0.004, W, G)
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        got = {k: v.cpu().numpy()[0] for k, v in L.stage_operator(0.004).items()}
    for k in ("L", "Lt", "gb", "gt"):
        assert rel(got[k], ref[k]) < 1e-12, (k, rel(got[k], ref[k]))


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_step_matches_oracle(name):
    case = CASES[name]()
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    ref = oracle.steps_1d(p, 0.004, 1, W, G)
    (gw, gg), flags = gpu_steps(case, [0.004])
    assert flags[0] == 0
    e = errs((gw[0], gg[0]), ref)
    assert max(e) < 1e-12, e


@pytest.mark.parametrize("name", ["periodic_64", "transmissive_viscous", "reflecting_char"])
def test_hundred_steps_match_oracle(name):
    case = CASES[name]()
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    ref = oracle.steps_1d(p, 0.004, 100, W, G)
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        L.steps(0.004, 100)                      # one launch
        gw, gg = L.get_state(device=False)
    e = errs((gw[0], gg[0]), ref)
    assert max(e) < 1e-10, e


TUBES = {
    "sod": lambda: (inputs.sod_strip(100, 1), 40),
    "lax_char": lambda: (inputs.lax_strip(100, 1, recon_vars=1), 40),
    "woodward_colella_62": lambda: (inputs.woodward_colella(400, flux_variant=62), 60),
}


@pytest.mark.parametrize("name", sorted(TUBES))
def test_shock_tube_steps_match_oracle(name):
    case, nsteps = TUBES[name]()
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    rng = np.random.default_rng(0)
    Wp, Gp = W * (1 + 1e-15 * rng.standard_normal(W.shape)), G * (1 + 1e-15 * rng.standard_normal(G.shape))
    dts = []
    ref, pert = (W, G), (Wp, Gp)
    for _ in range(nsteps):
        dts.append(oracle.cfl_dt_1d(p, 0.4, ref[0]))
        ref = oracle.steps_1d(p, dts[-1], 1, *ref)
        pert = oracle.steps_1d(p, dts[-1], 1, *pert)
    spread = max(errs(pert, ref))
    (gw, gg), flags = gpu_steps(case, dts)
    assert flags[0] == 0
    e = max(errs((gw[0], gg[0]), ref))
    assert e < max(1e-10, 100 * spread), (e, spread)


def test_batch_lines_are_independent():
    """A batch of different lines: each line equals its own single-line run
    (bit for bit: the same arithmetic in the same order) and the oracle."""
    cases = [random_line(24, s, 1) for s in (11, 12, 13)]
    states = [inputs.line_state(c) for c in cases]
    W = np.ascontiguousarray(np.stack([s[0] for s in states]))
    G = np.ascontiguousarray(np.stack([s[1] for s in states]))
    with fdcgks.Lines.from_case(cases[0], batch=3) as L:
        L.set_state(W, G)
        L.steps(0.003, 5)
        gw, gg = L.get_state(device=False)
    p = oracle.make_params(**cases[0].oracle_kwargs())
    for b, st in enumerate(states):
        (sw, sg), _ = gpu_steps(cases[0], [0.003] * 5, state=st)
        assert np.array_equal(gw[b], sw[0]) and np.array_equal(gg[b], sg[0])
        ref = oracle.steps_1d(p, 0.003, 5, *st)
        assert max(errs((gw[b], gg[b]), ref)) < 1e-12


def test_density_wave_table_1_on_the_gpu():
    """Table 1's h = 1/16 case through the GPU (2048 steps in one launch):
    the error against the exact solution equals the oracle's."""
    n = 32
    h = 2.0 / n
    nst = int(math.ceil(2.0 / (0.5 * h * h)))
    case = inputs.density_wave_1d(n, ny=1)
    W, G = inputs.line_state(case)
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        L.steps(2.0 / nst, nst)
        gw, _ = L.get_state(device=False)
    exact = inputs.line_state(inputs.density_wave_1d(n, ny=1, t=2.0))[0][0]
    e = np.abs(gw[0][0] - exact)
    assert e.mean() == pytest.approx(1.4734e-08, rel=0.02)        # the paper's Table 1 L1 error
    ref, _ = oracle.steps_1d(oracle.make_params(**case.oracle_kwargs()), 2.0 / nst, nst, W, G)
    assert rel(gw[0], ref) < 1e-10


def test_cfl_run_reaches_the_final_time_like_the_oracle():
    """fdcgks_line_run: each line's own CFL steps in one launch, the last one
    clipped.  Against the oracle's CFL loop: the same number of steps and the
    same state up to the scheme's amplification of rounding over ~190 steps
    of a shock tube (the two reduce h / (|U| + c) differently, so their time
    steps differ in the last bits): 100 times the oracle's own response to a
    1e-15 relative perturbation of the initial data (about 1e-5 measured:
    GENO's weights in the nearly uniform states next to the waves amplify
    perturbations, see the adjoint tests)."""
    case = inputs.sod_strip(100, 1)
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)

    def oracle_run(state):
        t, k = 0.0, 0
        while t < 0.2 * (1 - 1e-14):
            dt = min(oracle.cfl_dt_1d(p, 0.4, state[0]), 0.2 - t)
            state = oracle.steps_1d(p, dt, 1, *state)
            t += dt
            k += 1
        return state, k
    ref, k = oracle_run((W, G))
    rng = np.random.default_rng(1)
    pert, _ = oracle_run((W * (1 + 1e-15 * rng.standard_normal(W.shape)), G))
    spread = max(errs(pert, ref))
    other = inputs.lax_strip(100, 1)          # a second line with other data
    Wl, Gl = inputs.line_state(other)
    with fdcgks.Lines.from_case(case, batch=2) as L:
        L.set_state(np.stack([W, Wl]), np.stack([G, Gl]))
        tt, kk = L.run(0.2, 0.4)
        gw, gg = L.get_state(device=False)
        flags, anyf = L.check()
    assert anyf == 0
    assert tt[0] == pytest.approx(0.2, rel=1e-14) and tt[1] == pytest.approx(0.2, rel=1e-14)
    assert kk[0] == k
    assert max(errs((gw[0], gg[0]), ref)) < max(1e-9, 100 * spread), spread


def test_cfl_run_on_smooth_data_matches_the_oracle_loop():
    """On smooth data rounding is not amplified: the in-kernel CFL loop and the
    oracle's host loop take the same steps and agree to 1e-10."""
    case = random_line(40, 7, 1, mu=0.005, Pr=0.72)
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    t, k, ref = 0.0, 0, (W, G)
    while t < 0.1 * (1 - 1e-14):
        dt = min(oracle.cfl_dt_1d(p, 0.4, ref[0]), 0.1 - t)
        ref = oracle.steps_1d(p, dt, 1, *ref)
        t += dt
        k += 1
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        tt, kk = L.run(0.1, 0.4)
        gw, gg = L.get_state(device=False)
    assert kk[0] == k and k >= 15
    assert tt[0] == pytest.approx(0.1, rel=1e-14)
    assert max(errs((gw[0], gg[0]), ref)) < 1e-10


def test_nonphysical_line_is_flagged_and_stops():
    case = inputs.sod_strip(50, 1)
    W, G = inputs.line_state(case)
    bad = W.copy()
    bad[2, 10] = -1.0                            # negative energy: negative pressure
    with fdcgks.Lines.from_case(case, batch=2) as L:
        L.set_state(np.stack([W, bad]), np.stack([G, G]))
        tt, kk = L.run(0.05, 0.4, max_steps=50)
        flags, anyf = L.check()
    assert flags[0] == 0 and flags[1] & 1 and anyf & 1
    assert tt[0] == pytest.approx(0.05) and kk[1] == 1      # stopped after the first step


def test_argument_errors():
    case = inputs.sod_strip(20, 1)
    for bad in (dict(n=2), dict(batch=0), dict(bc=(0, 1)), dict(bc=(3, 3)), dict(flux_variant=63)):
        kw = dict(n=20, batch=1, bc=(1, 1))
        kw.update(bad)
        with pytest.raises(fdcgks.FdcgksError) as e:
            fdcgks.Lines(fdcgks.line_params(**kw))
        assert e.value.status == 1
    with fdcgks.Lines.from_case(case) as L:
        for call in (lambda: L.steps(0.0, 1), lambda: L.steps(float("nan"), 1), lambda: L.run(0.1, -1.0),
                     lambda: L.steps(0.01, -1)):
            with pytest.raises(fdcgks.FdcgksError) as e:
                call()
            assert e.value.status == 1


def test_sod_200_to_final_time_on_both_paths():
    """The Sod tube with 200 primary nodes, CFL 0.3, to t = 0.2, on the GPU
    through both schemes: the 1-D scheme (one launch, in-kernel CFL loop) and
    the 2-D scheme on a one-row strip (host CFL loop).  Checked against the
    exact Riemann solution: mean density error 0.0030 / 0.0029 and mean
    velocity error 0.0078 / 0.0060 measured by the oracle on the two paths;
    bounded overshoot."""
    case = inputs.sod_strip(200, 1)
    X, _ = case.node_xy(False)
    ex = exact_riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), X[0], 0.2)
    W, G = inputs.line_state(case)
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        tt, kk = L.run(0.2, 0.3)
        lw, _ = L.get_state(device=False)
        assert L.check()[1] == 0
    assert tt[0] == pytest.approx(0.2, rel=1e-14)
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*case.initial_state())
        t = 0.0
        while t < 0.2 * (1 - 1e-14):
            dt = min(s.cfl_dt(0.3), 0.2 - t)
            s.step(dt)
            t += dt
        assert not s.check()
        Wp = s.get_state(device=False)[0]
    for rho, u, er, eu, top in ((lw[0][0], lw[0][1] / lw[0][0], 0.0040, 0.0105, 1.001),
                                (Wp[0, 0], Wp[1, 0] / Wp[0, 0], 0.0040, 0.0080, 1.002)):
        assert np.abs(rho - ex[0]).mean() < er
        assert np.abs(u - ex[1]).mean() < eu
        assert rho.max() < top and rho.min() > 0.125 * 0.99


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_cluster_spread_line_equals_single_block(cluster):
    """A line spread over a thread-block cluster computes every item with the
    same arithmetic as one block: fixed steps and CFL runs agree bit for bit."""
    cases = [inputs.lax_strip(96, 1, recon_vars=1), inputs.woodward_colella(128, flux_variant=62, geno_variant=1)]
    for case in cases:
        W, G = inputs.line_state(case)
        out = {}
        for cs in (1, cluster):
            with fdcgks.Lines.from_case(case, batch=3, cluster=cs) as L:
                L.set_state(np.ascontiguousarray(np.broadcast_to(W, (3,) + W.shape)),
                            np.ascontiguousarray(np.broadcast_to(G, (3,) + G.shape)))
                L.steps(1e-4, 7)
                tt, kk = L.run(0.01, 0.4)
                out[cs] = (L.get_state(device=False), tt, kk, L.check()[0])
        (a, ta, ka, fa), (b, tb, kb, fb) = out[1], out[cluster]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(ta, tb) and np.array_equal(ka, kb) and np.array_equal(fa, fb)
        assert ka[0] >= 5


@pytest.mark.parametrize("name", ["periodic_64", "transmissive_viscous", "reflecting_char"])
def test_mixed_precision_steps_within_fp32_error(name):
    """Mixed precision (FP32 reconstruction and kinetic solves, FP64 state and
    accumulation): 20 steps of smooth lines against the FP64 oracle, within
    the FP32 arithmetic's error accumulated over the steps (5e-6 of the state,
    5e-4 of the gradients, relative to each group's magnitude; 1.4e-6 and
    1.4e-4 measured on the periodic line: the averaged gradients are
    differences of interface values over h, which loses FP32 digits)."""
    case = CASES[name]()
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    ref = oracle.steps_1d(p, 0.004, 20, W, G)
    with fdcgks.Lines.from_case(case, precision=fdcgks.MIXED) as L:
        L.set_state(W, G)
        L.steps(0.004, 20)
        gw, gg = L.get_state(device=False)
        assert L.check()[1] == 0
    ew, eg = errs((gw[0], gg[0]), ref)
    assert ew < 5e-6 and eg < 5e-4, (ew, eg)
    assert ew > 0.0                               # the FP32 arithmetic is in use


def test_mixed_precision_sod_and_blast_waves_to_final_time():
    """Mixed-precision CFL runs of the Sod tube (exact solution as for FP64) and
    of the Woodward-Colella blast waves (stays physical; density peak within
    2 % of the FP64 run), each on a cluster and bit-identical on one block."""
    sod = inputs.sod_strip(200, 1)
    X, _ = sod.node_xy(False)
    ex = exact_riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), X[0], 0.2)
    W, G = inputs.line_state(sod)
    res = {}
    for cs in (0, 1):
        with fdcgks.Lines.from_case(sod, precision=fdcgks.MIXED, cluster=cs) as L:
            L.set_state(W, G)
            tt, kk = L.run(0.2, 0.3)
            res[cs] = L.get_state(device=False)
            assert L.check()[1] == 0
    assert np.array_equal(res[0][0], res[1][0])
    rho = res[0][0][0][0]
    assert np.abs(rho - ex[0]).mean() < 0.0040
    assert np.abs(res[0][0][0][1] / rho - ex[1]).mean() < 0.0105
    wc = inputs.woodward_colella(400, flux_variant=62, geno_variant=1)
    W, G = inputs.line_state(wc)
    peaks = {}
    for prec in (fdcgks.FP64, fdcgks.MIXED):
        with fdcgks.Lines.from_case(wc, precision=prec) as L:
            L.set_state(W, G)
            tt, kk = L.run(0.038, 0.4)
            assert L.check()[1] == 0 and tt[0] == pytest.approx(0.038)
            peaks[prec] = L.get_state(device=False)[0][0][0].max()
    assert peaks[fdcgks.MIXED] == pytest.approx(peaks[fdcgks.FP64], rel=0.02)


@pytest.mark.parametrize("n", [1, 2, 5])
def test_tiny_periodic_lines_match_oracle(n):
    """Degenerate periodic lines (fewer nodes than ghost layers: the ghost map
    wraps around more than once); n = 1 is a uniform state and stays so."""
    case = inputs.random_smooth(n, 1, seed=30 + n, amp=0.1, bc=(0, 0, 0, 0), tau_c1=0.05, tau_c2=1.0)
    p = oracle.make_params(**case.oracle_kwargs())
    W, G = inputs.line_state(case)
    ref = oracle.steps_1d(p, 0.002, 3, W, G)
    with fdcgks.Lines.from_case(case) as L:
        L.set_state(W, G)
        L.steps(0.002, 3)
        gw, gg = L.get_state(device=False)
    assert max(errs((gw[0], gg[0]), ref)) < 1e-12
    if n == 1:
        assert np.array_equal(gw[0], W)

