"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (relative, norm-wise per field: max|gpu - oracle| / max|oracle|):
1e-12 after one step and 1e-10 after 100 steps for the FP64 path.  The two
implementations round differently (fused multiply-adds, reciprocal
multiplication, closed-form instead of eliminated slope systems), and the
fitted time derivatives divide differences by dt^2, so agreement is to a
few hundred ulps, not bitwise.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import field_errors, gpu_run, oracle_run, rel_err
from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

GAMMA = 1.4


def _rand_states(rng, n):
    rho = rng.uniform(0.5, 2.0, n)
    U, V = rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n)
    p = rng.uniform(0.3, 2.0, n)
    return np.stack([rho, rho * U, rho * V, p / (GAMMA - 1) + 0.5 * rho * (U * U + V * V)], 1)


GAS = [dict(mu=0.0, Pr=1.0, tau_c1=0.05, tau_c2=1.0), dict(mu=0.01, Pr=0.73, tau_c1=0.0, tau_c2=1.0),
       dict(mu=0.0, Pr=1.0, tau_c1=0.0, tau_c2=0.0), dict(mu=0.5, Pr=0.72, tau_c1=0.0, tau_c2=1.0)]


@pytest.mark.parametrize("gas", range(len(GAS)))
@pytest.mark.parametrize("normal", [0, 1])
def test_interface_solve_matches_oracle(gas, normal):
    rng = np.random.default_rng(10 * gas + normal)
    n, dt = 97, 0.004
    Wl = _rand_states(rng, n)
    Wr = Wl * (1 + 0.05 * rng.normal(size=(n, 4)))
    Wr[: n // 3] = _rand_states(rng, n // 3)           # strong jumps too
    inp = np.concatenate([Wl, Wr] + [0.3 * rng.normal(size=(n, 4)) for _ in range(3)], 1)
    prm = fdcgks.make_params(8, 8, gamma=GAMMA, **GAS[gas])
    out = fdcgks.iface_batch(prm, normal, dt, torch.from_numpy(np.ascontiguousarray(inp)).cuda()).cpu().numpy()
    op = oracle.make_params(8, 8, gamma=GAMMA, **GAS[gas])
    ref = np.array([np.concatenate([o[k] for k in ("Fh", "Fht", "Whl", "Whr", "Whlt", "Whrt")]) for o in
                    (oracle.iface_solve(op, normal, dt, *[inp[t, 4 * k:4 * k + 4] for k in range(5)])
                     for t in range(n))])
    for k in range(6):
        assert rel_err(out[:, 4 * k:4 * k + 4], ref[:, 4 * k:4 * k + 4]) < 1e-12, k


@pytest.mark.parametrize("gas", range(len(GAS)))
def test_nodal_flux_matches_oracle(gas):
    rng = np.random.default_rng(40 + gas)
    n, dt = 77, 0.004
    inp = np.concatenate([_rand_states(rng, n), 0.3 * rng.normal(size=(n, 8))], 1)
    prm = fdcgks.make_params(8, 8, gamma=GAMMA, **GAS[gas])
    out = fdcgks.nodal_batch(prm, dt, torch.from_numpy(np.ascontiguousarray(inp)).cuda()).cpu().numpy()
    op = oracle.make_params(8, 8, gamma=GAMMA, **GAS[gas])
    ref = np.array([np.concatenate(list(oracle.nodal_flux(op, dt, inp[t, :4], inp[t, 4:8], inp[t, 8:]).values()))
                    for t in range(n)])
    for k in range(4):
        assert rel_err(out[:, 4 * k:4 * k + 4], ref[:, 4 * k:4 * k + 4]) < 1e-12


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_reconstruction_matches_oracle(variant):
    rng = np.random.default_rng(variant)
    n, h = 300, 0.07
    Q = 1 + 0.3 * rng.normal(size=(n, 4))
    Q[: n // 2] = 1 + np.cumsum(0.02 * rng.normal(size=(n // 2, 4)), axis=1)   # smooth rows
    Qx = 0.5 * rng.normal(size=(n, 4))
    prm = fdcgks.make_params(8, 8, geno_variant=variant)
    inp = torch.from_numpy(np.ascontiguousarray(np.concatenate([Q, Qx], 1))).cuda()
    out = fdcgks.recon_batch(prm, 0, h, inp).cpu().numpy()
    ref = np.array([np.concatenate([oracle.recon_left(variant, Q[t], Qx[t, :3], h),
                                    oracle.recon_right(variant, Q[t], Qx[t, 1:], h)]) for t in range(n)])
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    if variant != 2:
        # the path function is compared inside its intermediate regime too, not only at its limits
        chi = np.concatenate([ref[:, 2], ref[:, 5]])
        assert ((chi > 0.01) & (chi < 0.99)).sum() >= 100
    inp = torch.from_numpy(np.ascontiguousarray(np.concatenate([Q[:, :3], Qx[:, :3]], 1))).cuda()
    out = fdcgks.recon_batch(prm, 1, h, inp).cpu().numpy()[:, 0]
    ref = np.array([oracle.recon_node(variant, Q[t, :3], Qx[t, :3], h)[0] for t in range(n)])
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_empty_batches_are_noops():
    prm = fdcgks.make_params(8, 8)
    e = torch.empty((0, 20), dtype=torch.float64, device="cuda")
    assert fdcgks.iface_batch(prm, 0, 0.01, e).shape == (0, 24)


STAGE_CASES = {
    "periodic_ragged": lambda: inputs.random_smooth(37, 21, seed=11, amp=0.08, tau_c1=0.05, tau_c2=1.0),
    "char_periodic_ragged": lambda: inputs.random_smooth(37, 21, seed=11, amp=0.08, tau_c1=0.05, tau_c2=1.0,
                                                         recon_vars=1),
    "walls_viscous": lambda: inputs.random_smooth(21, 13, seed=12, amp=0.08, bc=(3, 3, 3, 2), mu=0.01, Pr=0.73,
                                                  tau_c2=1.0),
    "transmissive_6_2_appD": lambda: inputs.random_smooth(19, 6, seed=13, amp=0.08, bc=(1, 1, 0, 0),
                                                          flux_variant=62, geno_variant=1, tau_c1=0.05,
                                                          tau_c2=1.0),
    "symmetry_linear_readingA": lambda: inputs.random_smooth(14, 17, seed=14, amp=0.08, bc=(2, 2, 2, 2),
                                                             geno_variant=2, grad_base=1, tau_c1=0.05),
}


@pytest.mark.parametrize("name", sorted(STAGE_CASES))
def test_stage_operator_matches_oracle(name):
    case = STAGE_CASES[name]()
    dt = 0.004
    S = case.initial_state()
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*[torch.from_numpy(a).cuda() for a in S])
        got = {k: v.cpu().numpy() for k, v in s.stage_operator(dt).items()}
    ref = oracle.stage(oracle.make_params(**case.oracle_kwargs()), dt, *S)
    for k in ref:
        assert rel_err(got[k], ref[k]) < 1e-12, (k, rel_err(got[k], ref[k]))


STEP_CASES = {
    "vortex_40": (lambda: inputs.vortex(40), 0.02),
    # characteristic components (recon_vars = 1) on every boundary kind
    "char_vortex_40": (lambda: inputs.vortex(40, recon_vars=1), 0.02),
    "char_sod_strip_64x4": (lambda: inputs.sod_strip(64, 4, recon_vars=1), 0.002),
    "char_walls_6_2_appD": (lambda: inputs.random_smooth(17, 11, seed=21, amp=0.1, bc=(3, 3, 2, 2), flux_variant=62,
                                                         geno_variant=1, mu=0.002, Pr=0.7, tau_c1=0.02, tau_c2=1.0,
                                                         recon_vars=1), 0.003),
    "sod_strip_64x4": (lambda: inputs.sod_strip(64, 4), 0.002),
    "viscous_tube_24x12": (lambda: inputs.viscous_shock_tube(24, 12), 2e-4),
    "walls_6_2_appD_readingA": (lambda: inputs.random_smooth(17, 11, seed=21, amp=0.1, bc=(3, 3, 2, 2),
                                                             flux_variant=62, geno_variant=1, grad_base=1,
                                                             mu=0.002, Pr=0.7, tau_c1=0.02, tau_c2=1.0), 0.003),
    "strip_1d_16x1": (lambda: inputs.density_wave_1d(16, ny=1), 0.01),
    "strip_sod_40x2": (lambda: inputs.sod_strip(40, 2), 0.003),
}


@pytest.mark.parametrize("name", sorted(STEP_CASES))
def test_one_step_matches_oracle(name):
    mk, dt = STEP_CASES[name]
    case = mk()
    errs = field_errors(gpu_run(case, dt, 1), oracle_run(case, dt, 1))
    worst = max(errs, key=errs.get)
    assert errs[worst] < 1e-12, (worst, errs[worst])


HUNDRED = {
    # smooth 2-D wave, FD-CGKS(6-4), collisionless interfaces
    "density_wave_2d_16": lambda: (inputs.density_wave_2d(16, flux_variant=64), 0.02),
    # Sod tube on a y-periodic strip: shock, contact and rarefaction through GENO
    "sod_strip_64x4": lambda: (inputs.sod_strip(64, 4), 0.002),
}


@pytest.mark.parametrize("name", sorted(HUNDRED))
def test_hundred_steps_match_oracle(name):
    """1e-10 after 100 steps.  Cases are chosen where the scheme itself is not
    chaotic: on an under-resolved vortex (16^2 on [0,10]^2) the oracle
    amplifies a 1e-15 perturbation to 2e-4 in 100 steps through GENO
    switching, so no non-bitwise implementation can agree there."""
    case, dt = HUNDRED[name]()
    nsteps = 100
    errs = field_errors(gpu_run(case, dt, nsteps), oracle_run(case, dt, nsteps))
    worst = max(errs, key=errs.get)
    assert errs[worst] < 1e-10, (worst, errs[worst])


STRONG = {
    # density and pressure ratio 100: the positivity safeguard of the interface states acts
    # near the diaphragm in the first steps
    "strong_shock_strip_100x2": lambda: (inputs.strong_shock_strip(100, 2), 12),
    # the viscous shock tube itself (no-slip walls, symmetry top) on a coarse grid
    "viscous_tube_24x12": lambda: (inputs.viscous_shock_tube(24, 12), 6),
    "strong_shock_strip_char_100x2": lambda: (inputs.strong_shock_strip(100, 2, recon_vars=1), 12),
    # Sec. 5.2 Lax tube (a moving initial state), 6-4 and 6-2 fluxes
    "lax_strip_100x2": lambda: (inputs.lax_strip(100, 2), 20),
    "lax_strip_62_100x2": lambda: (inputs.lax_strip(100, 2, flux_variant=62), 20),
}


@pytest.mark.parametrize("name", sorted(STRONG))
def test_strong_shock_steps_match_oracle(name):
    """CFL-0.4 steps (the oracle's time steps replayed on the GPU) through the
    first steps of a strong Riemann problem, where reconstructed interface
    states with non-positive pressure are replaced by node states.

    Near the diaphragm the scheme itself amplifies rounding: on the coarse
    viscous tube the oracle turns a 1e-15 relative perturbation of the initial
    data into 1e-11 after 2 steps and 5e-9 after 6.  The GPU rounds every
    operation differently, so the bound is 1e-10 or 100 times the oracle's own
    spread under such a perturbation, whichever is larger."""
    case, nsteps = STRONG[name]()
    p = oracle.make_params(**case.oracle_kwargs())
    S = case.initial_state()
    rng = np.random.default_rng(0)
    Sp = tuple(a * (1 + 1e-15 * rng.standard_normal(a.shape)) for a in S)
    dts = []
    for _ in range(nsteps):
        dts.append(oracle.cfl_dt(p, 0.4, S[0], S[2]))
        S = oracle.steps(p, dts[-1], 1, *S)
        Sp = oracle.steps(p, dts[-1], 1, *Sp)
    spread = max(field_errors(Sp, S).values())
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*case.initial_state())
        for dt in dts:
            s.step(dt)
        got = s.get_state(device=False)
        assert not s.check()
    errs = field_errors(got, S)
    worst = max(errs, key=errs.get)
    assert errs[worst] < max(1e-10, 100 * spread), (worst, errs[worst], spread)


def test_cfl_dt_sum_matches_oracle():
    for case in (inputs.vortex(32), inputs.viscous_shock_tube(40, 20), inputs.random_smooth(20, 13, seed=2, amp=0.2)):
        S = case.initial_state()
        ref = oracle.cfl_dt_sum(oracle.make_params(**case.oracle_kwargs()), 0.4, S[0], S[2])
        with fdcgks.Solver.from_case(case) as s:
            s.set_state(*S)
            got = s.cfl_dt(0.4, form="sum")
            assert got <= s.cfl_dt(0.4)
        assert got == pytest.approx(ref, rel=1e-14)


def test_cfl_dt_matches_oracle():
    for case, cfl in ((inputs.vortex(32), 0.4), (inputs.viscous_shock_tube(40, 20), 0.3)):
        S = case.initial_state()
        with fdcgks.Solver.from_case(case) as s:
            s.set_state(*[torch.from_numpy(a).cuda() for a in S])
            got = s.cfl_dt(cfl)
        ref = oracle.cfl_dt(oracle.make_params(**case.oracle_kwargs()), cfl, S[0], S[2])
        assert got == pytest.approx(ref, rel=1e-14)


def test_host_and_device_state_round_trip():
    case = inputs.random_smooth(13, 9, seed=5, bc=(3, 3, 2, 2))
    S = case.initial_state()
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*S)                                     # host pointers
        back = s.get_state(device=False)
        for a, b in zip(S, back):
            assert np.array_equal(a, b)
        dev = s.get_state()                                 # device pointers
        for a, b in zip(S, dev):
            assert np.array_equal(a, b.cpu().numpy())


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
@pytest.mark.parametrize("nx,ny,bc", [(13, 9, (3, 3, 2, 2)), (16, 12, (0, 0, 0, 0)), (7, 30, (1, 2, 0, 0))])
def test_host_copies_equal_device_copies(precision, nx, ny, bc):
    """Host state goes through one contiguous copy per array and a device
    kernel into the padded layout (both directions); it must give exactly
    what the device-pointer path gives, after a step too (the staging area
    is the point-output buffer, overwritten by every step)."""
    case = inputs.random_smooth(nx, ny, seed=11, bc=bc)
    S = case.initial_state()
    Sd = [torch.from_numpy(a).cuda() for a in S]
    out = {}
    for path in ("host", "device"):
        with fdcgks.Solver.from_case(case, precision) as s:
            s.set_state(*(S if path == "host" else Sd))
            a = [np.asarray(t) for t in s.get_state(device=False)] if path == "host" else \
                [t.cpu().numpy() for t in s.get_state()]
            s.step(1e-3)
            b = [np.asarray(t) for t in s.get_state(device=False)] if path == "host" else \
                [t.cpu().numpy() for t in s.get_state()]
            out[path] = a + b
    for x, y in zip(out["host"], out["device"]):
        assert np.array_equal(x, y)
    if precision == fdcgks.FP64:
        for x, y in zip(S, out["host"][:4]):
            assert np.array_equal(x, y)


def test_split_run_equals_straight_run():
    """Checkpoint/resume through get_state/set_state is bit-exact."""
    case = inputs.vortex(24)
    dt = 0.03
    straight = gpu_run(case, dt, 6)
    mid = gpu_run(case, dt, 3)
    resumed = gpu_run(case, dt, 3, state=mid)
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


def test_error_statuses():
    case = inputs.vortex(8)
    S = [a.copy() for a in case.initial_state()]
    with fdcgks.Solver.from_case(case) as s:
        with pytest.raises(fdcgks.FdcgksError) as e:
            s.step(0.01)
        assert e.value.status == 4                          # no state loaded
        bad = [a.copy() for a in S]
        bad[0][0, 3, 4] = -1.0                              # negative density
        with pytest.raises(fdcgks.FdcgksError) as e:
            s.set_state(*bad)
        assert e.value.status == 3
        bad = [a.copy() for a in S]
        bad[2][3, 1, 1] = np.nan                            # non-finite energy on the dual grid
        with pytest.raises(fdcgks.FdcgksError) as e:
            s.set_state(*[torch.from_numpy(a).cuda() for a in bad])
        assert e.value.status == 3
        s.set_state(*S)
        for dt in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(fdcgks.FdcgksError) as e:
                s.step(dt)
            assert e.value.status == 1
        assert not s.check()


def test_nonphysical_step_sets_flag_without_fault():
    """A step far beyond the CFL limit on a strong shock yields negative
    pressure; the kernels flag it and the context stays usable."""
    case = inputs.viscous_shock_tube(16, 8, mu=0.0, tau_c1=0.0, tau_c2=0.0)
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*case.initial_state())
        s.steps(0.5, 3)
        assert s.check()
        rest = case.__class__(**{**case.__dict__, "prim": lambda x, y: (1.0, 0.0, 0.0, 1.0)})
        s.set_state(*rest.initial_state())                  # still usable
        s.step(1e-3)
        assert not s.check()
        out = s.get_state(device=False)
        assert np.array_equal(out[0], rest.initial_state()[0])


# ---------------------------------------------------------------------------
# full-size configuration (the throughput workload): sampled parity and
# size-independent properties
# ---------------------------------------------------------------------------

def _patch(S, i0, j0, P):
    """P x P periodic sub-problem of both grids starting at global node (i0, j0)."""
    out = []
    for a in S:
        idx_j = (j0 + np.arange(P)) % a.shape[-2]
        idx_i = (i0 + np.arange(P)) % a.shape[-1]
        out.append(np.ascontiguousarray(a[..., idx_j[:, None], idx_i[None, :]]))
    return out


@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
def test_full_size_vortex_sampled_against_oracle(precision):
    """1024^2 isentropic vortex (both grids, 2.1M nodes), one step as timed by
    the benchmark.  A node's new state depends only on nodes within 7 of it,
    so the oracle computes sampled nodes on 21 x 21 periodic patches around
    them; conservation is checked over the whole grid.  FP64: 1e-12 of the
    field's magnitude.  Mixed precision: 1e-6 for the values; for the
    averaged gradients the FP32 path's GENO floor (data varying by less than
    64 u |W|, u = 2^-24, count as smooth) decides the weights differently from
    FP64 in the far field, where the high- and low-order derivatives differ by
    up to that variation over one cell, 64 u max|W| / h (1.4e-3 at 1024^2; the
    largest difference seen is 2.2e-5); conservation to 1e-9 (FP32 increments
    added to float-float pairs)."""
    n = 1024
    case = inputs.vortex(n)
    S = case.initial_state()
    if precision == fdcgks.FP64:
        tol_w, tol_g, tol_c = 1e-12, 1e-12, 1e-11
    else:
        wmax = max(np.abs(S[0]).max(), np.abs(S[2]).max())
        tol_w, tol_g, tol_c = 1e-6, 64 * 2.0 ** -24 * wmax / case.hx, 1e-9
    dt = 0.4 * case.hx / (math.sqrt(2.0) + math.sqrt(1.4)) * 0.9
    got = gpu_run(case, dt, 1, precision)
    rng = np.random.default_rng(7)
    P, c = 21, 10
    samples = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(6, 2))] + [(512 - c, 512 - c), (0, n - c)]
    for i0, j0 in samples:
        sub = case.__class__(**{**case.__dict__, "nx": P, "ny": P, "x0": case.x0 + i0 * case.hx,
                                "x1": case.x0 + (i0 + P) * case.hx, "y0": case.y0 + j0 * case.hy,
                                "y1": case.y0 + (j0 + P) * case.hy})
        ref = oracle_run(sub, dt, 1, state=_patch(S, i0, j0, P))
        gp = _patch(got, i0, j0, P)
        for k, (a, b) in enumerate(zip(gp, ref)):
            aa, bb = a[..., c, c], b[..., c, c]
            tol = tol_w if k % 2 == 0 else tol_g
            assert np.abs(aa - bb).max() <= tol * max(1.0, np.abs(bb).max()), (i0, j0, k)
    for g in (0, 2):
        tot0, tot1 = S[g].sum(axis=(1, 2)), got[g].sum(axis=(1, 2))
        assert np.all(np.abs(tot1 - tot0) <= tol_c * np.abs(S[g]).sum(axis=(1, 2)))


# ---------------------------------------------------------------------------
# mixed precision: FP32 reconstruction/flux arithmetic, FP64 state and time
# coefficients; bounded error against the FP64 oracle
# ---------------------------------------------------------------------------

def test_mixed_interface_solve_within_fp32_bounds():
    rng = np.random.default_rng(77)
    n, dt = 200, 0.004
    Wl = _rand_states(rng, n)
    Wr = Wl * (1 + 0.02 * rng.normal(size=(n, 4)))
    inp = np.concatenate([Wl, Wr] + [0.3 * rng.normal(size=(n, 4)) for _ in range(3)], 1)
    gas = dict(mu=0.0, Pr=1.0, tau_c1=0.05, tau_c2=1.0)
    prm = fdcgks.make_params(8, 8, gamma=GAMMA, precision=fdcgks.MIXED, **gas)
    out = fdcgks.iface_batch(prm, 0, dt, torch.from_numpy(np.ascontiguousarray(inp)).cuda()).cpu().numpy()
    op = oracle.make_params(8, 8, gamma=GAMMA, **gas)
    ref = np.array([np.concatenate([o[k] for k in ("Fh", "Fht", "Whl", "Whr", "Whlt", "Whrt")]) for o in
                    (oracle.iface_solve(op, 0, dt, *[inp[t, 4 * k:4 * k + 4] for k in range(5)]) for t in range(n))])
    bounds = [2e-6, 1e-4, 2e-6, 2e-6, 1e-4, 1e-4]   # values vs time derivatives (fitted, divided by dt^2)
    for k in range(6):
        assert rel_err(out[:, 4 * k:4 * k + 4], ref[:, 4 * k:4 * k + 4]) < bounds[k], k


@pytest.mark.parametrize("nsteps,bound_w,bound_g", [(1, 1e-6, 2e-5), (20, 1e-5, 2e-4)])
def test_mixed_steps_within_stated_error(nsteps, bound_w, bound_g):
    case = inputs.vortex(40)
    dt = 0.02
    errs = field_errors(gpu_run(case, dt, nsteps, fdcgks.MIXED), oracle_run(case, dt, nsteps))
    w = max(v for k, v in errs.items() if k.startswith("W"))
    g = max(v for k, v in errs.items() if k.startswith("G"))
    assert w < bound_w and g < bound_g, errs


def test_characteristic_reconstruction_is_single_context_only():
    case = inputs.vortex(12, recon_vars=1)
    with pytest.raises(fdcgks.FdcgksError) as e:
        fdcgks.Ensemble.from_cases([case])
    assert e.value.status == 1
    with fdcgks.Solver.from_case(case) as s:
        S0 = [torch.from_numpy(a).cuda() for a in case.initial_state()]
        with pytest.raises(fdcgks.FdcgksError) as e:
            s.vjp_steps(0.01, 1, S0, S0)
        assert e.value.status == 1
    with pytest.raises(fdcgks.FdcgksError) as e:
        fdcgks.Solver(fdcgks.make_params(8, 8, recon_vars=2))
    assert e.value.status == 1
