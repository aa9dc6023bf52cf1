"""GPU tests of the adjoint (fdcgks_vjp_steps), through the C ABI.

The adjoint is the transpose of the step's Jacobian, so for any direction v
of the initial state and any seed a of the final state
    <a, (S(x + eps v) - S(x - eps v)) / (2 eps)> = <vjp(a), v>
up to the central difference's O(eps^2) error and rounding.  These tests
check that identity for one and several steps on every boundary kind and
variant, check the objective's gradient against central differences of the
FP64 oracle (an implementation that shares no code with the kernels), and
check the torch.autograd wrapper.

GENO's path function (tanh of C = 20 times a ratio of smoothness
indicators) is smooth but steep: central differences reach the derivative
to 1e-9 only below relative steps of about 1e-7 (at 1e-6 their truncation
error is still 1e-5 on these fields), so the steps are 1e-8 relative.

Where the data are nearly uniform the same ratios make the step's curvature
grow like 1/delta, delta the local variation: in the far field of a vortex
(delta ~ 1e-6) a perturbation of 1e-8 moves the GENO weights by O(1), and no
central difference above rounding is in the linear regime there.  The
derivative itself is exact and finite (the weights' changes multiply
differences of size delta), so the checks here use data without such
regions: seeded random smooth fields, and the vortex with the linear
reconstruction (GENO variant 2) and no |p_l - p_r| term in tau (whose kink
at p_l = p_r every smooth interface sits next to).
"""
import numpy as np
import pytest

import oracle
from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def dev(arrs):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs)


def run(solver, state, dt, n):
    solver.set_state(*dev(state))
    solver.steps(dt, n)
    return tuple(t.cpu().numpy() for t in solver.get_state())


def dot(a, b):
    return float(sum(np.vdot(x, y) for x, y in zip(a, b)))


CASES = {
    # periodic random smooth field, FD-CGKS(6-4), GENO blending active, large dt
    "periodic_geno": lambda: (inputs.random_smooth(15, 13, seed=40, amp=0.08, tau_c1=0.05, tau_c2=1.0), 0.03),
    # vortex, linear reconstruction, tau = c1 dt (no kinks anywhere)
    "vortex_15_linear": lambda: (inputs.vortex(15, strength=3.0, xc=4.37, yc=5.61, geno_variant=2, tau_c1=0.05,
                                               tau_c2=0.0), 0.05),
    # no-slip and symmetry walls, viscous: the wall reset and mirrored ghosts
    "walls_viscous": lambda: (inputs.random_smooth(13, 11, seed=41, amp=0.06, bc=(3, 3, 3, 2), mu=0.01,
                                                   Pr=0.73, tau_c2=1.0), 0.004),
    # the same with the linear reconstruction: after the first wall resets the
    # momenta next to a no-slip wall vary by little, which puts GENO's
    # curvature (above) out of reach of central differences on the 3-step map
    "walls_viscous_linear": lambda: (inputs.random_smooth(13, 11, seed=41, amp=0.06, bc=(3, 3, 3, 2), mu=0.01,
                                                          Pr=0.73, tau_c2=1.0, geno_variant=2), 0.004),
    # transmissive ends, 6-2 flux, App. D GENO constants, stored gradient base
    "transmissive_62_appD_A": lambda: (inputs.random_smooth(15, 6, seed=42, amp=0.08, bc=(1, 1, 0, 0),
                                                            flux_variant=62, geno_variant=1, grad_base=1,
                                                            tau_c1=0.05, tau_c2=1.0), 0.004),
    # symmetry everywhere, linear reconstruction, ragged sizes
    "symmetry_linear": lambda: (inputs.random_smooth(9, 12, seed=43, amp=0.05, bc=(2, 2, 2, 2), geno_variant=2,
                                                     tau_c1=0.05), 0.005),
}


@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_is_the_transpose_of_the_step(name, nsteps):
    if name == "walls_viscous" and nsteps > 1:
        pytest.skip("GENO near reset no-slip walls: see walls_viscous_linear")
    case, dt = CASES[name]()
    S0 = case.initial_state()
    rng = np.random.default_rng(7)
    v = [rng.standard_normal(a.shape) * (np.abs(a).max() + 1e-3) for a in S0]
    seed = [rng.standard_normal(a.shape) for a in S0]
    eps = 1e-8
    with fdcgks.Solver.from_case(case) as s:
        plus = run(s, [a + eps * b for a, b in zip(S0, v)], dt, nsteps)
        minus = run(s, [a - eps * b for a, b in zip(S0, v)], dt, nsteps)
        g = s.vjp_steps(dt, nsteps, dev(S0), dev(seed), checkpoint_every=2)
        g = [t.cpu().numpy() for t in g]
    fd = dot(seed, [(p - m) / (2 * eps) for p, m in zip(plus, minus)])
    ad = dot(g, v)
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-9, (ad, fd)


def test_checkpoint_interval_does_not_change_the_gradient():
    case, dt = CASES["walls_viscous"]()
    S0 = dev(case.initial_state())
    rng = np.random.default_rng(8)
    seed = dev([rng.standard_normal(a.shape) for a in case.initial_state()])
    grads = []
    with fdcgks.Solver.from_case(case) as s:
        for ck in (1, 2, 3, 7):
            grads.append([t.cpu().numpy() for t in s.vjp_steps(dt, 7, S0, seed, checkpoint_every=ck)])
        final = [t.cpu().numpy() for t in s.get_state()]
        ref = run(s, case.initial_state(), dt, 7)
    for a, b in zip(final, ref):
        assert np.array_equal(a, b)            # the context keeps the final state
    for g in grads[1:]:
        for a, b in zip(g, grads[0]):
            # the same arithmetic; only the order of atomic additions differs
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def objective(Wp, Wp_target, h2):
    return 0.5 * float(((Wp[0] - Wp_target[0]) ** 2).sum()) * h2


def test_objective_gradient_matches_oracle_differences():
    """J = 1/2 sum (rho - rho_target)^2 h^2 on the primary grid after 3 steps on a
    12^2 periodic smooth field, differentiated with respect to the primary W^0:
    the GPU adjoint against central differences of the CPU oracle along 4
    random directions (the oracle's gradient along them)."""
    case = inputs.random_smooth(12, 12, seed=44, amp=0.08, tau_c1=0.05, tau_c2=1.0)
    dt, n = 0.01, 3
    S0 = case.initial_state()
    p = oracle.make_params(**case.oracle_kwargs())
    rng = np.random.default_rng(3)
    target = oracle.steps(p, dt, n, *[a * (1 + 1e-3 * rng.standard_normal(a.shape)) for a in S0])
    h2 = case.hx * case.hy
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*dev(S0))
        s.steps(dt, n)
        Wp = s.get_state()[0].cpu().numpy()
        seed = [np.zeros_like(a) for a in S0]
        seed[0][0] = (Wp[0] - target[0][0]) * h2
        g = [t.cpu().numpy() for t in s.vjp_steps(dt, n, dev(S0), dev(seed), checkpoint_every=2)]
    for k in range(4):
        d = rng.standard_normal(S0[0].shape)
        d /= np.linalg.norm(d)
        eps = 1e-7                      # entries of eps d about 1e-8
        Jp = objective(oracle.steps(p, dt, n, S0[0] + eps * d, *S0[1:])[0], target[0], h2)
        Jm = objective(oracle.steps(p, dt, n, S0[0] - eps * d, *S0[1:])[0], target[0], h2)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.vdot(g[0], d))
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-14, (k, ad, fd)


def test_autograd_wrapper():
    case, dt = CASES["periodic_geno"]()
    S0 = dev(case.initial_state())
    with fdcgks.Solver.from_case(case) as s:
        Wp = S0[0].clone().requires_grad_(True)
        out = fdcgks.steps_autograd(s, Wp, S0[1], S0[2], S0[3], dt, 4, checkpoint_every=2)
        J = 0.5 * (out[0][0] ** 2).sum() + (out[2][3] * 0.1).sum()
        J.backward()
        seed = [torch.zeros_like(t) for t in S0]
        seed[0][0] = out[0][0].detach()
        seed[2][3] = 0.1
        ref = s.vjp_steps(dt, 4, S0, seed, checkpoint_every=4)
    assert torch.allclose(Wp.grad, ref[0], rtol=1e-10, atol=1e-14)


def test_adjoint_rejects_bad_arguments():
    case, dt = CASES["periodic_geno"]()
    S0 = dev(case.initial_state())
    with fdcgks.Solver.from_case(case) as s:
        for bad in (lambda: s.vjp_steps(-1.0, 1, S0, S0), lambda: s.vjp_steps(dt, 1, S0, S0, checkpoint_every=0)):
            with pytest.raises(fdcgks.FdcgksError) as e:
                bad()
            assert e.value.status == 1


# ---------------------------------------------------------------------------
# mixed-precision contexts: the mixed trajectory, the FP64 reverse pass


@pytest.mark.parametrize("ck", [1, 3])
def test_mixed_adjoint_keeps_the_mixed_run(ck):
    """The final state a mixed context keeps after the adjoint is the plain
    mixed run's to FP64 rounding: the trajectory is replayed through FP64
    buffers, where a float-float pair keeps its FP64 value but its low part
    can lose bits below 2^-53 of it (tests/test_float_float_host.py); on this
    case the two runs were found identical."""
    case, dt = CASES["periodic_geno"]()
    S0 = case.initial_state()
    rng = np.random.default_rng(9)
    seed = dev([rng.standard_normal(a.shape) for a in S0])
    with fdcgks.Solver.from_case(case, fdcgks.MIXED) as s:
        s.vjp_steps(dt, 5, dev(S0), seed, checkpoint_every=ck)
        kept = [t.cpu().numpy() for t in s.get_state()]
        ref = run(s, S0, dt, 5)
    for a, b in zip(kept, ref):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def _grad(case, prec, dt, S0, seed, n=3):
    with fdcgks.Solver.from_case(case, prec) as s:
        return [t.cpu().numpy() for t in s.vjp_steps(dt, n, dev(S0), seed, checkpoint_every=2)]


def _rel(a, b):
    return (np.sqrt(sum(float(((x - y) ** 2).sum()) for x, y in zip(a, b))) /
            np.sqrt(sum(float((y ** 2).sum()) for y in b)))


@pytest.mark.parametrize("name", ["vortex_15_linear", "walls_viscous_linear"])
def test_mixed_adjoint_is_close_to_the_fp64_adjoint(name):
    """With the linear reconstruction the step's Jacobian varies slowly with
    the state, so the FP64 reverse pass along the mixed trajectory gives the
    FP64 gradient to within 1e-6 relative in norm (2e-8 to 6e-8 measured)."""
    case, dt = CASES[name]()
    S0 = case.initial_state()
    rng = np.random.default_rng(10)
    seed = dev([rng.standard_normal(a.shape) for a in S0])
    d = _rel(_grad(case, fdcgks.MIXED, dt, S0, seed), _grad(case, fdcgks.FP64, dt, S0, seed))
    print("mixed vs FP64 adjoint, relative difference in norm:", name, d)
    assert d < 1e-6


def test_mixed_adjoint_with_geno_weights():
    """GENO's weights are steep functions of the data, so the gradient moves
    with the point it is taken at: the FP64 gradient at initial data changed
    by 1e-6 relative moves by a measured amount `sens`.  The mixed trajectory
    differs from the FP64 one by FP32 flux rounding and by the FP32 path's
    rounding floor in the smoothness indicators; its gradient stays within
    a few `sens` of the FP64 gradient (0.07 % apart measured)."""
    case, dt = CASES["periodic_geno"]()
    S0 = case.initial_state()
    rng = np.random.default_rng(10)
    seed = dev([rng.standard_normal(a.shape) for a in S0])
    g64 = _grad(case, fdcgks.FP64, dt, S0, seed)
    Sp = [a * (1 + 1e-6 * rng.standard_normal(a.shape)) for a in S0]
    sens = _rel(_grad(case, fdcgks.FP64, dt, Sp, seed), g64)
    d = _rel(_grad(case, fdcgks.MIXED, dt, S0, seed), g64)
    finals = []
    for prec in (fdcgks.FP64, fdcgks.MIXED):
        with fdcgks.Solver.from_case(case, prec) as s:
            finals.append(run(s, S0, dt, 3))
    print("GENO: mixed vs FP64 adjoint %.3g, FP64 gradient moved by a 1e-6 change of the data %.3g, "
          "trajectories %.3g apart" % (d, sens, _rel(finals[1], finals[0])))
    assert d < max(5 * sens, 1e-5) and d < 3e-3


def test_mixed_adjoint_against_differences_of_the_mixed_step():
    """Central differences of the mixed run itself (steps 1e-4 relative, where
    the differences are linear and well above the float-float state's
    rounding) against the mixed context's adjoint, on the vortex with the
    linear reconstruction: within 1e-3 relative, the FP32 rounding of the
    mixed map's fluxes."""
    case, dt = CASES["vortex_15_linear"]()
    S0 = case.initial_state()
    rng = np.random.default_rng(11)
    v = [rng.standard_normal(a.shape) * (np.abs(a).max() + 1e-3) for a in S0]
    seed = [rng.standard_normal(a.shape) for a in S0]
    eps = 1e-4
    with fdcgks.Solver.from_case(case, fdcgks.MIXED) as s:
        plus = run(s, [a + eps * b for a, b in zip(S0, v)], dt, 3)
        minus = run(s, [a - eps * b for a, b in zip(S0, v)], dt, 3)
        g = [t.cpu().numpy() for t in s.vjp_steps(dt, 3, dev(S0), dev(seed), checkpoint_every=2)]
    fd = dot(seed, [(p - m) / (2 * eps) for p, m in zip(plus, minus)])
    ad = dot(g, v)
    print("mixed adjoint against mixed differences:", ad, fd, abs(ad - fd) / abs(fd))
    assert abs(ad - fd) <= 1e-3 * abs(fd), (ad, fd)



def test_mixed_adjoint_takes_the_rounding_floor():
    """The mixed context's reverse pass linearises GENO with the FP32 path's
    rounding floor (its reverse functions are checked against dual numbers of
    the floored function on the host, tests/test_adjoint_host.py).  Through
    the C ABI on a 32^2 vortex over 3 steps: for a direction confined to the
    far field (r > 4.5), where the data vary below the floor, the floored
    linearisation differs from the FP64 one by more than 10 %; for a direction
    in the core (r < 2), where they vary far above it, the two agree to 1e-3.
    Central differences of the mixed run itself cannot decide between the two
    in the far field: at steps small enough to stay below the floor they
    scatter by a factor of about 2 with the run's FP32 rounding (printed)."""
    case = inputs.vortex(32)
    S0 = case.initial_state()
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*S0)
        dt = s.cfl_dt(0.2)
    X, Y = case.node_xy(False)
    r = np.hypot(X - 5.0, Y - 5.0)
    rng = np.random.default_rng(3)
    seed = [rng.standard_normal(a.shape) for a in S0]
    scale = np.abs(S0[0]).max(axis=(1, 2))[:, None, None]
    dirs = {}
    for name, mask in (("far", r > 4.5), ("core", r < 2.0)):
        v = [np.zeros_like(a) for a in S0]
        v[0] = rng.standard_normal(S0[0].shape) * mask[None] * scale
        dirs[name] = v
    n = 3
    ad = {}
    for prec in (fdcgks.FP64, fdcgks.MIXED):
        with fdcgks.Solver.from_case(case, prec) as s:
            g = [t.cpu().numpy() for t in s.vjp_steps(dt, n, dev(S0), dev(seed), checkpoint_every=2)]
            ad[prec] = {k: dot(g, v) for k, v in dirs.items()}
            if prec == fdcgks.MIXED:
                fds = []
                v = dirs["far"]
                for eps in (1e-5, 3e-6, 1e-6, 3e-7, 1e-7):
                    p = run(s, [a + eps * b for a, b in zip(S0, v)], dt, n)
                    m = run(s, [a - eps * b for a, b in zip(S0, v)], dt, n)
                    fds.append(dot(seed, [(x - y) / (2 * eps) for x, y in zip(p, m)]))
    print("far field: mixed-run differences", fds, "mixed adjoint", ad[fdcgks.MIXED]["far"],
          "FP64 adjoint", ad[fdcgks.FP64]["far"])
    far64, farmx = ad[fdcgks.FP64]["far"], ad[fdcgks.MIXED]["far"]
    assert abs(farmx - far64) > 0.1 * abs(far64), (farmx, far64)
    core64, coremx = ad[fdcgks.FP64]["core"], ad[fdcgks.MIXED]["core"]
    assert abs(coremx - core64) < 1e-3 * abs(core64), (coremx, core64)
