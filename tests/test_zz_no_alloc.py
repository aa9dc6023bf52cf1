"""The allocation-free CFL entry point against the context-based one.

fdcgks_cfl_dt_noalloc serves callers that cannot allocate device memory when
they need a time step (an application that gives the library a fixed share of
the GPU's memory, a time loop that must not risk an allocation failure or the
synchronisation of cudaMalloc/cudaFree); it keeps its partial maxima in a fixed
device array of the library.  Its result must equal fdcgks_cfl_dt's on the
same state, on consecutive calls (the shared array keeps the previous call's
contents: a larger rate or more tiles left by one call must not reach the
next), and grids beyond its stated limit must be refused.  This file is
collected last.
"""
import numpy as np
import pytest

from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _context_dt(case, S, cfl):
    with fdcgks.Solver.from_case(case) as s:
        s.set_state(*[torch.from_numpy(a).cuda() for a in S])
        return s.cfl_dt(cfl)


@pytest.mark.parametrize("name", ["vortex_64", "viscous_tube_40x20", "sod_strip_50x3"])
def test_noalloc_cfl_equals_context_cfl_on_consecutive_calls(name):
    case = {"vortex_64": lambda: inputs.vortex(64), "viscous_tube_40x20": lambda: inputs.viscous_shock_tube(40, 20),
            "sod_strip_50x3": lambda: inputs.sod_strip(50, 3)}[name]()
    cfl = 0.37
    S = case.initial_state()
    # a second, different state: the scratch must not carry the first call's maxima over
    S2 = [a.copy() for a in S]
    S2[0][1] *= 1.5
    S2[0][3] += 0.5 * (S2[0][1] ** 2 - S[0][1] ** 2) / S2[0][0]
    params = fdcgks.params_for_case(case)
    # S2 has the larger wave rate: run it both before and after S
    for state in (S, S, S2, S2, S, S2, S):
        ref = _context_dt(case, state, cfl)
        Wp = torch.from_numpy(state[0]).cuda()
        Wd = torch.from_numpy(state[2]).cuda()
        got = fdcgks.cfl_dt_noalloc(params, Wp, Wd, cfl)
        assert got == pytest.approx(ref, rel=1e-12)


def test_noalloc_cfl_after_a_larger_grid():
    """A multi-tile call with a fast state, then a one-tile call with a slow
    one: the second must see neither the first's tiles nor its maxima."""
    cfl = 0.4
    big = inputs.vortex(96, strength=5.0)          # 2 * 96^2 nodes: 5 tiles
    small = inputs.vortex(16, strength=1.0)        # 512 nodes: 1 tile
    Sb, Ss = big.initial_state(), small.initial_state()
    Sb[0][1] *= 3.0                                # faster flow in the big grid
    Sb[0][3] += 0.5 * (Sb[0][1] ** 2 - (Sb[0][1] / 3.0) ** 2) / Sb[0][0]
    pb, ps = fdcgks.params_for_case(big), fdcgks.params_for_case(small)
    for case, S, prm in ((big, Sb, pb), (small, Ss, ps), (big, Sb, pb), (small, Ss, ps)):
        got = fdcgks.cfl_dt_noalloc(prm, torch.from_numpy(S[0]).cuda(), torch.from_numpy(S[2]).cuda(), cfl)
        assert got == pytest.approx(_context_dt(case, S, cfl), rel=1e-12)


def test_noalloc_cfl_rejects_grids_beyond_its_limit():
    n = 4096     # 2 * 4096^2 nodes > 4096 tiles x 4096 nodes
    params = fdcgks.make_params(n, n)
    small = torch.ones((4, 2, 2), dtype=torch.float64, device="cuda")
    lib = fdcgks.load()
    out = fdcgks.ctypes.c_double()
    st = lib.fdcgks_cfl_dt_noalloc(fdcgks.ctypes.byref(params), fdcgks.ctypes.c_void_p(small.data_ptr()),
                                   fdcgks.ctypes.c_void_p(small.data_ptr()), fdcgks.ctypes.c_double(0.4),
                                   fdcgks.ctypes.byref(out))
    assert st == 1
    assert "allocation-free limit" in lib.fdcgks_last_error(None).decode()
