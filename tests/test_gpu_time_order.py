"""Temporal order of the two-dimensional scheme on the GPU (a property that
holds at any size, measured where the CPU oracle cannot go).

The nodal values advance by S2O4 (Eq. eq-nodal-update) and the averaged
gradients by the two-stage midpoint form of Eq. eq-interface-update, whose
local error is O(dt^3).  With the gradient base re-evaluated every step (the
default reading) that error does not accumulate, and nodal values and
gradients converge at third order in dt at fixed h; with the stored base the
gradients converge at second order.  The 1-D oracle pins the same analysis
(tests/test_oracle_line.py); here the 2-D density wave of Sec. 5.1 at 64^2
(both grids, tau = 0, where the kinetic flux is linear in t) is run to
t = 0.5 with 100, 200 and 400 steps against a 3200-step run on the same grid,
so the spatial error cancels.  Measured on a GB300: error ratios per halving
7.99, 8.00 (nodal values) and 7.94, 7.98 (gradients) with the re-evaluated
base; 3.66, 3.85 (gradients) with the stored base.
"""
import numpy as np
import pytest

from paper_2606_17772_gb300 import fdcgks, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _errors(grad_base, n=64, T=0.5, Ns=(100, 200, 400), Nref=3200):
    case = inputs.density_wave_2d(n, grad_base=grad_base)
    S0 = case.initial_state()
    out = {}
    with fdcgks.Solver.from_case(case) as s:
        for N in Ns + (Nref,):
            s.set_state(*S0)
            s.steps(T / N, N)
            out[N] = s.get_state(device=False)
            assert not s.check()
    eW = [np.abs(out[N][0] - out[Nref][0]).max() for N in Ns]
    eG = [np.abs(out[N][1] - out[Nref][1]).max() for N in Ns]
    return eW, eG


def test_third_order_in_time_with_the_re_evaluated_gradient_base():
    eW, eG = _errors(0)
    print("re-evaluated base: W", eW, "ratios", [a / b for a, b in zip(eW, eW[1:])],
          "gradients", eG, "ratios", [a / b for a, b in zip(eG, eG[1:])])
    for e in (eW, eG):
        for a, b in zip(e, e[1:]):
            assert 6.5 < a / b < 9.5, e


def test_second_order_gradients_with_the_stored_gradient_base():
    eW, eG = _errors(1)
    print("stored base: W", eW, "ratios", [a / b for a, b in zip(eW, eW[1:])],
          "gradients", eG, "ratios", [a / b for a, b in zip(eG, eG[1:])])
    for a, b in zip(eG, eG[1:]):
        assert 3.3 < a / b < 4.7, eG
