"""The CFL time step of a context (fdcgks_cfl_dt, fdcgks_cfl_dt_sum) against
the oracle's all-node FP64 evaluation (Sec. 5 time step), for both
precisions and both forms of the bound.

The library screens the nodes with FP32 estimates of the rates and evaluates
in FP64 only those that can hold the maxima, so the step must equal the
all-node FP64 value to rounding on every case, including cases built to
defeat a wrong screening: rates tied to 1e-9 over the whole grid, the
largest rate at a node whose FP32 estimate is unreliable (Mach 250, p/E ~
1e-5), a second node within 1e-7 of the largest, and steps that the
viscous limit decides.  The mixed context is compared on its own state (the
float-float pairs joined), which get_state returns.
"""
import pytest

import oracle
from cfl_cases import cases
from paper_2606_17772_gb300 import fdcgks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = cases()


@pytest.mark.parametrize("form", ["direction", "sum"])
@pytest.mark.parametrize("precision", [fdcgks.FP64, fdcgks.MIXED])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_cfl_step_equals_all_node_fp64(k, precision, form):
    name, case, S = CASES[k]
    p = oracle.make_params(**case.oracle_kwargs())
    ref_fn = oracle.cfl_dt if form == "direction" else oracle.cfl_dt_sum
    with fdcgks.Solver.from_case(case, precision) as s:
        s.set_state(*S)
        got = s.cfl_dt(0.37, form=form)
        St = s.get_state(device=False)
    ref = ref_fn(p, 0.37, St[0], St[2])
    assert got == pytest.approx(ref, rel=1e-14), (name, got, ref)
