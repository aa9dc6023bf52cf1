"""Host-side checks of the CFL test cases (tests/cfl_cases.py) with the
oracle alone: the planted nodes and the viscous limit really decide the
step, so that the GPU test (tests/test_gpu_cfl.py) exercises the screening
paths it names."""
import numpy as np
import pytest

import oracle
from cfl_cases import cases, planted


def test_planted_cases_decide_the_step():
    """The planted nodes hold the maxima: without them the step is larger."""
    for kind in ("unreliable", "near_tie"):
        case, S = planted(kind)
        p = oracle.make_params(**case.oracle_kwargs())
        base = case.initial_state()
        with_node = oracle.cfl_dt(p, 0.37, S[0], S[2])
        assert with_node < oracle.cfl_dt(p, 0.37, base[0], base[2]) * 0.9, kind
    case, S = planted("near_tie")
    p = oracle.make_params(**case.oracle_kwargs())
    S2 = [a.copy() for a in S]
    S2[2][:, 17, 30] = S[2][:, 5, 7]                 # drop the larger of the tied pair
    assert oracle.cfl_dt(p, 0.37, S2[0], S2[2]) > oracle.cfl_dt(p, 0.37, S[0], S[2]) * (1 + 5e-8)


def test_viscous_limit_decides_the_step():
    """mu = 0.5 on a 30 x 20 grid: dt = cfl h^2 / (8 max nu), below cfl/rate."""
    _, case, S = next(c for c in cases() if c[1].mu > 0 and c[1].name == "random_smooth")
    p = oracle.make_params(**case.oracle_kwargs())
    W = np.concatenate([S[0].reshape(4, -1), S[2].reshape(4, -1)], axis=1)
    h = min(case.hx, case.hy)
    nu = 0.5 / W[0]
    assert oracle.cfl_dt(p, 0.37, S[0], S[2]) == pytest.approx(0.37 * h * h / (8 * nu.max()), rel=1e-14)
