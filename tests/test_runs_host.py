"""Host-side logic of the run driver (paper_2606_17772_gb300.runs.advance),
with a fake solver in place of the library: CFL steps until the final time,
the last step clipped onto it, positivity checked periodically and at the
end (no GPU involved)."""
import pytest

from paper_2606_17772_gb300 import runs


class FakeSolver:
    def __init__(self, dts, bad_after=None):
        self.dts = list(dts)
        self.k = 0
        self.t = 0.0
        self.taken = []
        self.bad_after = bad_after

    def cfl_dt(self, cfl):
        dt = self.dts[min(self.k, len(self.dts) - 1)] * cfl / 0.4
        return dt

    def step(self, dt):
        self.taken.append(dt)
        self.t += dt
        self.k += 1

    def check(self):
        return self.bad_after is not None and self.k > self.bad_after


def test_last_step_lands_on_the_final_time():
    s = FakeSolver([0.03])
    t, n = runs.advance(s, 0.1, 0.4)
    assert n == 4 and s.taken[:3] == [0.03] * 3
    assert s.taken[3] == pytest.approx(0.01)
    assert t == pytest.approx(0.1, rel=1e-15)


def test_time_step_follows_the_solver_and_the_cfl_number():
    s = FakeSolver([0.02, 0.01, 0.05])
    t, n = runs.advance(s, 0.1, 0.2)          # half the steps of CFL 0.4
    assert s.taken[:3] == pytest.approx([0.01, 0.005, 0.025])
    assert t == pytest.approx(0.1) and sum(s.taken) == pytest.approx(0.1)


def test_nonphysical_state_raises_with_time_and_step():
    s = FakeSolver([0.001], bad_after=5)
    with pytest.raises(RuntimeError, match="non-physical state at t = .* after 10 steps"):
        runs.advance(s, 1.0, 0.4, check_every=10)


def test_start_time_and_no_steps_when_already_there():
    s = FakeSolver([0.01])
    t, n = runs.advance(s, 0.5, 0.4, t0=0.5)
    assert n == 0 and t == 0.5 and s.taken == []
