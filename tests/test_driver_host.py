"""Host logic of the adaptive load stepping (no GPU): the step controller of
LoadStepper.advance halves a failing increment, regrows it after successes,
never passes the target and gives up after the allowed number of cuts."""
import pytest

from paper_2607_21150_gb300.driver import StepController, StepFailed


def _run(limit, start=0.0, target=1.0, max_cuts=6):
    tried = []

    def attempt(f0, f1):
        tried.append((f0, f1))
        return f1 - f0 <= limit

    done = StepController(max_cuts=max_cuts).run(start, target, attempt)
    return done, tried


def test_no_cut_when_the_step_converges():
    done, tried = _run(limit=1.0)
    assert done == [(0.0, 1.0)] and tried == [(0.0, 1.0)]


def test_halving_and_regrowth():
    done, tried = _run(limit=0.3)
    assert tried == [(0.0, 1.0), (0.0, 0.5), (0.0, 0.25), (0.25, 0.75), (0.25, 0.5), (0.5, 1.0), (0.5, 0.75),
                     (0.75, 1.0)]
    assert done == [(0.0, 0.25), (0.25, 0.5), (0.5, 0.75), (0.75, 1.0)]


def test_sub_steps_tile_the_interval_exactly():
    done, _ = _run(limit=0.2, start=3.0, target=4.0)
    assert done[0][0] == 3.0 and done[-1][1] == 4.0
    assert all(a[1] == b[0] for a, b in zip(done, done[1:]))
    assert all(f1 - f0 <= 0.2 for f0, f1 in done)


def test_gives_up_after_max_cuts():
    with pytest.raises(StepFailed):
        _run(limit=1e-3, max_cuts=4)


def test_state_stays_at_the_last_converged_factor():
    state = {"f": 0.0}

    def attempt(f0, f1):
        assert f0 == state["f"]  # every attempt starts from the last converged factor
        if f1 - f0 > 0.4:
            return False
        state["f"] = f1
        return True

    StepController().run(0.0, 2.0, attempt)
    assert state["f"] == 2.0
