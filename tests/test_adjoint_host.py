"""Host logic of the differentiable reaction curve, without a GPU: a fake load
stepper and fake library calls stand in for the device work.

* forward records every converged sub-step (state after, history before, time
  step, end load factor) and the schedule of sub-step ends per load step, and
  replays a given schedule;
* backward walks the sub-steps in reverse, sets each one's time step before
  its adjoint step, gives the reaction weight dL/dF_n only to the sub-step that
  ends load step n (zero to the others), and chains the history adjoint: none
  for the last sub-step, then the previous step's output.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_21150_gb300 import adjoint, inputs  # noqa: E402


class _FakeSession:
    dev = torch.device("cpu")
    ctx = "ctx"
    stream = None


class _FakeStepper:
    """Sub-step ends: the given schedule, else load step 2 in two halves."""
    instances = []

    def __init__(self, w, **kw):
        self.s = _FakeSession()
        self.solver = "solver"
        self.z = torch.zeros(4)
        self.on_substep = None
        self.dt = 0.01
        self.f = 0.0
        self.schedules = []
        _FakeStepper.instances.append(self)

    def advance(self, k, schedule=None):
        self.schedules.append(schedule)
        ends = schedule if schedule is not None else ([k - 0.5, k] if k == 2 else [k])
        out = []
        for f1 in ends:
            dt = self.dt * (f1 - self.f)
            hist_before = torch.full((3,), self.f)
            self.z = torch.full((4,), f1)
            self.on_substep(self.f, f1, dt, hist_before, {})
            out.append({"load": f1, "reaction": 10.0 * f1})
            self.f = f1
        return out

    def close(self):
        pass


def test_forward_records_and_backward_replays(monkeypatch):
    calls = []
    state = {"dt": None}
    monkeypatch.setattr(adjoint, "LoadStepper", _FakeStepper)
    monkeypatch.setattr(adjoint.pff, "pff_context_set_time_step", lambda ctx, dt: state.update(dt=dt))

    def fake_step(solver, z, h, sel, wF, hbar, hb_prev, grad, rtol, maxit, stream):
        calls.append(dict(f1=float(z[0]), h0=float(h[0]), wF=wF, dt=state["dt"],
                          hbar=None if hbar is None else hbar.clone(), n=len(calls)))
        hb_prev.fill_(float(len(calls)))      # this step's history adjoint output
        grad += 1.0
        return 7

    monkeypatch.setattr(adjoint.pff, "pff_adjoint_step", fake_step)
    w = inputs.cube(nx=2, p=2)
    runner = adjoint.ReactionCurveRunner(w, nsteps=3)
    theta = inputs.params_of(w.phases)
    F = runner.forward(theta)
    assert np.allclose(F, [10.0, 20.0, 30.0])
    assert runner.schedule == [[1], [1.5, 2], [3]]
    assert [s["f1"] for s in runner.subs] == [1, 1.5, 2, 3]
    dLdF = np.array([0.1, 0.2, 0.3])
    g = runner.backward(dLdF)
    assert [c["f1"] for c in calls] == [3.0, 2.0, 1.5, 1.0]
    assert [c["h0"] for c in calls] == [2.0, 1.5, 1.0, 0.0]          # history entering each sub-step
    assert [c["wF"] for c in calls] == [0.3, 0.2, 0.0, 0.1]          # weight only where a load step ends
    assert np.allclose([c["dt"] for c in calls], [0.01, 0.005, 0.005, 0.01])
    assert calls[0]["hbar"] is None
    for k in range(1, 4):                                            # chained history adjoint
        assert torch.all(calls[k]["hbar"] == float(k))
    assert np.all(g == 4.0) and runner.adjoint_iters == [7, 7, 7, 7]
    # a recorded schedule is replayed as given
    runner.forward(theta, schedule=runner.schedule)
    assert _FakeStepper.instances[-1].schedules == [[1], [1.5, 2], [3]]
    runner.close()


def test_backward_of_a_replaced_forward_run_raises(monkeypatch):
    """Two ReactionCurve graphs on one runner: the second forward replaces the
    checkpoints, so the first graph's backward must raise instead of returning
    the gradient of the second run; the second graph's backward works."""
    monkeypatch.setattr(adjoint, "LoadStepper", _FakeStepper)
    monkeypatch.setattr(adjoint.pff, "pff_context_set_time_step", lambda ctx, dt: None)

    def fake_step(solver, z, h, sel, wF, hbar, hb_prev, grad, rtol, maxit, stream):
        grad += wF
        return 1

    monkeypatch.setattr(adjoint.pff, "pff_adjoint_step", fake_step)
    w = inputs.cube(nx=2, p=2)
    runner = adjoint.ReactionCurveRunner(w, nsteps=2)
    th = torch.tensor(inputs.params_of(w.phases), dtype=torch.float64, requires_grad=True)
    F1 = adjoint.ReactionCurve.apply(th, runner)
    F2 = adjoint.ReactionCurve.apply(th * 1.0, runner)
    with pytest.raises(adjoint.StaleCheckpoints):
        F1.sum().backward()
    F2.sum().backward()
    assert torch.all(th.grad == 2.0)          # dL/dF = 1 at both load-step ends
    runner.close()
    with pytest.raises(adjoint.StaleCheckpoints):
        runner.backward(np.ones(2))
