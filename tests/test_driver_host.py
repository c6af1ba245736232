"""Host logic of the adaptive load stepping (no GPU): the step controller of
LoadStepper.advance halves a failing increment, regrows it after successes,
never passes the target and gives up after the allowed number of cuts; and,
with a fake session and fake library calls, what LoadStepper.advance does
around the device work."""
import numpy as np
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


# ---------------------------------------------------------------------------
# LoadStepper.advance with a fake session and fake library calls: what the
# stepper does around the device work (time step per sub-step, predictor,
# undo of a failed sub-step, commit only after convergence, callbacks, replay).
# ---------------------------------------------------------------------------
class _FakeSession:
    def __init__(self, w):
        import torch
        self.w = w
        self.dev = torch.device("cpu")
        self.ctx = "ctx"
        self.op = "op"
        self.mask = None
        self.stream = None
        self.hist = torch.zeros(3)

    def solver(self, levels, **params):
        return "solver"

    def history(self, which=0):
        return self.hist

    def close(self):
        pass


def _fake_library(monkeypatch, limit, device_error_above=None):
    import torch
    from paper_2607_21150_gb300 import driver
    log = {"dt": [], "commits": 0, "solves": []}

    def set_dt(ctx, dt):
        log["dt"].append(dt)

    def axpby(prec, n, a, x, b, y, stream=None):
        y.mul_(b).add_(a * x)

    def newton(solver, z, stream=None):
        f0, f1 = log["from"], log["to"]
        log["solves"].append((f0, f1))
        if device_error_above is not None and f1 - f0 > device_error_above:
            z.add_(1e6)
            raise driver.pff.PffError("no admissible step", driver.pff.ERR_DEVICE)
        ok = f1 - f0 <= limit
        z.add_(1e6 if not ok else 0.0)          # a failed solve leaves garbage behind
        return {"converged": int(ok), "status": 0, "newton_iterations": 3, "krylov_iterations": 9}

    def commit(op, stream=None):
        log["commits"] += 1

    monkeypatch.setattr(driver.pff, "pff_context_set_time_step", set_dt)
    monkeypatch.setattr(driver.pff, "pff_vec_axpby", axpby)
    monkeypatch.setattr(driver.pff, "pff_set_dirichlet", lambda *a, **k: None)
    monkeypatch.setattr(driver.pff, "pff_apply_dirichlet", lambda *a, **k: None)
    monkeypatch.setattr(driver.pff, "pff_newton_solve", newton)
    monkeypatch.setattr(driver.pff, "pff_commit_history", commit)
    monkeypatch.setattr(driver.pff, "pff_reaction", lambda op, top, stream=None: [0.0, 0.0, 5.0 * log["to"], 0.0])
    return log


def _stepper(monkeypatch, limit, **kw):
    from paper_2607_21150_gb300 import inputs
    from paper_2607_21150_gb300.driver import LoadStepper
    w = inputs.cube(nx=2, p=2)
    w.mask, w.dvals = inputs.dirichlet_tension(w.mesh, 1e-3)
    log = _fake_library(monkeypatch, limit, **kw)
    lsp = LoadStepper(w, session=_FakeSession(w))
    orig = lsp._solve_to

    def solve_to(factor, dt):        # remember the sub-step the fake Newton works on
        log["from"], log["to"] = lsp.loaded, factor
        return orig(factor, dt)

    lsp._solve_to = solve_to
    return lsp, log, w


def test_advance_cuts_back_and_undoes_failed_substeps(monkeypatch):
    import torch
    lsp, log, w = _stepper(monkeypatch, limit=0.3)
    seen = []
    lsp.on_substep = lambda f0, f1, dt, h, st: seen.append((f0, f1, dt))
    z0 = lsp.z.clone()
    out = lsp.advance(1)
    ends = [st["load"] for st in out]
    assert ends == [0.25, 0.5, 0.75, 1.0]
    assert log["commits"] == 4                                   # failed attempts never commit
    dt0 = float(w.glob[3])
    assert [s[2] for s in seen] == [0.25 * dt0] * 4
    assert [(s[0], s[1]) for s in seen] == [(0.0, 0.25), (0.25, 0.5), (0.5, 0.75), (0.75, 1.0)]
    # every attempt's time step is its increment times the nominal one
    assert np.allclose(log["dt"], [dt0 * (b - a) for a, b in log["solves"]])
    # z = start + the predictor of the converged increments only (failed solves undone)
    assert torch.allclose(lsp.z, z0 + 1.0 * lsp.extension)
    assert out[-1]["reaction"] == 5.0 and lsp.loaded == 1.0


def test_device_error_counts_as_a_failed_substep(monkeypatch):
    import torch
    lsp, log, w = _stepper(monkeypatch, limit=1.0, device_error_above=0.5)
    z0 = lsp.z.clone()
    out = lsp.advance(1)
    assert [st["load"] for st in out] == [0.5, 1.0]
    assert torch.allclose(lsp.z, z0 + lsp.extension)


def test_replayed_schedule_must_converge_and_end_at_the_target(monkeypatch):
    from paper_2607_21150_gb300.driver import StepFailed
    lsp, log, w = _stepper(monkeypatch, limit=0.3)
    out = lsp.advance(1, schedule=[0.25, 0.5, 0.75, 1.0])
    assert [st["load"] for st in out] == [0.25, 0.5, 0.75, 1.0]
    assert log["solves"] == [(0.0, 0.25), (0.25, 0.5), (0.5, 0.75), (0.75, 1.0)]   # no cut-back in a replay
    with pytest.raises(StepFailed, match="did not converge"):
        lsp.advance(2, schedule=[2.0])
    lsp2, _, _ = _stepper(monkeypatch, limit=1.0)
    with pytest.raises(StepFailed, match="schedule ends"):
        lsp2.advance(1, schedule=[0.5])


def test_checkpoint_round_trip(monkeypatch, tmp_path):
    """save_checkpoint writes z, the committed history, the phase map, the load
    factor and the log; load_checkpoint on a fresh stepper restores them (the
    history through the session, the Dirichlet values of the load factor) and
    refuses a checkpoint of another microstructure."""
    import torch
    lsp, log, w = _stepper(monkeypatch, limit=1.0)
    lsp.s.hist = torch.arange(15 * w.mesh.nq, dtype=torch.float64).view(15, -1)
    lsp.advance(1)
    lsp.advance(2)
    lsp.save_checkpoint(str(tmp_path / "ck"), {"step": 2})
    lsp2, log2, _ = _stepper(monkeypatch, limit=1.0)
    got = {}
    lsp2.s.set_history = lambda h: got.update(hist=np.array(h))
    loads = []
    lsp2.set_load = lambda f: loads.append(f)
    info = lsp2.load_checkpoint(str(tmp_path / "ck"))
    assert info["step"] == 2 and info["loaded"] == 2.0 and len(info["log"]) == 2
    assert lsp2.loaded == 2.0 and loads == [2.0]
    assert torch.equal(lsp2.z, lsp.z)
    assert np.array_equal(got["hist"], lsp.s.hist.numpy())
    lsp3, _, _ = _stepper(monkeypatch, limit=1.0)
    lsp3.w.phase = lsp3.w.phase.copy()
    lsp3.w.phase[0] ^= 1
    with pytest.raises(ValueError, match="microstructure"):
        lsp3.load_checkpoint(str(tmp_path / "ck"))


def test_failed_substeps_are_recorded(monkeypatch):
    lsp, log, w = _stepper(monkeypatch, limit=0.3)
    lsp.advance(1)
    fails = [(f["from"], f["to"]) for f in lsp.failures]
    assert fails[:2] == [(0.0, 1.0), (0.0, 0.5)]
    assert all(b - a > 0.3 for a, b in fails) and all(f["converged"] == 0 for f in lsp.failures)
    assert len(fails) + len(lsp.history) == len(log["solves"])


def test_controller_grows_only_after_repeated_successes():
    """grow_after = 2: after a cut the increment stays at its halved size for
    two converged sub-steps before it doubles; with grow_after = 1 (the
    default) it doubles after every success."""
    from paper_2607_21150_gb300.driver import StepController

    def run(grow_after):
        tried = []

        def attempt(f0, f1):
            tried.append((f0, f1))
            return f1 - f0 <= 0.25
        done = StepController(grow_after=grow_after).run(0.0, 2.0, attempt)
        return tried, done

    t1, d1 = run(1)
    t2, d2 = run(2)
    assert [b for _, b in d1] == [b for _, b in d2] == [0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0]
    fails1 = [x for x in t1 if x[1] - x[0] > 0.25]
    fails2 = [x for x in t2 if x[1] - x[0] > 0.25]
    assert len(fails2) < len(fails1)
    assert t2[:5] == [(0.0, 2.0), (0.0, 1.0), (0.0, 0.5), (0.0, 0.25), (0.25, 0.5)]
    assert t2[5] == (0.5, 1.0)        # grows only after the second success
