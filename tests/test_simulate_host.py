"""The load-stepping command line without a GPU: a fake load stepper stands in
for the device solver.  One JSON line per load step with the last sub-step's
reaction and the summed iteration counts, a summary line, the --fp64 switch,
and a clean stop (status line, exit 0) when a load step cannot be completed."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2607_21150_gb300 import driver, simulate  # noqa: E402


class _Fake:
    made = []

    def __init__(self, w, mixed=True, max_cuts=6, grow_after=1, **kw):
        self.mixed, self.max_cuts, self.grow_after, self.kw = mixed, max_cuts, grow_after, kw
        self.history = []
        self.failures = []
        _Fake.made.append(self)

    def advance(self, k):
        if k == 3:
            raise driver.StepFailed("no convergence from load factor 2.0 after 6 cuts")
        subs = [{"load": k - 0.5, "reaction": 1.0, "newton_iterations": 4, "krylov_iterations": 20},
                {"load": k, "reaction": 2.0 * k, "newton_iterations": 3, "krylov_iterations": 15}]
        self.history += subs
        return subs

    def close(self):
        pass


def test_cli_lines_and_clean_stop(monkeypatch, capsys):
    monkeypatch.setattr(driver, "LoadStepper", _Fake)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    rc = simulate.main(["--workload", "tension_q4", "--n", "2", "--steps", "5", "--fp64", "--max-cuts", "3"])
    assert rc == 0
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines() if x.startswith("{")]
    head, steps, tail = lines[0], lines[1:-1], lines[-1]
    assert head["workload"] == "tension_q4" and head["steps"] == 5 and head["mixed"] is False
    assert [s["step"] for s in steps] == [1, 2]
    assert steps[1]["reaction"] == 4.0 and steps[1]["sub_steps"] == 2
    assert steps[1]["newton_iterations"] == 7 and steps[1]["krylov_iterations"] == 35
    assert tail["status"].startswith("stopped at step 3") and tail["attempts"] == 4
    assert _Fake.made[-1].mixed is False and _Fake.made[-1].max_cuts == 3


def test_cli_solver_parameters(monkeypatch, capsys):
    monkeypatch.setattr(driver, "LoadStepper", _Fake)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    rc = simulate.main(["--workload", "tension_q4", "--n", "2", "--steps", "1", "--verbose",
                        "--param", "cheb_degree=6", "--param", "krylov_rtol=1e-4", "--param", "eig_every=0"])
    assert rc == 0
    kw = _Fake.made[-1].kw
    assert kw == {"cheb_degree": 6, "krylov_rtol": 1e-4, "eig_every": 0, "verbose": 1}
    assert isinstance(kw["cheb_degree"], int) and isinstance(kw["krylov_rtol"], float)
    head = json.loads(capsys.readouterr().out.splitlines()[0])
    assert head["solver_params"]["cheb_degree"] == 6
    with pytest.raises(SystemExit):
        simulate.main(["--workload", "tension_q4", "--n", "2", "--param", "no_such=1"])
