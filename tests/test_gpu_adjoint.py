"""Discrete adjoint on the GPU vs the oracle's assembled-transpose adjoint and
central finite differences.

Three load steps of a two-phase Q2 tension box (history carried between
steps): the GPU reactions equal the oracle's (1e-9), the adjoint gradient of the
reaction-curve misfit equals the oracle's (1e-9 relative per component, plus
1e-11 of the largest |dL/dtheta_j theta_j| / |theta_i| for components that
vanish) and central differences of the GPU loss in all twelve parameters
(1e-6, plus 1e-9 of the same scale), and torch autograd through
ReactionCurve returns the same gradient.  The forward Newton solves run to
1e-12, their linear solves to 1e-10 and the adjoint solves to 1e-12 (measured
on a GB300: largest component deviation from the oracle 3e-11 at these
tolerances, 2.5e-10 at the runner's defaults 1e-11 / 1e-8 / 1e-10).

Second variant: hardening Prandtl branches (linear + Voce, test values) with
a live accumulated plastic strain, so that the return map's implicit
derivatives and the history word eps_p enter the adjoint.  Third variant: a
curved mesh (mapped geometry).
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_21150_gb300.adjoint import ReactionCurve, ReactionCurveRunner  # noqa: E402


def _adjoint_box():
    w = inputs.adjoint_q2(n=2)
    w.mesh = inputs.Mesh(2, 2, 2, 2, 3, w.mesh.L)
    return w


def _hardened_box():
    w = _adjoint_box()
    rows = inputs.harden(w.phases, 0.0, 0.0, 0.0)
    rows[0, 11] = 300.0                       # matrix yields within the three steps
    rows[:, 12] = 2000.0                      # H_lin
    rows[:, 13] = 1.6 * rows[:, 11]           # sigma_inf
    rows[:, 14] = 40.0                        # beta
    w.phases = rows
    w.hist[12] = np.random.default_rng(8).uniform(0.0, 0.02, w.mesh.nq)
    return w


def _mapped_box():
    w = _adjoint_box()
    w.X = inputs.mapped_coords(w.mesh, "smooth", amp=0.15)
    return w


@pytest.fixture(scope="module", params=["perfect", "hardening", "mapped"])
def problem(orc, request):
    w = {"perfect": _adjoint_box, "hardening": _hardened_box, "mapped": _mapped_box}[request.param]()
    top = inputs.top_face_mask(w.mesh)
    theta0 = inputs.params_of(w.phases)
    nsteps = 3
    target, _, _ = orc.load_steps(w, inputs.twin_target(theta0), nsteps, top)
    g_ref, F_ref = orc.adjoint_gradient(w, theta0, nsteps, top, target)
    runner = ReactionCurveRunner(w, nsteps, levels=[2, 1], newton_rtol=1e-12, krylov_rtol=1e-10, adjoint_rtol=1e-12)
    return w, theta0, nsteps, target, g_ref, F_ref, runner


def test_reactions_match_oracle(problem):
    w, theta0, nsteps, target, g_ref, F_ref, runner = problem
    F = runner.forward(theta0)
    assert np.allclose(F, F_ref, rtol=1e-9, atol=0)


def test_adjoint_gradient_matches_oracle(problem):
    w, theta0, nsteps, target, g_ref, F_ref, runner = problem
    F = runner.forward(theta0)
    g = runner.backward(2.0 * (F - target))
    scale = np.abs(g_ref * theta0).max()
    for i in range(12):
        assert abs(g[i] - g_ref[i]) <= 1e-9 * abs(g_ref[i]) + 1e-11 * scale / abs(theta0[i]), (i, g[i], g_ref[i])


def test_adjoint_gradient_matches_central_differences(problem):
    w, theta0, nsteps, target, g_ref, F_ref, runner = problem
    F = runner.forward(theta0)
    g = runner.backward(2.0 * (F - target))
    loss = lambda th: float(np.sum((runner.forward(th) - target) ** 2))
    for i in range(12):
        h = 1e-5 * abs(theta0[i])
        tp, tm = theta0.copy(), theta0.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 1e-9 * np.abs(g * theta0).max() / abs(theta0[i]), (i, g[i], fd)


def test_autograd_function(problem):
    w, theta0, nsteps, target, g_ref, F_ref, runner = problem
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    F = ReactionCurve.apply(theta, runner)
    loss = ((F - torch.as_tensor(target)) ** 2).sum()
    loss.backward()
    scale = np.abs(g_ref * theta0).max()
    g = theta.grad.numpy()
    for i in range(12):
        assert abs(g[i] - g_ref[i]) <= 1e-9 * abs(g_ref[i]) + 1e-11 * scale / abs(theta0[i])
    runner.close()
