"""Pins of the oracle's discrete adjoint: the gradient of a reaction-curve
misfit through three load steps (history carried between steps) equals central
finite differences of the loss, for all twelve per-phase parameters on the box,
and for four of them on a curved mesh and with a hardening Prandtl branch."""
import numpy as np

from paper_2607_21150_gb300 import inputs


def _adjoint_box():
    w = inputs.adjoint_q2(n=2)
    w.mesh = inputs.Mesh(2, 2, 2, 2, 3, w.mesh.L)
    return w


def test_oracle_adjoint_matches_central_differences(orc):
    w = _adjoint_box()
    top = inputs.top_face_mask(w.mesh)
    theta0 = orc.get_params(w.phases)
    nsteps = 3
    target, _, _ = orc.load_steps(w, inputs.twin_target(theta0), nsteps, top)
    g, F = orc.adjoint_gradient(w, theta0, nsteps, top, target)
    loss = lambda th: float(np.sum((orc.load_steps(w, th, nsteps, top)[0] - target) ** 2))
    assert np.count_nonzero(g) >= 11  # the stiff particle never yields here: d/d sigma0 = 0
    for i in range(12):
        h = 1e-5 * abs(theta0[i])
        tp, tm = theta0.copy(), theta0.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 1e-9 * np.abs(g * theta0).max() / abs(theta0[i]), (i, g[i], fd)


def test_oracle_adjoint_on_a_curved_mesh(orc):
    """The same check on a smoothly curved mesh (the geometric factors enter the
    residual, the pull-back and the reaction), for four parameters."""
    w = _adjoint_box()
    w.X = inputs.mapped_coords(w.mesh, "smooth", amp=0.15)
    top = inputs.top_face_mask(w.mesh)
    theta0 = orc.get_params(w.phases)
    nsteps = 3
    target, _, _ = orc.load_steps(w, inputs.twin_target(theta0), nsteps, top)
    g, F = orc.adjoint_gradient(w, theta0, nsteps, top, target)
    loss = lambda th: float(np.sum((orc.load_steps(w, th, nsteps, top)[0] - target) ** 2))
    for i in (0, 2, 4, 11):   # E_inf, sigma0, Gc of the matrix; l0 of the particle
        h = 1e-5 * abs(theta0[i])
        tp, tm = theta0.copy(), theta0.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 1e-9 * np.abs(g * theta0).max() / abs(theta0[i]), (i, g[i], fd)


def test_oracle_adjoint_with_hardening(orc):
    """The same check with linear + Voce hardening (test values, not Table 2
    data) and a live accumulated plastic strain: the implicit derivative of the
    return map enters both the tangent and the parameter partials."""
    w = _adjoint_box()
    rows = inputs.harden(w.phases, 0.0, 0.0, 0.0)
    rows[0, 11] = 300.0                       # the matrix yields within the three steps
    rows[:, 12] = 2000.0                      # H_lin
    rows[:, 13] = 1.6 * rows[:, 11]           # sigma_inf
    rows[:, 14] = 40.0                        # beta
    w.phases = rows
    w.hist[12] = np.random.default_rng(8).uniform(0.0, 0.02, w.mesh.nq)
    top = inputs.top_face_mask(w.mesh)
    theta0 = orc.get_params(w.phases)
    nsteps = 3
    target, _, hs = orc.load_steps(w, inputs.twin_target(theta0), nsteps, top)
    assert np.any(hs[-1][12] > w.hist[12] + 1e-9)   # plastic flow happened
    g, F = orc.adjoint_gradient(w, theta0, nsteps, top, target)
    loss = lambda th: float(np.sum((orc.load_steps(w, th, nsteps, top)[0] - target) ** 2))
    for i in (0, 2, 3, 4):   # E_inf, sigma0, eta_d, Gc of the matrix
        h = 1e-5 * abs(theta0[i])
        tp, tm = theta0.copy(), theta0.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 1e-9 * np.abs(g * theta0).max() / abs(theta0[i]), (i, g[i], fd)
    assert abs(g[2]) > 0
