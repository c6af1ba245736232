"""Pins of the oracle's hardening Prandtl branch (Box 2, Eq.
plasticity-strain-hardening-law, degraded consistency condition
g q_tr - 3 g mu dgam - sigma_y(eps_p,n + dgam) = 0):

* linear hardening has the closed form dgam = (g q_tr - sigma_y(eps_p,n)) / (3 g mu + H)
  and returns the degraded von Mises stress onto sigma_y(eps_p,n+1);
* with Voce hardening the returned stress is on the current yield surface;
* the dual-number tangent equals the independent restatement of Eq.
  plasticity-dtau-vonMises (H != 0) and App. C (tests/appendix_tangent.py);
* the assembled Jacobian equals central differences of the residual with a live
  accumulated plastic strain.

The hardening values (H_lin 2 GPa, sigma_inf 800 MPa, beta 40) are test inputs:
the paper's examples are perfectly plastic.
"""
import numpy as np

from paper_2607_21150_gb300 import inputs
import appendix_tangent as app

E2, NU2, S0 = 198000.0, 0.3, 500.0
MU = E2 / (2 * (1 + NU2))
HLIN, SINF, BETA = 2000.0, 800.0, 40.0


def _row(Hl, sinf, beta, E0=1e-9):
    ph = inputs.phase_vector(dict(Gc=0.8, l0=0.005, E0=E0, nu0=0.3, prandtl=(E2, NU2, S0)))
    return inputs.harden(ph[None], Hl, sinf, beta)[0]


def _sy(ep, Hl, sinf, beta):
    return S0 + Hl * ep + (sinf - S0) * (1 - np.exp(-beta * ep))


def _uniaxial(orc, row, lam, phi, epn, eta=1e-3):
    G = np.diag([lam - 1, 0.0, 0.0])
    inp = np.zeros(13)
    inp[:9] = G.ravel()
    inp[9] = phi
    hist = inputs.zero_history(1).T.copy()
    hist[0, 12] = epn
    glob = np.array([2, eta, 0.0, 0.01, 1.0])
    out = orc.pointwise(inp[None], hist, np.zeros(1, np.uint8), row[None], glob)
    tau = out["f1"][0, :3] @ np.diag([lam, 1, 1])
    td = tau - np.trace(tau) / 3 * np.eye(3)
    return out, np.sqrt(1.5) * np.linalg.norm(td)


def test_linear_hardening_closed_form(orc):
    row = _row(HLIN, S0, 0.0)
    for lam, phi, epn in ((1.01, 0.0, 0.0), (1.02, 0.3, 0.01), (0.985, 0.1, 0.05)):
        g = (1 - phi) ** 2 + 1e-3
        q = 2 * MU * abs(np.log(lam))
        out, vm = _uniaxial(orc, row, lam, phi, epn)
        assert out["flags"][0] & 1
        dgam = (g * q - (S0 + HLIN * epn)) / (3 * g * MU + HLIN)
        assert np.isclose(out["hist_new"][0, 12] - epn, dgam, rtol=1e-12)
        assert np.isclose(vm, S0 + HLIN * (epn + dgam), rtol=1e-12)


def test_voce_return_onto_yield_surface(orc):
    row = _row(HLIN, SINF, BETA)
    for lam, phi, epn in ((1.01, 0.0, 0.0), (1.03, 0.2, 0.02), (0.97, 0.0, 0.1)):
        out, vm = _uniaxial(orc, row, lam, phi, epn)
        assert out["flags"][0] & 1
        ep1 = out["hist_new"][0, 12]
        assert ep1 > epn
        assert np.isclose(vm, _sy(ep1, HLIN, SINF, BETA), rtol=1e-12)


def test_elastic_below_the_hardened_yield_stress(orc):
    """A state that yields for sigma_y(0) stays elastic once eps_p,n has hardened the branch."""
    row = _row(HLIN, SINF, BETA)
    lam = 1.0045  # q_tr = 2 mu ln lam ~ 682 MPa
    out0, _ = _uniaxial(orc, row, lam, 0.0, 0.0, eta=0.0)
    out1, vm = _uniaxial(orc, row, lam, 0.0, 0.2, eta=0.0)
    assert out0["flags"][0] & 1 and not (out1["flags"][0] & 1)
    assert np.isclose(vm, 2 * MU * np.log(lam), rtol=1e-12)


def test_tangent_matches_appendix_with_hardening(orc):
    rng = np.random.default_rng(17)
    ph = inputs.harden(inputs.phase_vector(inputs.EX3_MATRIX)[None], HLIN, SINF, BETA)[0]
    seen = 0
    for at in (1, 2):
        glob = np.array([at, 1e-3, 1e-2, 0.01, 1234.5])
        for trial in range(12):
            amp = [3e-3, 1e-2, 3e-2][trial % 3]
            inp = np.zeros(13)
            inp[:9] = amp * rng.standard_normal(9)
            inp[9] = rng.uniform(0, 0.9)
            inp[10:] = rng.standard_normal(3)
            hist = inputs.random_history(1, 200 + trial, H_max=[0.0, 1.0, 1e3][trial % 3]).T[0]
            hist[12] = rng.uniform(0.0, 0.05)
            out = orc.pointwise(inp[None], hist[None], np.zeros(1, np.uint8), ph[None], glob)
            D = out["D"][0]
            Dref = app.tangent16(inp, hist, ph, glob)
            err = np.abs(D - Dref).max() / np.abs(Dref).max()
            assert err < 1e-10, (err, trial)
            seen += int(out["flags"][0]) & 1
    assert seen >= 8  # most of the points yield


def test_fd_of_residual_with_hardening(orc):
    w = inputs.cube(nx=2, p=2, hist_seed=2, H_max=80.0, u_amp=5e-3)
    w.phases = inputs.harden(w.phases, HLIN, SINF, BETA)
    w.hist[12] = np.random.default_rng(4).uniform(0.0, 0.05, w.mesh.nq)
    out = orc.assemble(w, matrix=True)
    assert (out["flags"] & 1).mean() > 0.3  # a good share of the points yield
    K = out["K"]
    v = inputs.random_vector(w.mesh.ndof, 1)
    eps = 1e-6 * np.linalg.norm(w.z) / np.linalg.norm(v)
    op = orc.assemble(w, z=w.z + eps * v.reshape(4, -1), matrix=False)
    om = orc.assemble(w, z=w.z - eps * v.reshape(4, -1), matrix=False)
    assert np.array_equal(op["flags"], out["flags"]) and np.array_equal(om["flags"], out["flags"])
    fd = (op["r"] - om["r"]).ravel() / (2 * eps)
    Kv = K @ v
    assert np.linalg.norm(Kv - fd) <= 1e-7 * np.linalg.norm(Kv)
