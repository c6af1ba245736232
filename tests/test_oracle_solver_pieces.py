"""Pins of the oracle routines that the GPU parity tests compare against at
full size or inside the solver:

* the oracle's C SpMV equals scipy's CSR product;
* the 1D Lagrange basis is cardinal at the GLL nodes and reproduces
  polynomials of degree p with their derivatives;
* `sample_rows` (rows formed element by element, no assembly) equals the rows
  of the assembled residual, J x, J^T x and diag(J), Dirichlet rows included;
* the p-multigrid V-cycle (masked prolongation, Galerkin coarse operator,
  Chebyshev smoothing, restriction P^T) is a linear operator, symmetric for a
  symmetric fine operator, and as a stationary iteration x <- x + M (b - K x)
  it contracts the error (a transposed or missing transfer fails one of the
  three).
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs


def _hooke_cube(nx=2, p=2, tension=True):
    w = inputs.cube(nx=nx, p=p)
    w.phases = np.stack([inputs.phase_vector(dict(Gc=0.8, l0=0.05, E0=1000.0, nu0=0.3))])
    w.hist = inputs.zero_history(w.mesh.nq)
    if tension:
        w.mask, w.dvals = inputs.dirichlet_tension(w.mesh, 0.0)
    w.z = np.zeros((4, w.mesh.nn))   # zero state: no damage driving force, K symmetric
    return w


def test_spmv_matches_scipy(orc):
    w = inputs.cube(nx=2, p=2)
    K = orc.assemble(w)["K"]
    x = np.random.default_rng(3).uniform(-1, 1, K.shape[0])
    ref = K @ x
    assert np.linalg.norm(orc.spmv(K, x) - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_lagrange_cardinal_and_exact(orc, p):
    xg = orc.basis(p, p + 1)[0]
    L, dL = orc.lagrange(p, xg)
    assert np.abs(L - np.eye(p + 1)).max() <= 1e-14
    t = np.linspace(-1.0, 1.0, 11)
    L, dL = orc.lagrange(p, t)
    c = np.random.default_rng(p).uniform(-1, 1, p + 1)   # polynomial of degree p
    f, df = np.polynomial.polynomial.polyval(xg, c), np.polynomial.polynomial.polyval(t, np.polynomial.polynomial.polyder(c))
    assert np.abs(L @ f - np.polynomial.polynomial.polyval(t, c)).max() <= 1e-13
    assert np.abs(dL @ f - df).max() <= 1e-12


def test_sample_rows_match_assembly(orc):
    w = inputs.cube(nx=2, p=2, hist_seed=2, H_max=80.0)
    w.mask, w.dvals = inputs.dirichlet_tension(w.mesh, 1e-3)
    mk = w.mask.astype(bool)
    w.z[mk] = w.dvals[mk]
    out = orc.assemble(w)
    K, r = out["K"], out["r"].ravel()
    x = np.random.default_rng(4).uniform(-1, 1, K.shape[0])
    rng = np.random.default_rng(5)
    dofs = np.unique(np.concatenate([rng.choice(K.shape[0], 40, replace=False), np.flatnonzero(mk.ravel())[:10]]))
    s = orc.sample_rows(w, dofs, x)
    scale = np.abs(K).max() * np.abs(x).sum()
    assert np.abs(s["r"] - r[dofs]).max() <= 1e-12 * np.abs(r).max()
    assert np.abs(s["jx"] - (K @ x)[dofs]).max() <= 1e-13 * scale
    assert np.abs(s["jtx"] - (K.T @ x)[dofs]).max() <= 1e-13 * scale
    assert np.abs(s["diag"] - K.diagonal()[dofs]).max() <= 1e-13 * np.abs(K.diagonal()).max()


def _two_levels(orc):
    w = _hooke_cube()
    m = w.mesh
    K = orc.assemble(w)["K"]
    mc = inputs.coarsen_mask(m, w.mask, 1)
    P = orc.masked_prolongation(orc.prolongation(m, 1), w.mask, mc)
    Kc = orc.coarse_operator(K, P, mc)
    lams = []
    for A in (K, Kc):
        Ad = A.toarray()
        lams.append(float(np.max(np.abs(np.linalg.eigvals(Ad / Ad.diagonal()[:, None])))))
    return K, Kc, P, lams


def test_vcycle_linear_symmetric_contracting(orc):
    K, Kc, P, lams = _two_levels(orc)
    assert np.abs((K - K.T).toarray()).max() <= 1e-12 * np.abs(K).max()
    Ks, Ps, diags = [K, Kc], [P], [K.diagonal(), Kc.diagonal()]

    def M(r):
        return orc.vcycle(Ks, Ps, diags, lams, r)

    rng = np.random.default_rng(6)
    n = K.shape[0]
    r1, r2 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    m1, m2 = M(r1), M(r2)
    assert np.linalg.norm(M(2.0 * r1 - 3.0 * r2) - (2.0 * m1 - 3.0 * m2)) <= 1e-12 * np.linalg.norm(m1)
    assert abs(m1 @ r2 - r1 @ m2) <= 1e-12 * np.linalg.norm(m1) * np.linalg.norm(r2)
    # stationary iteration on K x = b from 0: the error contracts
    x_true = rng.uniform(-1, 1, n)
    b = K @ x_true
    x = np.zeros(n)
    e0 = np.linalg.norm(x_true)
    for _ in range(8):
        x = x + M(b - K @ x)
    assert np.linalg.norm(x - x_true) <= 1e-2 * e0
