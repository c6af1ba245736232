"""Newton-Krylov / p-multigrid solver on the GPU vs the oracle.

* assembled order-1 coarse operator = P^T K P (masked), relative L2 <= 1e-12;
* one FP64 V-cycle = the oracle's textbook V-cycle with the same lambda_max
  estimates (the interval is an input of both), relative L2 <= 1e-11; the
  mixed-precision V-cycle within FP32 rounding of it;
* FGMRES solves J x = b to its tolerance (checked against a direct solve);
* the Newton solution (FP64 and mixed p-MG) equals the oracle's Newton solution
  with direct solves to 1e-9 relative, with quadratic convergence.
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_21150_gb300 import pff  # noqa: E402
from paper_2607_21150_gb300.session import Session  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def np_(t):
    return t.detach().double().cpu().numpy()


def _box(nx, ny, nz, p, seed, state=True):
    m = inputs.Mesh(nx, ny, nz, p, p + 1, (0.01 * nx, 0.01 * ny, 0.01 * nz))
    rng = np.random.default_rng(seed)
    phases = np.stack([inputs.phase_vector(inputs.EX3_MATRIX), inputs.phase_vector(inputs.EX3_PARTICLE)])
    glob = inputs.glob_vector(2, 1e-3, 1e-2, 0.005, inputs.EX3_MATRIX["s_phi"][2])
    phase = (rng.random(m.nq) < 0.4).astype(np.uint8)
    mask, dv = inputs.dirichlet_tension(m, 2e-4 * m.L[2])
    if state:
        z = inputs.random_state(m, seed, u_amp=2e-4, phi_max=0.5)
        hist = inputs.random_history(m.nq, seed + 1, H_max=3000.0)
    else:
        z = np.zeros((4, m.nn))
        hist = inputs.zero_history(m.nq)
    z[mask.astype(bool)] = dv[mask.astype(bool)]
    return inputs.Workload("box", m, phases, glob, phase, z, hist, mask, dv)


def _hierarchy(orc, w, levels):
    """Oracle level matrices, prolongations and diagonals for level orders ``levels``."""
    ref = orc.assemble(w)
    Ks, Ps, masks = [ref["K"]], [], [w.mask]
    m = w.mesh
    prev_p, prev_mask = m.p, w.mask
    P_tot = None
    for pc in levels[1:]:
        mc = inputs.coarsen_mask(m, w.mask, pc)
        Pf = orc.prolongation(inputs.Mesh(m.nx, m.ny, m.nz, prev_p, m.Q, m.L), pc, prev_p)
        Pm = orc.masked_prolongation(Pf, prev_mask, mc)
        Ps.append(Pm)
        P_tot = Pm if P_tot is None else P_tot @ Pm
        Pfull = orc.masked_prolongation(orc.prolongation(m, pc), w.mask, mc)
        Ks.append(orc.coarse_operator(ref["K"], Pfull, mc))
        prev_p, prev_mask = pc, mc
    return ref, Ks, Ps


@pytest.fixture(scope="module")
def setup64(orc):
    w = _box(3, 2, 2, 4, 3)
    s = Session(w, levels=(2, 1))
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    solver = s.solver([4, 2, 1], mixed=0, coarse_solver=0)
    pff.pff_solver_setup(solver)
    ref, Ks, Ps = _hierarchy(orc, w, [4, 2, 1])
    return w, s, solver, ref, Ks, Ps


def test_assembled_coarse_operator(setup64):
    w, s, solver, ref, Ks, Ps = setup64
    xc = inputs.random_vector(Ks[-1].shape[0], 5)
    y = torch.zeros(len(xc), dtype=torch.float64, device="cuda")
    pff.pff_solver_coarse_apply(solver, torch.from_numpy(xc).cuda(), y)
    assert rel(np_(y), Ks[-1] @ xc) <= 1e-12


def test_vcycle_matches_oracle(orc, setup64):
    w, s, solver, ref, Ks, Ps = setup64
    lams = [pff.pff_solver_level_lambda(solver, l) for l in range(3)]
    r = inputs.random_vector(w.mesh.ndof, 6)
    z = torch.zeros(w.mesh.ndof, dtype=torch.float64, device="cuda")
    pff.pff_solver_vcycle(solver, torch.from_numpy(r).cuda(), z)
    zr = orc.vcycle(Ks, Ps, [K.diagonal() for K in Ks], lams, r)
    assert rel(np_(z), zr) <= 1e-11
    # eigenvalue estimates are below and near lambda_max of D^-1 K
    import scipy.linalg as sla
    for K, lam in zip(Ks, lams):
        ev = sla.eigvals(K.toarray() / K.diagonal()[:, None]).real.max()
        assert 0.85 * ev <= lam <= 1.05 * ev


def test_mixed_vcycle_close_to_fp64(orc, setup64):
    w, s64, solver64, ref, Ks, Ps = setup64
    s = Session(w, levels=(2, 1), f32=True)
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    solver = s.solver([4, 2, 1], mixed=1, coarse_solver=0)
    pff.pff_solver_setup(solver)
    lams = [pff.pff_solver_level_lambda(solver, l) for l in range(3)]
    r = inputs.random_vector(w.mesh.ndof, 6)
    z = torch.zeros(w.mesh.ndof, dtype=torch.float64, device="cuda")
    pff.pff_solver_vcycle(solver, torch.from_numpy(r).cuda(), z)
    zr = orc.vcycle(Ks, Ps, [K.diagonal() for K in Ks], lams, r)
    assert rel(np_(z), zr) <= 1e-4
    pff.pff_destroy_solver(solver)


def test_fgmres_linear_solve(orc):
    """On a physical state (undeformed, Dirichlet loading) D^-1 J is positive
    definite and the V-cycle a good preconditioner.  (The random large-strain state
    of the parity fixture makes D^-1 J indefinite, where Chebyshev smoothing
    amplifies the negative modes; parity of the V-cycle there is still checked.)"""
    import scipy.sparse.linalg as spla
    w = _box(3, 2, 2, 4, 3, state=False)
    ref = orc.assemble(w)
    s = Session(w, levels=(2, 1))
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    solver = s.solver([4, 2, 1], mixed=0)
    pff.pff_solver_setup(solver)
    b = inputs.random_vector(w.mesh.ndof, 7)
    x = torch.zeros(w.mesh.ndof, dtype=torch.float64, device="cuda")
    its, relres = pff.pff_solver_krylov(solver, torch.from_numpy(b).cuda(), x, 1e-10, 400)
    assert relres <= 1e-10 and its < 400
    assert its <= 40
    xr = spla.spsolve(ref["K"].tocsc(), b)
    assert rel(np_(x), xr) <= 1e-6
    pff.pff_destroy_solver(solver)


@pytest.mark.parametrize("mixed,outer,eig_every,words", [(0, 0, 1, 32), (1, 0, 1, 32), (1, 2, 1, 32), (1, 0, 0, 32),
                                                         (1, 2, 1, 16)])
def test_newton_solution_matches_oracle(orc, mixed, outer, eig_every, words):
    """outer = 2: the FGMRES operator is the double-float action (PFF_DF64);
    eig_every = 0: eigenvalue bounds estimated on the first Newton iteration only;
    words = 16: BF16 stored words in the FP32 levels and smoothers."""
    w = _box(2, 2, 3, 2, 11, state=False)
    z_ref, hist_ref, _ = orc.newton(w, rtol=1e-13)
    s = Session(w, levels=(1,), f32=bool(mixed), df=(outer == pff.PFF_DF64), bf16=(words == 16))
    solver = s.solver([2, 1], mixed=mixed, newton_rtol=1e-11, krylov_rtol=1e-6, outer_prec=outer,
                      eig_every=eig_every, level_words=words)
    z = torch.from_numpy(w.z.ravel().copy()).cuda()
    st = pff.pff_newton_solve(solver, z)
    assert st["converged"] == 1, st
    assert rel(np_(z), z_ref) <= 1e-9
    h = np.array(st["res_history"])
    assert h[-1] <= 1e-11 * h[0]
    # superlinear contraction once close (quadratic up to the Krylov tolerance)
    rates = h[1:] / h[:-1]
    assert rates.min() < 1e-2
    pff.pff_destroy_solver(solver)


@pytest.fixture(scope="module")
def setup_h(orc):
    """Q2 box of 8 x 8 x 4 elements: order-1 level 8 x 8 x 4, one h-coarsening to 4 x 4 x 2."""
    w = _box(8, 8, 4, 2, 21)
    s = Session(w, levels=(1,))
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    solver = s.solver([2, 1], mixed=0, coarse_solver=2)
    pff.pff_solver_setup(solver)
    ref = orc.assemble(w)
    m = w.mesh
    mc0 = inputs.coarsen_mask(m, w.mask, 1)
    A0 = orc.coarse_operator(ref["K"], orc.masked_prolongation(orc.prolongation(m, 1), w.mask, mc0), mc0)
    mc1 = orc.h_coarse_mask(mc0, 4, 4, 2)
    Ph = orc.masked_prolongation(orc.h_prolongation(4, 4, 2), mc0, mc1)
    A1 = orc.coarse_operator(A0, Ph, mc1)
    return w, s, solver, [A0, A1], [Ph]


def test_h_hierarchy_galerkin_operators(setup_h):
    w, s, solver, As, Ps = setup_h
    assert pff.pff_solver_num_hlevels(solver) == 2
    assert pff.pff_solver_hlevel_info(solver, 0)[0] == (8, 8, 4)
    assert pff.pff_solver_hlevel_info(solver, 1)[0] == (4, 4, 2)
    for l, A in enumerate(As):
        x = inputs.random_vector(A.shape[0], 30 + l)
        y = torch.zeros(len(x), dtype=torch.float64, device="cuda")
        pff.pff_solver_hlevel_apply(solver, l, torch.from_numpy(x).cuda(), y)
        assert rel(np_(y), A @ x) <= 1e-12, l


def test_h_vcycle_matches_oracle(orc, setup_h):
    w, s, solver, As, Ps = setup_h
    lams = [pff.pff_solver_hlevel_info(solver, l)[1] for l in range(2)]
    b = inputs.random_vector(As[0].shape[0], 40)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    pff.pff_solver_hcycle(solver, torch.from_numpy(b).cuda(), x)
    xr = orc.vcycle(As, Ps, [A.diagonal() for A in As], lams, b)
    assert rel(np_(x), xr) <= 1e-11


def test_newton_with_h_multigrid_coarse_solver(orc):
    """Same Newton solution with the Jacobi-GMRES and the h-multigrid coarse
    solver; the h-multigrid preconditioned coarse GMRES needs fewer iterations."""
    w = _box(8, 8, 4, 2, 23, state=False)
    z_ref, _, _ = orc.newton(w, rtol=1e-13)
    its = {}
    for cs in (1, 2):
        s = Session(w, levels=(1,))
        solver = s.solver([2, 1], mixed=0, coarse_solver=cs, newton_rtol=1e-11, krylov_rtol=1e-6)
        z = torch.from_numpy(w.z.ravel().copy()).cuda()
        st = pff.pff_newton_solve(solver, z)
        assert st["converged"] == 1, (cs, st)
        assert rel(np_(z), z_ref) <= 1e-9, cs
        its[cs] = st["coarse_iterations"]
        pff.pff_destroy_solver(solver)
    assert its[2] < its[1]


def test_mapped_mesh_coarse_operator_and_vcycle(orc):
    """Curved Q4 mesh: the assembled order-1 operator (with the off-diagonal
    phase-gradient combinations) equals P^T K P of the oracle, and one FP64
    V-cycle equals the oracle's."""
    w = _box(3, 2, 2, 4, 3)
    w.X = inputs.mapped_coords(w.mesh, "smooth", amp=0.15)
    s = Session(w, levels=(2, 1))
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    solver = s.solver([4, 2, 1], mixed=0, coarse_solver=0)
    pff.pff_solver_setup(solver)
    ref, Ks, Ps = _hierarchy(orc, w, [4, 2, 1])
    xc = inputs.random_vector(Ks[-1].shape[0], 5)
    y = torch.zeros(len(xc), dtype=torch.float64, device="cuda")
    pff.pff_solver_coarse_apply(solver, torch.from_numpy(xc).cuda(), y)
    assert rel(np_(y), Ks[-1] @ xc) <= 1e-12
    lams = [pff.pff_solver_level_lambda(solver, l) for l in range(3)]
    r = inputs.random_vector(w.mesh.ndof, 6)
    z = torch.zeros(w.mesh.ndof, dtype=torch.float64, device="cuda")
    pff.pff_solver_vcycle(solver, torch.from_numpy(r).cuda(), z)
    zr = orc.vcycle(Ks, Ps, [K.diagonal() for K in Ks], lams, r)
    assert rel(np_(z), zr) <= 1e-11
    pff.pff_destroy_solver(solver)
