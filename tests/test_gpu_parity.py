"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (FP64): relative L2 error <= 1e-12 for the residual, the Jacobian
action and its transpose, the diagonal, the transfers and the Chebyshev
smoother; flags bit-exact at every point whose decision margin exceeds 1e-10
(relative); trial history <= 1e-12 relative.  FP32 level applies are compared
with the FP64 ones at the FP32 rounding level (<= 2e-5 relative L2).  The
double-float action (PFF_DF64) is held to the FP64 bar against the oracle:
each of its operations errs by about 2^-47 of the magnitudes involved, some
200 operations feed one output, so its error stays near 1e-13.
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_21150_gb300.session import Session  # noqa: E402
from paper_2607_21150_gb300 import pff  # noqa: E402

TOL = 1e-12


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def np_(t):
    return t.detach().cpu().numpy()


def _flags_agree(gpu_flags, ref, margins, eps=1e-10):
    safe = (np.abs(margins[:, 0]) > eps) & (np.abs(margins[:, 1]) > eps) & (np.abs(margins[:, 2]) > eps)
    assert safe.mean() > 0.99
    assert np.array_equal(gpu_flags[safe], ref[safe])


def _two_phase(nx, ny, nz, p, seed, mask=True, at=2):
    """Small two-phase box with random state and history, tension Dirichlet data."""
    m = inputs.Mesh(nx, ny, nz, p, p + 1, (0.01 * nx, 0.01 * ny, 0.01 * nz))
    rng = np.random.default_rng(seed)
    phases = np.stack([inputs.phase_vector(inputs.EX3_MATRIX), inputs.phase_vector(inputs.EX3_PARTICLE)])
    glob = inputs.glob_vector(at, 1e-3, 1e-2, 0.005, inputs.EX3_MATRIX["s_phi"][at])
    phase = (rng.random(m.nq) < 0.4).astype(np.uint8)
    z = inputs.random_state(m, seed, u_amp=2e-4, phi_max=0.6)
    hist = inputs.random_history(m.nq, seed + 1, H_max=3000.0)
    mk = dv = None
    if mask:
        mk, dv = inputs.dirichlet_tension(m, 1e-4)
        z[mk.astype(bool)] = dv[mk.astype(bool)] + rng.uniform(-1e-5, 1e-5, mk.sum())
    return inputs.Workload("box", m, phases, glob, phase, z, hist, mk, dv)


def _hardened(nx, ny, nz, p, seed):
    """Two-phase box whose Prandtl branches harden (linear + Voce, test values)
    with a random accumulated plastic strain."""
    w = _two_phase(nx, ny, nz, p, seed)
    w.phases = inputs.harden(w.phases, 2000.0, 800.0, 40.0)
    w.hist[12] = np.random.default_rng(seed + 3).uniform(0.0, 0.05, w.mesh.nq)
    return w


def _mapped(nx, ny, nz, p, seed, kind):
    """Two-phase box on a mapped mesh: smoothly curved elements or straight-edged
    distorted hexahedra (isoparametric geometry from nodal coordinates)."""
    w = _two_phase(nx, ny, nz, p, seed)
    w.X = inputs.mapped_coords(w.mesh, kind, amp=0.15, seed=seed)
    return w


CASES = {
    "cube_q2": lambda: inputs.cube(),
    "cube_b_q2": lambda: inputs.cube(hist_seed=2, H_max=80.0),
    "box_q4_ragged": lambda: _two_phase(3, 2, 2, 4, 5),      # 12 elements: 2 blocks of 10, ragged
    "box_q3_ragged": lambda: _two_phase(3, 3, 2, 3, 7, at=1),  # 18 elements: blocks of 16
    "box_q1": lambda: _two_phase(5, 4, 4, 1, 9),              # 80 elements: blocks of 64
    "box_q3_hardening": lambda: _hardened(3, 2, 2, 3, 31),
    "box_q4_curved": lambda: _mapped(3, 2, 2, 4, 41, "smooth"),
    "box_q2_distorted": lambda: _mapped(3, 3, 2, 2, 43, "vertices"),
    "box_q4_single": lambda: _two_phase(1, 1, 1, 4, 51),      # one element: 9 of the block's 10 idle
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, orc):
    w = CASES[request.param]()
    ref = orc.assemble(w)
    s = Session(w, df=True)
    r = s.residual(w.z)
    torch.cuda.synchronize()
    return request.param, w, ref, s, r


def test_residual(case):
    name, w, ref, s, r = case
    assert s.status() == 0
    assert rel(np_(r), ref["r"]) <= TOL, name


def test_flags_and_trial_history(case):
    name, w, ref, s, r = case
    _flags_agree(np_(s.flags()), ref["flags"], ref["margins"])
    h = np_(s.history(1))
    assert rel(h, ref["hist_new"]) <= TOL, name
    s.commit()
    assert rel(np_(s.history(0)), ref["hist_new"]) <= TOL


def test_jacobian_apply(case):
    name, w, ref, s, r = case
    v = inputs.random_vector(w.mesh.ndof, 1)
    x = torch.from_numpy(v).cuda()
    y = s.apply(x)
    assert rel(np_(y), ref["K"] @ v) <= TOL, name
    yt = s.apply(x, transpose=True)
    assert rel(np_(yt), ref["K"].T @ v) <= TOL, name


def test_df64_apply(case):
    name, w, ref, s, r = case
    v = inputs.random_vector(w.mesh.ndof, 1)
    x = torch.from_numpy(v).cuda()
    y = s.apply(x, prec=pff.PFF_DF64)
    assert rel(np_(y), ref["K"] @ v) <= TOL, name
    yt = s.apply(x, prec=pff.PFF_DF64, transpose=True)
    assert rel(np_(yt), ref["K"].T @ v) <= TOL, name
    # Dirichlet rows are the identity, bit for bit
    if w.mask is not None:
        mk = w.mask.ravel().astype(bool)
        assert np.array_equal(np_(y)[mk], v[mk])


def test_df64_needs_planes(orc):
    w = inputs.cube()
    s = Session(w)
    s.residual(w.z)
    x = torch.from_numpy(inputs.random_vector(w.mesh.ndof, 2)).cuda()
    with pytest.raises(pff.PffError, match="pff_op_enable_df"):
        s.apply(x, prec=pff.PFF_DF64)
    with pytest.raises(pff.PffError):
        pff.pff_assemble_diagonal(s.levels[w.mesh.p], pff.PFF_DF64, x, s.stream)


def test_degenerate_actions(orc):
    """x = 0 gives y = 0 exactly in every precision; with every DoF prescribed
    the action is the identity, bit for bit."""
    w = _two_phase(3, 2, 2, 4, 53)
    s = Session(w, f32=True, df=True)
    s.residual(w.z)
    L = s.levels[w.mesh.p]
    n = w.mesh.ndof
    for prec, dt in ((pff.PFF_F64, torch.float64), (pff.PFF_DF64, torch.float64), (pff.PFF_F32, torch.float32)):
        x = torch.zeros(n, dtype=dt, device="cuda")
        y = torch.full((n,), 7.0, dtype=dt, device="cuda")
        pff.pff_jacobian_apply(L, prec, x, y, s.stream)
        torch.cuda.synchronize()
        assert torch.count_nonzero(y).item() == 0
    full = torch.ones(n, dtype=torch.uint8, device="cuda")
    pff.pff_set_dirichlet(s.op, full, torch.zeros(n, dtype=torch.float64, device="cuda"), s.stream)
    v = torch.from_numpy(inputs.random_vector(n, 5)).cuda()
    for prec, xv in ((pff.PFF_F64, v), (pff.PFF_DF64, v), (pff.PFF_F32, v.float())):
        for fn in (pff.pff_jacobian_apply, pff.pff_jacobian_transpose_apply):
            y = torch.empty_like(xv)
            fn(L, prec, xv, y, s.stream)
            torch.cuda.synchronize()
            assert torch.equal(y, xv)


def test_diagonal(case):
    name, w, ref, s, r = case
    d = s.diag()
    assert rel(np_(d), ref["K"].diagonal()) <= TOL, name


def test_offsets_restriction_matches_structured(orc):
    w = _two_phase(3, 2, 2, 4, 11)
    a = Session(w)
    b = Session(w, offsets=True)
    ra, rb = a.residual(w.z), b.residual(w.z)
    v = torch.from_numpy(inputs.random_vector(w.mesh.ndof, 3)).cuda()
    assert rel(np_(rb), np_(ra)) <= 1e-14
    assert rel(np_(b.apply(v)), np_(a.apply(v))) <= 1e-14


def test_fp32_apply_matches_oracle(orc):
    """FP32 action and its transpose (FP32 vectors, FP32 stored words) against
    the oracle's assembled K and K^T at the FP32 rounding level: each of the
    ~200 operations that feed one output errs by at most 2^-24 of the
    magnitudes involved, and the inputs themselves are rounded to FP32, so the
    relative L2 error stays near 1e-6; the bound is 2e-5."""
    w = _two_phase(3, 2, 2, 4, 13)
    ref = orc.assemble(w)
    s = Session(w, f32=True)
    s.residual(w.z)
    v = inputs.random_vector(w.mesh.ndof, 4)
    v32 = torch.from_numpy(v.astype(np.float32)).cuda()
    y32 = np_(s.apply(v32, prec=pff.PFF_F32))
    yt32 = np_(s.apply(v32, prec=pff.PFF_F32, transpose=True))
    assert rel(y32, ref["K"] @ v) <= 2e-5, rel(y32, ref["K"] @ v)
    assert rel(yt32, ref["K"].T @ v) <= 2e-5, rel(yt32, ref["K"].T @ v)


@pytest.mark.parametrize("pf,levels", [(4, (2, 1)), (2, (1,)), (3, (1,))])
def test_multigrid_levels(orc, pf, levels):
    """Level operator = P^T K_f P (R9); transfers = oracle P with Dirichlet rows/cols
    removed; level diagonal = diag(P^T K_f P)."""
    w = _two_phase(2, 3, 2, pf, 17 + pf)
    ref = orc.assemble(w)
    s = Session(w, levels=levels)
    s.residual(w.z)
    Kf = ref["K"]
    for pc in levels:
        P = orc.prolongation(w.mesh, pc)
        mc = inputs.coarsen_mask(w.mesh, w.mask, pc)
        Pm = orc.masked_prolongation(P, w.mask, mc)
        Kc = orc.coarse_operator(Kf, Pm, mc)
        nc = Pm.shape[1]
        xc = inputs.random_vector(nc, 21)
        yc = np_(s.apply(torch.from_numpy(xc).cuda(), p=pc))
        assert rel(yc, Kc @ xc) <= TOL, pc
        ytc = np_(s.apply(torch.from_numpy(xc).cuda(), p=pc, transpose=True))
        assert rel(ytc, Kc.T @ xc) <= TOL, pc
        assert rel(np_(s.diag(pc)), Kc.diagonal()) <= TOL, pc
        # transfers to the finest level
        xf = np_(s.prolong(torch.from_numpy(xc).cuda(), pc, pf))
        assert rel(xf, Pm @ xc) <= 1e-14
        rf = inputs.random_vector(Pm.shape[0], 22)
        rc = np_(s.restrict(torch.from_numpy(rf).cuda(), pc, pf))
        assert rel(rc, Pm.T @ rf) <= 1e-14
    if len(levels) == 2:  # level-to-level transfer 2 -> 1
        P21 = orc.prolongation(inputs.Mesh(2, 3, 2, 2, pf + 1, w.mesh.L), 1, 2)
        m2 = inputs.coarsen_mask(w.mesh, w.mask, 2)
        m1 = inputs.coarsen_mask(w.mesh, w.mask, 1)
        P21m = orc.masked_prolongation(P21, m2, m1)
        x1 = inputs.random_vector(P21m.shape[1], 23)
        x2 = np_(s.prolong(torch.from_numpy(x1).cuda(), 1, 2))
        assert rel(x2, P21m @ x1) <= 1e-14


def test_chebyshev_smoother(orc):
    w = _two_phase(3, 2, 2, 4, 31)
    ref = orc.assemble(w)
    s = Session(w)
    s.residual(w.z)
    K = ref["K"]
    dg = K.diagonal()
    b = inputs.random_vector(w.mesh.ndof, 5)
    x0 = inputs.random_vector(w.mesh.ndof, 6) * 1e-3
    for degree in (1, 3, 4):
        xr = orc.chebyshev(K, dg, b, x0, degree, 0.1, 1.9)
        x = torch.from_numpy(x0.copy()).cuda()
        s.chebyshev(torch.from_numpy(b).cuda(), x, s.diag(), degree, 0.1, 1.9)
        assert rel(np_(x), xr) <= TOL, degree


def test_linearization_vs_oracle_tangent(orc):
    """Stored 67 words = the oracle's dual-number tangent scaled by w detJ and the
    parent factors (a direct check of Appendix B/C on the GPU)."""
    w = inputs.cube(nx=2, hist_seed=2, H_max=80.0)
    s = Session(w)
    s.residual(w.z)
    lin = np_(s.linearization())
    # oracle pointwise inputs at the Gauss points of the GPU's own interpolation
    m = w.mesh
    xg, xq, wq, B, D = orc.basis(m.p, m.Q)
    P = m.p + 1
    h = np.array(m.h)
    sc = 2.0 / h
    detJ = np.prod(h) / 8
    nodes = inputs.element_offsets(m)
    inp = np.zeros((m.nq, 13))
    wdet = np.zeros(m.nq)
    for e in range(m.nel):
        ze = w.z[:, nodes[e]].reshape(4, P, P, P)  # [f][c][b][a]
        for k in range(m.Q):
            for j in range(m.Q):
                for i in range(m.Q):
                    q = e * m.Q ** 3 + i + m.Q * (j + m.Q * k)
                    Bi, Bj, Bk = B[i], B[j], B[k]
                    Di, Dj, Dk = D[i], D[j], D[k]
                    for f in range(4):
                        zf = ze[f]
                        gx = np.einsum("c,b,a,cba->", Bk, Bj, Di, zf) * sc[0]
                        gy = np.einsum("c,b,a,cba->", Bk, Dj, Bi, zf) * sc[1]
                        gz = np.einsum("c,b,a,cba->", Dk, Bj, Bi, zf) * sc[2]
                        if f < 3:
                            inp[q, 3 * f:3 * f + 3] = gx, gy, gz
                        else:
                            inp[q, 10:13] = gx, gy, gz
                            inp[q, 9] = np.einsum("c,b,a,cba->", Bk, Bj, Bi, zf)
                    wdet[q] = wq[i] * wq[j] * wq[k] * detJ
    out = orc.pointwise(inp, w.hist.T.copy(), w.phase, w.phases, w.glob)
    Dh = out["D"]
    # rebuild the 67 words from the oracle tangent
    ref = np.zeros((67, m.nq))
    k = 0
    for mm in range(9):
        for nn in range(mm, 9):
            ref[k] = wdet * sc[mm % 3] * sc[nn % 3] * Dh[:, 4 + mm, 4 + nn]
            k += 1
    for mm in range(9):
        ref[45 + mm] = wdet * sc[mm % 3] * Dh[:, 4 + mm, 3]
        ref[54 + mm] = wdet * sc[mm % 3] * Dh[:, 3, 4 + mm]
    ref[63] = wdet * Dh[:, 3, 3]
    for a in range(3):
        ref[64 + a] = wdet * sc[a] ** 2 * Dh[:, 13 + a, 13 + a]
    for blk, sl in (("A", slice(0, 45)), ("P", slice(45, 54)), ("C", slice(54, 63)), ("D", slice(63, 64)),
                    ("K", slice(64, 67))):
        assert rel(lin[sl], ref[sl]) <= 1e-11, blk


def test_full_size_tension_q4_sampled_rows(orc):
    """16^3 Q4 two-phase tension workload (1.1 M DoF) at full size: residual,
    J x, J^T x and diag(J) at sampled rows against the oracle's element rows,
    relative L2 over the sampled rows <= 1e-12."""
    w = inputs.tension_q4()
    rng = np.random.default_rng(3)
    w.z = w.z + 0.0
    w.z[:3] += rng.uniform(-2e-4, 2e-4, (3, w.mesh.nn))
    w.z[3] = rng.uniform(0, 0.4, w.mesh.nn)
    mk = w.mask.astype(bool)
    w.z[mk] = w.dvals[mk]
    w.hist = inputs.random_history(w.mesh.nq, 4, H_max=400.0)
    w.hist[13] = np.maximum(w.hist[13], inputs.zero_history(1)[13, 0])
    s = Session(w, df=True)
    r = np_(s.residual(w.z))
    x = inputs.random_vector(w.mesh.ndof, 8)
    xt = torch.from_numpy(x).cuda()
    jx, jtx, dg = np_(s.apply(xt)), np_(s.apply(xt, transpose=True)), np_(s.diag())
    jx_df = np_(s.apply(xt, prec=pff.PFF_DF64))
    jtx_df = np_(s.apply(xt, prec=pff.PFF_DF64, transpose=True))
    dofs = np.sort(rng.choice(w.mesh.ndof, 48, replace=False))
    dofs = np.concatenate([dofs, [0, w.mesh.ndof - 1, 3 * w.mesh.nn + w.mesh.nn // 2]])
    ref = orc.sample_rows(w, dofs, x)
    for key, g in (("r", r), ("jx", jx), ("jtx", jtx), ("diag", dg), ("jx", jx_df), ("jtx", jtx_df)):
        assert rel(g[dofs], ref[key]) <= 1e-12, (key, rel(g[dofs], ref[key]))


@pytest.mark.parametrize("name", ["compress_q4", "notched_q3", "adjoint_q2"])
def test_full_size_workloads_sampled_rows(orc, name):
    """The bench's workloads at full size and in its launch configuration (fine
    level of a session with the p-levels, FP32 and double-float copies):
    64^3 Q4 compression (67.9 M DoF), 48^3 Q3 notched bar (36.4 M DoF), 24^3 Q2
    adjoint box (0.47 M DoF).  Residual, J x, J^T x, diag(J) and the
    double-float action at sampled rows against the oracle's element rows at
    the FP64 bar (relative L2 over the sampled rows <= 1e-12); the FP32 action
    at the FP32 rounding level (2e-5)."""
    import bench
    w = bench.make_workload(name, seed=0)
    m = w.mesh
    s = Session(w, levels=(2, 1) if m.p == 4 else (1,), f32=True, df=True)
    r = np_(s.residual(w.z))
    assert s.status() == 0
    x = inputs.random_vector(m.ndof, 8)
    xt = torch.from_numpy(x).cuda()
    out = {"r": r, "jx": np_(s.apply(xt)), "jtx": np_(s.apply(xt, transpose=True)), "diag": np_(s.diag())}
    jx_df = np_(s.apply(xt, prec=pff.PFF_DF64))
    jx_32 = np_(s.apply(xt.float(), prec=pff.PFF_F32)).astype(np.float64)
    s.close()
    rng = np.random.default_rng(5)
    dofs = np.sort(rng.choice(m.ndof, 40, replace=False))
    dofs = np.concatenate([dofs, [0, m.ndof - 1, 3 * m.nn + m.nn // 2, 2 * m.nn + m.nn - 1]])
    ref = orc.sample_rows(w, dofs, x)
    for key, g in list(out.items()) + [("jx", jx_df)]:
        assert rel(g[dofs], ref[key]) <= 1e-12, (name, key, rel(g[dofs], ref[key]))
    assert rel(jx_32[dofs], ref["jx"]) <= 2e-5, (name, "fp32", rel(jx_32[dofs], ref["jx"]))
