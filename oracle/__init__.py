"""FP64 CPU oracle for the phase-field fracture operator (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with the CUDA library: the
compiled part (``pff_oracle.cpp``) has its own basis, kinematics, constitutive
update (matrix functions + dual numbers), element matrices and CSR assembly;
the Python part below adds what the paper states as textbook linear algebra:
sparse products, the Chebyshev iteration and direct solves.

Functions and the passages they follow:

* ``basis``            -- GLL / Gauss points and 1D Lagrange matrices (Sec. 4, B_I, B_xi).
* ``pointwise``        -- Box 1 + Sec. 3 pointwise update and its tangent (App. B, C by
                          dual numbers).
* ``assemble``         -- Eq. matrix-free-residual-compact / matrix-free-jacobian as a
                          global residual and an assembled CSR Jacobian (Dirichlet rows
                          and columns replaced by the identity).
* ``sample_rows``      -- the same quantities for selected rows of large meshes.
* ``prolongation``     -- p-prolongation P[f, c] = coarse basis at the fine nodes; R = P^T.
* ``coarse_operator``  -- Galerkin product P^T A P (equal to rediscretisation at the fine
                          Gauss points).
* ``chebyshev``        -- textbook Chebyshev iteration on D^-1 A (Saad, Alg. 12.1).
* ``masked_prolongation``, ``vcycle`` -- Dirichlet-masked transfers and the textbook
                          multigrid V-cycle of Sec. 5 (Chebyshev smoothing, R = P^T).
* ``h_prolongation``, ``h_coarse_mask`` -- trilinear full coarsening of the structured
                          order-1 grid (the geometric coarse solver standing in for the
                          paper's algebraic one, Sec. 5).
* ``newton``           -- Newton's method with direct solves (Sec. 5, exact linear solves).
* ``load_steps``, ``adjoint_gradient``, ``point_partials`` -- load-step sequences with
                          history commit (Box 1 step 4) and the discrete adjoint of a
                          reaction-curve misfit (assembled transposes, dual-number partials).
* ``geometry``         -- nodal coordinates of a mapped mesh: isoparametric element maps
                          of the Sec. 4 basis (the box is the special case).
* ``spmv``, ``lagrange``, ``logm1p``, ``expm`` -- the compiled loops exposed for pins.
* ``crack_c0``, ``s_phi``, ``psi_c`` -- the crack-density normalisation, the phase-field
                          residual scale (Eq. damage-residual-scaling) and the AT1
                          threshold (Sec. 3.1), derived here from the phase rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pff_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        llp = ctypes.POINTER(ctypes.c_longlong)
        L.orc_basis.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
        L.orc_lagrange_eval.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_pointwise.argtypes = [ctypes.c_int, dp, dp, u8p, dp, ctypes.c_int, dp,
                                    dp, dp, dp, dp, u8p, dp]
        L.orc_logm1p.argtypes = [dp, dp]
        L.orc_expm.argtypes = [dp, dp]
        L.orc_assemble.argtypes = [ip, dp, dp, ctypes.c_int, dp, dp, dp, u8p, u8p, dp,
                                   ctypes.c_int, dp, dp, u8p, dp, dp]
        L.orc_assemble.restype = ctypes.c_void_p
        L.orc_csr_nnz.argtypes = [ctypes.c_void_p]
        L.orc_csr_nnz.restype = ctypes.c_longlong
        L.orc_csr_get.argtypes = [ctypes.c_void_p, llp, llp, dp]
        L.orc_csr_free.argtypes = [ctypes.c_void_p]
        L.orc_sample_rows.argtypes = [ip, dp, dp, ctypes.c_int, dp, dp, dp, u8p, u8p, dp, dp,
                                      ctypes.c_int, llp, dp, dp, dp, dp, dp]
        L.orc_prolong_coo.argtypes = [ip, ctypes.c_int, ctypes.c_int, llp, llp, dp]
        L.orc_prolong_coo.restype = ctypes.c_longlong
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_csr_spmv.argtypes = [ctypes.c_longlong, llp, llp, dp, dp, dp]
        L.orc_point_partials.argtypes = [ctypes.c_int, dp, dp, u8p, dp, ctypes.c_int, dp, dp, dp]
        L.orc_qpoint_inputs.argtypes = [ip, dp, dp, dp, dp]
        L.orc_apply_bt.argtypes = [ip, dp, dp, ctypes.c_int, dp, dp]
        _lib = L
    return _lib


def _p(a, t=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(t))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def phase_rows(phases):
    """Phase parameter rows for the C oracle, 15 doubles each: the 12 of
    ``inputs.phase_vector`` and the hardening law (H_lin, sigma_inf, beta),
    padded with (0, sigma0, 0) = perfect plasticity when absent."""
    ph = np.atleast_2d(np.asarray(phases, dtype=np.float64))
    if ph.shape[1] == 15:
        return np.ascontiguousarray(ph)
    if ph.shape[1] != 12:
        raise ValueError("phase rows must have 12 or 15 entries")
    out = np.zeros((ph.shape[0], 15))
    out[:, :12] = ph
    out[:, 13] = ph[:, 11]
    return out


def crack_c0(at: int) -> float:
    """Normalisation c0 = 4 int_0^1 sqrt(alpha(s)) ds of the crack density
    (Sec. 3.1): alpha = s (AT1) gives 4 * 2/3 = 8/3, alpha = s^2 (AT2) gives 4 * 1/2 = 2."""
    return 4.0 * (2.0 / 3.0 if at == 1 else 0.5)


def s_phi(matrix_row, at: int) -> float:
    """Phase-field residual scale of Eq. damage-residual-scaling from the matrix
    phase's row (``phase_rows`` layout: Gc, l0, E_inf first): E c0 / (2 l0 Gc)."""
    Gc, l0, E = float(matrix_row[0]), float(matrix_row[1]), float(matrix_row[2])
    return E * crack_c0(at) / (2.0 * l0 * Gc)


def psi_c(phase_row) -> float:
    """AT1 elastic threshold of Sec. 3.1: the crack-driving energy below which the
    homogeneous AT1 local residual keeps phi = 0, psi_c = 3 Gc / (16 l0) (from
    g'(0) psi_c + Gc alpha'(0) / (c0 l0) = 0 with g'(0) = -2, alpha' = 1, c0 = 8/3)."""
    Gc, l0 = float(phase_row[0]), float(phase_row[1])
    return Gc / (crack_c0(1) * l0) / 2.0


def geometry(w):
    """Nodal coordinates [3][nn] of a mapped mesh (the workload's ``X``), or None
    for the affine box of ``w.mesh``."""
    X = getattr(w, "X", None)
    return None if X is None else np.ascontiguousarray(X, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops from now on."""
    lib().orc_set_num_threads(int(n))


def spmv(K, x):
    """y = K x with the oracle's OpenMP CSR loop (K from ``assemble``)."""
    indptr = np.ascontiguousarray(K.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(K.indices, dtype=np.int64)
    data = _f64(K.data)
    x = _f64(x)
    y = np.zeros(K.shape[0])
    lib().orc_csr_spmv(K.shape[0], _p(indptr, ctypes.c_longlong), _p(indices, ctypes.c_longlong), _p(data),
                       _p(x), _p(y))
    return y


# ---------------------------------------------------------------------------
def basis(p: int, Q: int):
    """GLL nodes xg[P], Gauss nodes xq[Q] and weights wq[Q], and the 1D Lagrange
    value / derivative matrices B[Q,P], D[Q,P] at the Gauss points."""
    P = p + 1
    xg, xq, wq = np.zeros(P), np.zeros(Q), np.zeros(Q)
    B, D = np.zeros((Q, P)), np.zeros((Q, P))
    lib().orc_basis(p, Q, _p(xg), _p(xq), _p(wq), _p(B), _p(D))
    return xg, xq, wq, B, D


def lagrange(p: int, t):
    t = _f64(np.atleast_1d(t))
    L = np.zeros((len(t), p + 1))
    dL = np.zeros((len(t), p + 1))
    lib().orc_lagrange_eval(p, len(t), _p(t), _p(L), _p(dL))
    return L, dL


def logm1p(X):
    X = _f64(X).reshape(3, 3)
    out = np.zeros((3, 3))
    lib().orc_logm1p(_p(X), _p(out))
    return out


def expm(A):
    A = _f64(A).reshape(3, 3)
    out = np.zeros((3, 3))
    lib().orc_expm(_p(A), _p(out))
    return out


def pointwise(inputs, hist, phase, phases, glob, tangent: bool = True, commit: bool = True):
    """Pointwise update at n points.  inputs [n,13] = (grad u row-major, phi,
    grad phi); hist [n,15] point-major; phase uint8 [n].  Returns a dict with
    f0 [n,4], f1 [n,4,3], D [n,16,16], hist_new [n,15], flags, psi_plus,
    margin_yield, margin_hist, theta."""
    inputs = _f64(inputs)
    n = inputs.shape[0]
    hist = _f64(hist)
    phase = _u8(phase)
    phases = _f64(phases)
    glob = _f64(glob)
    f0 = np.zeros((n, 4))
    f1 = np.zeros((n, 12))
    D = np.zeros((n, 16, 16)) if tangent else None
    hn = np.zeros((n, 15)) if commit else None
    flags = np.zeros(n, dtype=np.uint8)
    aux = np.zeros((n, 4))
    lib().orc_pointwise(n, _p(inputs), _p(hist), _p(phase, ctypes.c_uint8), _p(phase_rows(phases)), len(phases),
                        _p(glob), _p(f0), _p(f1), _p(D), _p(hn), _p(flags, ctypes.c_uint8), _p(aux))
    return dict(f0=f0, f1=f1.reshape(n, 4, 3), D=D, hist_new=hn, flags=flags,
                psi_plus=aux[:, 0], margin_yield=aux[:, 1], margin_hist=aux[:, 2], theta=aux[:, 3])


def _mesh_args(mesh):
    dims = np.ascontiguousarray(mesh.dims, dtype=np.int32)
    h = _f64(mesh.h)
    return dims, h


def assemble(w, z=None, hist=None, matrix: bool = True, mask="workload", dvals="workload"):
    """Residual, trial history, flags and (optionally) the assembled CSR Jacobian
    of workload ``w`` (see ``paper_2607_21150_gb300.inputs.Workload``)."""
    import scipy.sparse as sp

    m = w.mesh
    z = _f64(w.z if z is None else z)
    hist = _f64(w.hist if hist is None else hist)
    mask = w.mask if isinstance(mask, str) else mask
    dvals = w.dvals if isinstance(dvals, str) else dvals
    mask = _u8(mask)
    dvals = None if dvals is None else _f64(dvals)
    dims, h = _mesh_args(m)
    r = np.zeros(4 * m.nn)
    hn = np.zeros((15, m.nq))
    flags = np.zeros(m.nq, dtype=np.uint8)
    margins = np.zeros((m.nq, 3))
    L = lib()
    handle = L.orc_assemble(dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(h), _p(phase_rows(w.phases)),
                            len(w.phases), _p(_f64(w.glob)), _p(z), _p(hist),
                            _p(_u8(w.phase), ctypes.c_uint8), _p(mask, ctypes.c_uint8), _p(dvals),
                            1 if matrix else 0, _p(r), _p(hn), _p(flags, ctypes.c_uint8), _p(margins),
                            _p(geometry(w)))
    out = dict(r=r.reshape(4, m.nn), hist_new=hn, flags=flags, margins=margins)
    if matrix:
        nnz = L.orc_csr_nnz(handle)
        nd = 4 * m.nn
        indptr = np.zeros(nd + 1, dtype=np.int64)
        indices = np.zeros(nnz, dtype=np.int64)
        data = np.zeros(nnz)
        L.orc_csr_get(handle, _p(indptr, ctypes.c_longlong), _p(indices, ctypes.c_longlong), _p(data))
        L.orc_csr_free(handle)
        out["K"] = sp.csr_matrix((data, indices, indptr), shape=(nd, nd))
    return out


def sample_rows(w, dofs, x, z=None, hist=None):
    """For global DoFs ``dofs``: residual, (J x), (J^T x) and diag(J) entries."""
    m = w.mesh
    dofs = np.ascontiguousarray(dofs, dtype=np.int64)
    ns = len(dofs)
    z = _f64(w.z if z is None else z)
    hist = _f64(w.hist if hist is None else hist)
    x = _f64(x)
    dims, h = _mesh_args(m)
    r, jx, jtx, dg = np.zeros(ns), np.zeros(ns), np.zeros(ns), np.zeros(ns)
    lib().orc_sample_rows(dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(h), _p(phase_rows(w.phases)),
                          len(w.phases), _p(_f64(w.glob)), _p(z), _p(hist),
                          _p(_u8(w.phase), ctypes.c_uint8), _p(_u8(w.mask), ctypes.c_uint8),
                          _p(None if w.dvals is None else _f64(w.dvals)), _p(x), ns,
                          _p(dofs, ctypes.c_longlong), _p(r), _p(jx), _p(jtx), _p(dg), _p(geometry(w)))
    return dict(r=r, jx=jx, jtx=jtx, diag=dg)


def prolongation(mesh, pc: int, pf: int | None = None):
    """Sparse p-prolongation P (4 n_f x 4 n_c) from order pc to order pf (default
    mesh.p) on the element grid of ``mesh``: coarse Lagrange basis at fine nodes."""
    import scipy.sparse as sp

    pf = mesh.p if pf is None else pf
    dims = np.ascontiguousarray(mesh.dims, dtype=np.int32)
    L = lib()
    ip = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    n = L.orc_prolong_coo(ip, pc, pf, None, None, None)
    rows = np.zeros(n, dtype=np.int64)
    cols = np.zeros(n, dtype=np.int64)
    vals = np.zeros(n)
    L.orc_prolong_coo(ip, pc, pf, _p(rows, ctypes.c_longlong), _p(cols, ctypes.c_longlong), _p(vals))
    nf = (pf * mesh.nx + 1) * (pf * mesh.ny + 1) * (pf * mesh.nz + 1)
    nc = (pc * mesh.nx + 1) * (pc * mesh.ny + 1) * (pc * mesh.nz + 1)
    P1 = sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))
    return sp.block_diag([P1] * 4, format="csr")


def h_prolongation(nx: int, ny: int, nz: int):
    """Prolongation of vertex-centred full coarsening on a structured order-1
    grid of (2 nx, 2 ny, 2 nz) fine elements from (nx, ny, nz) coarse ones
    (4 n_f x 4 n_c, all four fields): the coarse hat functions evaluated at the
    fine vertices, P1[i, I] = max(0, 1 - |i / 2 - I|) per direction, and their
    tensor product (x fastest)."""
    import scipy.sparse as sp

    def one_d(nc):
        rows, cols, vals = [], [], []
        for i in range(2 * nc + 1):
            for I in range(nc + 1):
                v = max(0.0, 1.0 - abs(0.5 * i - I))
                if v > 0.0:
                    rows.append(i)
                    cols.append(I)
                    vals.append(v)
        return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc + 1, nc + 1))

    P1 = sp.kron(one_d(nz), sp.kron(one_d(ny), one_d(nx))).tocsr()
    return sp.block_diag([P1] * 4, format="csr")


def h_coarse_mask(mask_f, nx: int, ny: int, nz: int):
    """Coarse Dirichlet mask [4][n_c] of the h-coarsening: the mask of the
    coincident fine vertex (2 I, 2 J, 2 K)."""
    mf = np.asarray(mask_f).reshape(4, 2 * nz + 1, 2 * ny + 1, 2 * nx + 1)
    return np.ascontiguousarray(mf[:, ::2, ::2, ::2]).reshape(4, -1)


def masked_prolongation(P, mask_f, mask_c):
    """P with the rows of fine Dirichlet DoFs and columns of coarse Dirichlet
    DoFs removed: diag(1 - m_f) P diag(1 - m_c)."""
    import scipy.sparse as sp

    mf = 1.0 - np.asarray(mask_f, dtype=np.float64).ravel()
    mc = 1.0 - np.asarray(mask_c, dtype=np.float64).ravel()
    return (sp.diags(mf) @ P @ sp.diags(mc)).tocsr()


def coarse_operator(K_f, P, mask_c=None):
    """Galerkin coarse operator P^T K_f P, Dirichlet DoFs of the coarse level
    set to the identity (P must already be masked)."""
    import scipy.sparse as sp

    Kc = (P.T @ K_f @ P).tocsr()
    if mask_c is not None:
        mc = np.asarray(mask_c, dtype=bool).ravel()
        keep = sp.diags((~mc).astype(np.float64))
        Kc = (keep @ Kc @ keep + sp.diags(mc.astype(np.float64))).tocsr()
    return Kc


def chebyshev(A, diag, b, x0, degree: int, lmin: float, lmax: float):
    """Chebyshev iteration for A x = b preconditioned by D = diag(diag) on the
    eigenvalue interval [lmin, lmax] of D^-1 A (Saad, Iterative Methods for
    Sparse Linear Systems, Alg. 12.1): ``degree`` matrix-vector products, the
    error is multiplied by T_k((theta - D^-1 A)/delta) / T_k(theta/delta)."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.array(x0, dtype=np.float64, copy=True)
    r = (b - A @ x) / diag
    d = r / theta
    for k in range(degree):
        x = x + d
        if k == degree - 1:
            break
        r = r - (A @ d) / diag
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x


def vcycle(Ks, Ps, diags, lmaxs, r, degree=3, lo=0.1, hi=1.1, coarse_degree=16, coarse_lo=0.02):
    """Textbook p-multigrid V-cycle z = M^-1 r: on every level but the coarsest,
    Chebyshev(degree) pre-smoothing from 0 on [lo, hi] lambda_max, residual,
    restriction R = P^T, recursion, prolongation, Chebyshev post-smoothing; on the
    coarsest level Chebyshev(coarse_degree) from 0 on [coarse_lo, hi] lambda_max.
    Ks[l]: level matrices (fine first), Ps[l]: prolongation from level l+1 to l."""

    def cycle(l, b):
        K, d, lm = Ks[l], diags[l], lmaxs[l]
        x0 = np.zeros_like(b)
        if l == len(Ks) - 1:
            return chebyshev(K, d, b, x0, coarse_degree, coarse_lo * lm, hi * lm)
        x = chebyshev(K, d, b, x0, degree, lo * lm, hi * lm)
        rc = Ps[l].T @ (b - K @ x)
        x = x + Ps[l] @ cycle(l + 1, rc)
        return chebyshev(K, d, b, x, degree, lo * lm, hi * lm)

    return cycle(0, np.asarray(r, dtype=np.float64))


def newton(w, rtol=1e-12, maxit=20):
    """Newton's method on the assembled system with direct linear solves; returns
    the converged nodal state and the residual-norm history."""
    import scipy.sparse.linalg as spla

    z = np.array(w.z, dtype=np.float64).ravel()
    hist = []
    for _ in range(maxit + 1):
        out = assemble(w, z=z.reshape(4, -1))
        r = out["r"].ravel()
        hist.append(float(np.linalg.norm(r)))
        if hist[-1] <= rtol * hist[0] or hist[-1] == 0.0:
            break
        z = z - spla.spsolve(out["K"].tocsc(), r)
    return z.reshape(4, -1), hist, out


# ---------------------------------------------------------------------------
# Discrete adjoint of a load-step sequence (assembled transposes, direct solves)
# ---------------------------------------------------------------------------
# Parameter vector theta (12): for phase k in (0, 1) the six entries
# E_inf, nu_inf, sigma0, eta_d, Gc, l0 at 6 k + (0..5).
PARAM_SLOTS = (2, 3, 11, 7, 0, 1)   # positions in the 12-double phase row


def set_params(phases, theta):
    ph = np.array(phases, dtype=np.float64, copy=True)
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 6)
    for k in range(min(len(ph), len(th))):
        for j, slot in enumerate(PARAM_SLOTS):
            ph[k, slot] = th[k, j]
    return ph


def get_params(phases):
    return np.array([[p[s] for s in PARAM_SLOTS] for p in phases]).ravel()


def point_partials(inputs, hist, phase, phases, glob):
    """Values [n, 28] and partials [n, 28, 34] of (integrands, trial history) at n points."""
    inputs = _f64(inputs)
    n = inputs.shape[0]
    vals = np.zeros((n, 28))
    J = np.zeros((n, 28, 34))
    lib().orc_point_partials(n, _p(inputs), _p(_f64(hist)), _p(_u8(phase), ctypes.c_uint8), _p(phase_rows(phases)),
                             len(phases), _p(_f64(glob)), _p(vals), _p(J))
    return vals, J


def qpoint_inputs(mesh, y, X=None):
    dims, h = _mesh_args(mesh)
    out = np.zeros((mesh.nq, 14))
    lib().orc_qpoint_inputs(dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(h), _p(_f64(y)), _p(out),
                            _p(None if X is None else _f64(X)))
    return out[:, :13], out[:, 13]


def apply_bt(mesh, pseudo, weighted, X=None):
    dims, h = _mesh_args(mesh)
    out = np.zeros(4 * mesh.nn)
    lib().orc_apply_bt(dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(h), _p(_f64(pseudo)),
                       1 if weighted else 0, _p(out), _p(None if X is None else _f64(X)))
    return out


def load_steps(w, theta, nsteps, top, rtol=1e-13):
    """Forward load steps: step n imposes n times the workload's Dirichlet values,
    solves by Newton with direct solves and commits the trial history.  Returns
    reactions [nsteps], states z_n and committed histories h_0..h_nsteps."""
    import copy
    ww = copy.copy(w)
    ww.phases = set_params(w.phases, theta)
    z = np.array(w.z, dtype=np.float64, copy=True)
    hist = np.array(w.hist, dtype=np.float64, copy=True)
    mk = w.mask.astype(bool)
    zs, hs, F = [], [hist.copy()], []
    for n in range(1, nsteps + 1):
        ww.hist = hist
        ww.dvals = w.dvals * n
        z = z.copy()
        z[mk] = ww.dvals[mk]
        ww.z = z
        z, _, out = newton(ww, rtol=rtol)
        fint = assemble(ww, z=z, matrix=False, mask=None, dvals=None)["r"]
        F.append(float(fint[top.astype(bool)].sum()))
        zs.append(z.copy())
        hist = out["hist_new"]
        hs.append(hist.copy())
    return np.array(F), zs, hs


def adjoint_gradient(w, theta, nsteps, top, target):
    """Gradient of L = sum_n (F_n - target_n)^2 with respect to theta by the
    discrete adjoint: backward over the load steps, J_n^T lam = g with the
    assembled CSR transpose, local partials by dual numbers."""
    import copy
    import scipy.sparse.linalg as spla
    F, zs, hs = load_steps(w, theta, nsteps, top)
    ww = copy.copy(w)
    ww.phases = set_params(w.phases, theta)
    m = w.mesh
    mk = w.mask.astype(bool).ravel()
    sel = top.astype(np.float64).ravel()
    hbar = np.zeros((m.nq, 15))
    gtheta = np.zeros(12)
    for n in range(nsteps, 0, -1):
        z, hprev = zs[n - 1], hs[n - 1]
        ww.hist = hprev
        ww.dvals = w.dvals * n
        wF = 2.0 * (F[n - 1] - target[n - 1])
        a, wq = qpoint_inputs(m, z, geometry(w))
        _, Jp = point_partials(a, hprev.T.copy(), w.phase, ww.phases, w.glob)
        K = assemble(ww, z=z, matrix=True)["K"]
        Kint = assemble(ww, z=z, matrix=True, mask=None, dvals=None)["K"]
        qa = np.einsum("qr,qrc->qc", hbar, Jp[:, 13:28, 0:13])
        g = wF * (Kint.T @ sel) + apply_bt(m, qa, weighted=False, X=geometry(w))
        g[mk] = 0.0
        lam = spla.spsolve(K.T.tocsc(), g)
        pv, _ = qpoint_inputs(m, (wF * sel - lam).reshape(4, -1), geometry(w))
        p = pv * wq[:, None]
        hb_new = np.einsum("qr,qrc->qc", p, Jp[:, 0:13, 13:28]) + np.einsum("qr,qrc->qc", hbar, Jp[:, 13:28, 13:28])
        gq = np.einsum("qr,qrc->qc", p, Jp[:, 0:13, 28:34]) + np.einsum("qr,qrc->qc", hbar, Jp[:, 13:28, 28:34])
        for k in range(len(w.phases)):
            gtheta[6 * k:6 * k + 6] += gq[w.phase == k].sum(axis=0)
        hbar = hb_new
    return gtheta, F
