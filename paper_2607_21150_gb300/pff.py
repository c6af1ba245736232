"""Thin ctypes binding of libpff (include/pff.h): same names, argument
marshalling only.  Every computation runs in the CUDA library; if the library
is missing this module raises instead of falling back to anything else.

Pointer arguments accept torch tensors (their ``data_ptr()``), plain integers
or ``None``; streams accept a ``torch.cuda.Stream``, an integer handle or
``None`` (the current torch stream)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PFF_F64 = 0
PFF_F32 = 1
PFF_DF64 = 2
PFF_F32_BF16 = 3
PFF_PROBE_DFMA, PFF_PROBE_FFMA, PFF_PROBE_DMMA, PFF_PROBE_CVT = 0, 1, 2, 3
STATUS_EIGEN, STATUS_DETF, STATUS_NONFINITE = 1, 2, 4

_lib = None


ERR_INVALID, ERR_CUDA, ERR_DEVICE, ERR_UNSUPPORTED = -1, -2, -3, -4


class PffError(RuntimeError):
    """A libpff call returned a PFF_ERR_* code (``code``); ERR_DEVICE means a
    kernel status word was set (det F <= 0, non-finite values, ...) or a solve
    found no admissible step, with the device context intact."""

    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


class pff_problem(ctypes.Structure):
    _fields_ = [("nphase", ctypes.c_int), ("phase_params", ctypes.POINTER(ctypes.c_double)),
                ("at", ctypes.c_int), ("eta", ctypes.c_double), ("zeta", ctypes.c_double),
                ("dt", ctypes.c_double), ("s_phi", ctypes.c_double)]


class pff_box(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double)]


class pff_solver_params(ctypes.Structure):
    _fields_ = [("mixed", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("coarse_degree", ctypes.c_int), ("coarse_lo", ctypes.c_double),
                ("power_iters", ctypes.c_int), ("krylov_restart", ctypes.c_int), ("krylov_maxit", ctypes.c_int),
                ("krylov_rtol", ctypes.c_double), ("newton_maxit", ctypes.c_int), ("newton_rtol", ctypes.c_double),
                ("line_search_max", ctypes.c_int), ("coarse_solver", ctypes.c_int), ("coarse_rtol", ctypes.c_double),
                ("coarse_maxit", ctypes.c_int), ("verbose", ctypes.c_int), ("outer_prec", ctypes.c_int),
                ("newton_stall", ctypes.c_int), ("eig_every", ctypes.c_int), ("level_words", ctypes.c_int)]


class pff_newton_stats(ctypes.Structure):
    _fields_ = [("newton_iterations", ctypes.c_int), ("krylov_iterations", ctypes.c_int),
                ("converged", ctypes.c_int), ("status", ctypes.c_int), ("line_search_cuts", ctypes.c_int),
                ("coarse_iterations", ctypes.c_int),
                ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("last_krylov_relres", ctypes.c_double),
                ("t_residual", ctypes.c_double), ("t_setup", ctypes.c_double), ("t_krylov", ctypes.c_double),
                ("res_history", ctypes.c_double * 64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "res_history"}
        d["res_history"] = list(self.res_history[:max(1, self.newton_iterations + 1)])
        return d


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_I64 = ctypes.c_int64

_SIGS = {
    "pff_last_error_message": ([], ctypes.c_char_p),
    "pff_version": ([], _I),
    "pff_kernel_launches": ([], _I64),
    "pff_create_context": ([ctypes.POINTER(_VP), ctypes.POINTER(pff_problem)], _I),
    "pff_destroy_context": ([_VP], _I),
    "pff_context_set_time_step": ([_VP, _D], _I),
    "pff_context_set_hardening": ([_VP, _I, _D, _D, _D], _I),
    "pff_create_basis": ([_VP, _I, _I, ctypes.POINTER(_VP)], _I),
    "pff_basis_get": ([_VP, _VP, _VP, _VP, _VP, _VP], _I),
    "pff_destroy_basis": ([_VP], _I),
    "pff_create_restriction": ([_VP, ctypes.POINTER(pff_box), _I, _VP, _I64, ctypes.POINTER(_VP)], _I),
    "pff_destroy_restriction": ([_VP], _I),
    "pff_create_operator": ([_VP, _VP, _VP, ctypes.POINTER(_VP)], _I),
    "pff_destroy_operator": ([_VP], _I),
    "pff_op_enable_f32": ([_VP, _I], _I),
    "pff_op_enable_df": ([_VP, _I], _I),
    "pff_op_enable_bf16": ([_VP, _I], _I),
    "pff_op_set_deterministic": ([_VP, _I], _I),
    "pff_op_set_geometry": ([_VP, _VP, _VP], _I),
    "pff_op_num_qpoints": ([_VP], _I64),
    "pff_op_num_nodes": ([_VP], _I64),
    "pff_set_qpoint_state": ([_VP, _VP, _VP, _VP], _I),
    "pff_set_dirichlet": ([_VP, _VP, _VP, _VP], _I),
    "pff_residual": ([_VP, _VP, _VP, _VP], _I),
    "pff_apply_dirichlet": ([_VP, _VP, _VP], _I),
    "pff_reaction": ([_VP, _VP, ctypes.POINTER(_D), _VP], _I),
    "pff_create_level": ([_VP, _I, ctypes.POINTER(_VP)], _I),
    "pff_destroy_level": ([_VP], _I),
    "pff_level_num_nodes": ([_VP], _I64),
    "pff_level_set_mask": ([_VP, _VP, _VP], _I),
    "pff_jacobian_apply": ([_VP, _I, _VP, _VP, _VP], _I),
    "pff_jacobian_transpose_apply": ([_VP, _I, _VP, _VP, _VP], _I),
    "pff_jacobian_apply_host": ([_VP, _I, _VP, _VP, _I, _VP], _I),
    "pff_assemble_diagonal": ([_VP, _I, _VP, _VP], _I),
    "pff_prolong": ([_VP, _VP, _I, _VP, _VP, _VP], _I),
    "pff_restrict": ([_VP, _VP, _I, _VP, _VP, _VP], _I),
    "pff_chebyshev_smooth": ([_VP, _I, _I, _D, _D, _VP, _VP, _VP, _VP, _VP], _I),
    "pff_chebyshev_smooth_noalloc": ([_VP, _I, _I, _D, _D, _VP, _VP, _VP, _VP], _I),
    "pff_solver_default_params": ([ctypes.POINTER(pff_solver_params)], _I),
    "pff_create_solver": ([_VP, _I, ctypes.POINTER(_VP), ctypes.POINTER(pff_solver_params), ctypes.POINTER(_VP)], _I),
    "pff_destroy_solver": ([_VP], _I),
    "pff_solver_setup": ([_VP, _VP], _I),
    "pff_solver_level_lambda": ([_VP, _I, ctypes.POINTER(_D)], _I),
    "pff_solver_vcycle": ([_VP, _VP, _VP, _VP], _I),
    "pff_solver_coarse_apply": ([_VP, _VP, _VP, _VP], _I),
    "pff_solver_num_hlevels": ([_VP], _I),
    "pff_solver_hlevel_info": ([_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "pff_solver_hlevel_apply": ([_VP, _I, _VP, _VP, _VP], _I),
    "pff_solver_hcycle": ([_VP, _VP, _VP, _VP], _I),
    "pff_solver_krylov": ([_VP, _VP, _VP, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _VP], _I),
    "pff_newton_solve": ([_VP, _VP, ctypes.POINTER(pff_newton_stats), _VP], _I),
    "pff_vec_axpby": ([_I, _I64, _D, _VP, _D, _VP, _VP], _I),
    "pff_adjoint_step": ([_VP, _VP, _VP, _VP, _D, _VP, _VP, ctypes.POINTER(_D), _D, _I, ctypes.POINTER(_I), _VP], _I),
    "pff_commit_history": ([_VP, _VP], _I),
    "pff_get_history": ([_VP, _I, _VP, _VP], _I),
    "pff_get_flags": ([_VP, _VP, _VP], _I),
    "pff_get_linearization": ([_VP, _VP, _VP], _I),
    "pff_get_status": ([_VP, _VP, ctypes.POINTER(_I)], _I),
    "pff_state_summary": ([_VP, _VP, ctypes.POINTER(_D), _VP], _I),
    "pff_probe_pipe": ([_I, _I64, _I, _I, _VP, ctypes.POINTER(_D), _VP], _I),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libpff.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise PffError(f"libpff.so is not built ({path}); run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, ctypes.c_void_p):
        return x.value
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, name):
    if rc != 0:
        msg = lib().pff_last_error_message()
        raise PffError(f"{name} failed ({rc}): {msg.decode() if msg else ''}", rc)


def _call(name, *args):
    rc = getattr(lib(), name)(*args)
    _check(rc, name)


# ---------------------------------------------------------------- handles
def pff_create_context(phase_params, at, eta, zeta, dt, s_phi):
    import numpy as np
    rows = np.atleast_2d(np.asarray(phase_params, dtype=np.float64))
    pp = np.ascontiguousarray(rows[:, :12])
    pr = pff_problem(len(pp), pp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(at), float(eta),
                     float(zeta), float(dt), float(s_phi))
    h = _VP()
    _call("pff_create_context", ctypes.byref(h), ctypes.byref(pr))
    if rows.shape[1] == 15:  # hardening law of the Prandtl branches
        for k, r in enumerate(rows):
            if r[8] and (r[12] != 0.0 or r[13] != r[11]):
                pff_context_set_hardening(h, k, r[12], r[13], r[14])
    return h


def pff_destroy_context(ctx):
    _call("pff_destroy_context", ctx)


def pff_context_set_time_step(ctx, dt):
    _call("pff_context_set_time_step", ctx, float(dt))


def pff_context_set_hardening(ctx, phase, H_lin, sigma_inf, beta):
    _call("pff_context_set_hardening", ctx, int(phase), float(H_lin), float(sigma_inf), float(beta))


def pff_create_basis(ctx, p, q):
    h = _VP()
    _call("pff_create_basis", ctx, int(p), int(q), ctypes.byref(h))
    return h


def pff_basis_get(basis, p, q):
    import numpy as np
    P = p + 1
    xg, xq, wq = np.zeros(P), np.zeros(q), np.zeros(q)
    B, Dc = np.zeros((q, P)), np.zeros((q, q))
    _call("pff_basis_get", basis, xg.ctypes.data, xq.ctypes.data, wq.ctypes.data, B.ctypes.data, Dc.ctypes.data)
    return xg, xq, wq, B, Dc


def pff_destroy_basis(basis):
    _call("pff_destroy_basis", basis)


def pff_create_restriction(ctx, box, p, offsets, nnodes):
    """box = (nx, ny, nz, hx, hy, hz)."""
    b = pff_box(int(box[0]), int(box[1]), int(box[2]), float(box[3]), float(box[4]), float(box[5]))
    h = _VP()
    _call("pff_create_restriction", ctx, ctypes.byref(b), int(p), _ptr(offsets), int(nnodes), ctypes.byref(h))
    return h


def pff_destroy_restriction(r):
    _call("pff_destroy_restriction", r)


def pff_create_operator(ctx, basis, restr):
    h = _VP()
    _call("pff_create_operator", ctx, basis, restr, ctypes.byref(h))
    return h


def pff_destroy_operator(op):
    _call("pff_destroy_operator", op)


def pff_op_enable_f32(op, enable=True):
    _call("pff_op_enable_f32", op, 1 if enable else 0)


def pff_op_enable_df(op, enable=True):
    _call("pff_op_enable_df", op, 1 if enable else 0)


def pff_op_enable_bf16(op, enable=True):
    _call("pff_op_enable_bf16", op, 1 if enable else 0)


def pff_op_set_deterministic(op, enable=True):
    _call("pff_op_set_deterministic", op, 1 if enable else 0)


def pff_op_set_geometry(op, X, stream=None):
    _call("pff_op_set_geometry", op, _ptr(X), _stream(stream))


def pff_op_num_qpoints(op):
    return int(lib().pff_op_num_qpoints(op))


def pff_op_num_nodes(op):
    return int(lib().pff_op_num_nodes(op))


def pff_set_qpoint_state(op, phase, hist, stream=None):
    _call("pff_set_qpoint_state", op, _ptr(phase), _ptr(hist), _stream(stream))


def pff_set_dirichlet(op, mask, values, stream=None):
    _call("pff_set_dirichlet", op, _ptr(mask), _ptr(values), _stream(stream))


def pff_residual(op, z, r, stream=None):
    _call("pff_residual", op, _ptr(z), _ptr(r), _stream(stream))


def pff_apply_dirichlet(op, z, stream=None):
    _call("pff_apply_dirichlet", op, _ptr(z), _stream(stream))


def pff_reaction(op, sel, stream=None):
    out = (_D * 4)()
    _call("pff_reaction", op, _ptr(sel), out, _stream(stream))
    return [float(v) for v in out]


def pff_create_level(op, p):
    h = _VP()
    _call("pff_create_level", op, int(p), ctypes.byref(h))
    return h


def pff_destroy_level(level):
    _call("pff_destroy_level", level)


def pff_level_num_nodes(level):
    return int(lib().pff_level_num_nodes(level))


def pff_level_set_mask(level, mask, stream=None):
    _call("pff_level_set_mask", level, _ptr(mask), _stream(stream))


def pff_jacobian_apply(level, prec, x, y, stream=None):
    _call("pff_jacobian_apply", level, int(prec), _ptr(x), _ptr(y), _stream(stream))


def pff_jacobian_transpose_apply(level, prec, x, y, stream=None):
    _call("pff_jacobian_transpose_apply", level, int(prec), _ptr(x), _ptr(y), _stream(stream))


def pff_jacobian_apply_host(level, prec, x_host, y_host, nchunks=8, stream=None):
    """y = J x with x, y in (page-locked) host memory, the copies overlapped
    with the computation; asynchronous on the stream."""
    _call("pff_jacobian_apply_host", level, int(prec), _ptr(x_host), _ptr(y_host), int(nchunks), _stream(stream))


def pff_assemble_diagonal(level, prec, diag, stream=None):
    _call("pff_assemble_diagonal", level, int(prec), _ptr(diag), _stream(stream))


def pff_prolong(coarse, fine, prec, xc, xf, stream=None):
    _call("pff_prolong", coarse, fine, int(prec), _ptr(xc), _ptr(xf), _stream(stream))


def pff_restrict(coarse, fine, prec, rf, rc, stream=None):
    _call("pff_restrict", coarse, fine, int(prec), _ptr(rf), _ptr(rc), _stream(stream))


def pff_chebyshev_smooth(level, prec, degree, lmin, lmax, diag, b, x, work, stream=None):
    _call("pff_chebyshev_smooth", level, int(prec), int(degree), float(lmin), float(lmax), _ptr(diag), _ptr(b),
          _ptr(x), _ptr(work), _stream(stream))


def pff_chebyshev_smooth_noalloc(level, prec, degree, lmin, lmax, diag, b, x, stream=None):
    """Chebyshev smoothing with the library's built-in work space (no allocation)."""
    _call("pff_chebyshev_smooth_noalloc", level, int(prec), int(degree), float(lmin), float(lmax), _ptr(diag),
          _ptr(b), _ptr(x), _stream(stream))


def pff_solver_default_params(**overrides):
    prm = pff_solver_params()
    _call("pff_solver_default_params", ctypes.byref(prm))
    for k, v in overrides.items():
        setattr(prm, k, v)
    return prm


def pff_create_solver(op, levels, params):
    arr = (_VP * len(levels))(*[lv.value if isinstance(lv, _VP) else lv for lv in levels])
    h = _VP()
    _call("pff_create_solver", op, len(levels), arr, ctypes.byref(params), ctypes.byref(h))
    return h


def pff_destroy_solver(solver):
    _call("pff_destroy_solver", solver)


def pff_solver_setup(solver, stream=None):
    _call("pff_solver_setup", solver, _stream(stream))


def pff_solver_level_lambda(solver, level):
    v = _D()
    _call("pff_solver_level_lambda", solver, int(level), ctypes.byref(v))
    return float(v.value)


def pff_solver_vcycle(solver, r, z, stream=None):
    _call("pff_solver_vcycle", solver, _ptr(r), _ptr(z), _stream(stream))


def pff_solver_coarse_apply(solver, x, y, stream=None):
    _call("pff_solver_coarse_apply", solver, _ptr(x), _ptr(y), _stream(stream))


def pff_solver_num_hlevels(solver):
    return int(lib().pff_solver_num_hlevels(solver))


def pff_solver_hlevel_info(solver, level):
    """(element grid (nx, ny, nz), lambda_max estimate) of h-level ``level``."""
    dims = (_I * 3)()
    lam = _D()
    _call("pff_solver_hlevel_info", solver, int(level), dims, ctypes.byref(lam))
    return (dims[0], dims[1], dims[2]), lam.value


def pff_solver_hlevel_apply(solver, level, x, y, stream=None):
    _call("pff_solver_hlevel_apply", solver, int(level), _ptr(x), _ptr(y), _stream(stream))


def pff_solver_hcycle(solver, b, x, stream=None):
    _call("pff_solver_hcycle", solver, _ptr(b), _ptr(x), _stream(stream))


def pff_solver_krylov(solver, b, x, rtol, maxit, stream=None):
    it = _I()
    rel = _D()
    _call("pff_solver_krylov", solver, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(it),
          ctypes.byref(rel), _stream(stream))
    return int(it.value), float(rel.value)


def pff_newton_solve(solver, z, stream=None):
    st = pff_newton_stats()
    _call("pff_newton_solve", solver, _ptr(z), ctypes.byref(st), _stream(stream))
    return st.as_dict()


def pff_vec_axpby(prec, n, a, x, b, y, stream=None):
    _call("pff_vec_axpby", int(prec), int(n), float(a), _ptr(x), float(b), _ptr(y), _stream(stream))


def pff_adjoint_step(solver, z, hist_prev, sel, wF, hbar_n, hbar_prev, grad, rtol=1e-10, maxit=400, stream=None):
    """One reverse load step; grad (numpy float64 array of 6 nphase) is accumulated in place."""
    import numpy as np
    g = np.ascontiguousarray(grad, dtype=np.float64)
    it = _I()
    _call("pff_adjoint_step", solver, _ptr(z), _ptr(hist_prev), _ptr(sel), float(wF), _ptr(hbar_n), _ptr(hbar_prev),
          g.ctypes.data_as(ctypes.POINTER(_D)), float(rtol), int(maxit), ctypes.byref(it), _stream(stream))
    grad[:] = g
    return int(it.value)


def pff_commit_history(op, stream=None):
    _call("pff_commit_history", op, _stream(stream))


def pff_get_history(op, which, hist, stream=None):
    _call("pff_get_history", op, int(which), _ptr(hist), _stream(stream))


def pff_get_flags(op, flags, stream=None):
    _call("pff_get_flags", op, _ptr(flags), _stream(stream))


def pff_get_linearization(op, out, stream=None):
    _call("pff_get_linearization", op, _ptr(out), _stream(stream))


def pff_get_status(op, stream=None):
    st = _I()
    _call("pff_get_status", op, _stream(stream), ctypes.byref(st))
    return int(st.value)


def pff_probe_pipe(kind, iters, blocks, threads, sink, stream=None):
    """Launch the pipe-rate probe; returns the flops the launch performs."""
    f = _D()
    _call("pff_probe_pipe", int(kind), int(iters), int(blocks), int(threads), _ptr(sink), ctypes.byref(f),
          _stream(stream))
    return f.value


def pff_kernel_launches():
    """Kernels libpff has launched in this process so far."""
    return int(lib().pff_kernel_launches())


STATE_SUMMARY_KEYS = ("n_yield", "n_active", "n_tension", "phi_max", "phi_min", "n_phi_above_0.9", "eps_p_max",
                      "H_max")


def pff_state_summary(op, z, stream=None):
    """Per-step state summary (dict with STATE_SUMMARY_KEYS)."""
    out = (_D * 8)()
    _call("pff_state_summary", op, _ptr(z), out, _stream(stream))
    return dict(zip(STATE_SUMMARY_KEYS, [float(v) for v in out]))
