"""Host-side wiring of the libpff handles for a workload (device memory via
torch).  Marshalling only: every numerical step is a libpff call."""
from __future__ import annotations

import numpy as np
import torch

from . import pff
from .inputs import Workload, coarsen_mask, element_offsets


class Session:
    def __init__(self, w: Workload, levels=(), f32: bool = False, offsets: bool = False,
                 device: str = "cuda", stream=None, df: bool = False, bf16: bool = False):
        self.w = w
        self.dev = torch.device(device)
        self.stream = stream
        m = w.mesh
        self.ctx = pff.pff_create_context(w.phases, int(w.glob[0]), w.glob[1], w.glob[2], w.glob[3], w.glob[4])
        self.basis = pff.pff_create_basis(self.ctx, m.p, m.Q)
        self.offsets = None
        if offsets:
            self.offsets = torch.from_numpy(element_offsets(m)).to(self.dev)
        self.restr = pff.pff_create_restriction(self.ctx, (m.nx, m.ny, m.nz, *m.h), m.p, self.offsets, m.nn)
        self.op = pff.pff_create_operator(self.ctx, self.basis, self.restr)
        self.X = None
        if getattr(w, "X", None) is not None:  # mapped mesh
            self.X = torch.from_numpy(np.ascontiguousarray(w.X, dtype=np.float64)).to(self.dev)
            pff.pff_op_set_geometry(self.op, self.X, self.stream)
        if f32:
            pff.pff_op_enable_f32(self.op, True)
        if df:
            pff.pff_op_enable_df(self.op, True)
        if bf16:
            pff.pff_op_enable_bf16(self.op, True)
        self.phase = torch.from_numpy(np.ascontiguousarray(w.phase, dtype=np.uint8)).to(self.dev)
        self.set_history(w.hist)
        self.mask = None
        self.dvals = None
        if w.mask is not None:
            self.mask = torch.from_numpy(np.ascontiguousarray(w.mask, dtype=np.uint8).ravel()).to(self.dev)
            dv = w.dvals if w.dvals is not None else np.zeros(w.mask.shape)
            self.dvals = torch.from_numpy(np.ascontiguousarray(dv, dtype=np.float64).ravel()).to(self.dev)
            pff.pff_set_dirichlet(self.op, self.mask, self.dvals, self.stream)
        self.levels = {m.p: pff.pff_create_level(self.op, m.p)}
        self.level_masks = {}
        for p in levels:
            if p == m.p:
                continue
            L = pff.pff_create_level(self.op, p)
            self.levels[p] = L
            if w.mask is not None:
                mc = torch.from_numpy(coarsen_mask(m, w.mask, p).ravel()).to(self.dev)
                self.level_masks[p] = mc
                pff.pff_level_set_mask(L, mc, self.stream)

    # ------------------------------------------------------------------
    def set_history(self, hist):
        self.hist = torch.from_numpy(np.ascontiguousarray(hist, dtype=np.float64)).to(self.dev)
        pff.pff_set_qpoint_state(self.op, self.phase, self.hist, self.stream)

    def nn(self, p=None):
        m = self.w.mesh
        p = m.p if p is None else p
        return (p * m.nx + 1) * (p * m.ny + 1) * (p * m.nz + 1)

    def vec(self, p=None, dtype=torch.float64):
        return torch.zeros(4 * self.nn(p), dtype=dtype, device=self.dev)

    def residual(self, z):
        z = torch.as_tensor(np.ascontiguousarray(z, dtype=np.float64).ravel()).to(self.dev) if not torch.is_tensor(z) else z
        r = self.vec()
        pff.pff_residual(self.op, z, r, self.stream)
        return r

    def apply(self, x, p=None, prec=pff.PFF_F64, transpose=False):
        p = self.w.mesh.p if p is None else p
        y = torch.empty_like(x)
        fn = pff.pff_jacobian_transpose_apply if transpose else pff.pff_jacobian_apply
        fn(self.levels[p], prec, x, y, self.stream)
        return y

    def diag(self, p=None, prec=pff.PFF_F64):
        p = self.w.mesh.p if p is None else p
        d = self.vec(p, torch.float64 if prec == pff.PFF_F64 else torch.float32)
        pff.pff_assemble_diagonal(self.levels[p], prec, d, self.stream)
        return d

    def prolong(self, xc, pc, pf, prec=pff.PFF_F64):
        xf = self.vec(pf, xc.dtype)
        pff.pff_prolong(self.levels[pc], self.levels[pf], prec, xc, xf, self.stream)
        return xf

    def restrict(self, rf, pc, pf, prec=pff.PFF_F64):
        rc = self.vec(pc, rf.dtype)
        pff.pff_restrict(self.levels[pc], self.levels[pf], prec, rf, rc, self.stream)
        return rc

    def chebyshev(self, b, x, diag, degree, lmin, lmax, p=None, prec=pff.PFF_F64):
        p = self.w.mesh.p if p is None else p
        work = torch.zeros(3 * b.numel(), dtype=b.dtype, device=self.dev)
        pff.pff_chebyshev_smooth(self.levels[p], prec, degree, lmin, lmax, diag, b, x, work, self.stream)
        return x

    def solver(self, levels=None, **params):
        """FGMRES / p-multigrid solver over the given level orders (fine first)."""
        m = self.w.mesh
        levels = [m.p] + sorted([p for p in self.levels if p != m.p], reverse=True) if levels is None else levels
        prm = pff.pff_solver_default_params(**params)
        handles = [self.levels[p] for p in levels]
        return pff.pff_create_solver(self.op, handles, prm)

    def flags(self):
        f = torch.zeros(self.w.mesh.nq, dtype=torch.uint8, device=self.dev)
        pff.pff_get_flags(self.op, f, self.stream)
        return f

    def history(self, which=1):
        h = torch.zeros(15 * self.w.mesh.nq, dtype=torch.float64, device=self.dev)
        pff.pff_get_history(self.op, which, h, self.stream)
        return h.view(15, -1)

    def linearization(self):
        out = torch.zeros(67 * self.w.mesh.nq, dtype=torch.float64, device=self.dev)
        pff.pff_get_linearization(self.op, out, self.stream)
        return out.view(67, -1)

    def commit(self):
        pff.pff_commit_history(self.op, self.stream)

    def status(self):
        return pff.pff_get_status(self.op, self.stream)

    def close(self):
        for L in self.levels.values():
            pff.pff_destroy_level(L)
        self.levels = {}
        if self.op is not None:
            pff.pff_destroy_operator(self.op)
            pff.pff_destroy_restriction(self.restr)
            pff.pff_destroy_basis(self.basis)
            pff.pff_destroy_context(self.ctx)
            self.op = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
