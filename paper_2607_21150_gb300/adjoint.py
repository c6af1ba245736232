"""Differentiable reaction-force curve: load steps forward, discrete adjoint
backward, behind a torch.autograd.Function.

Forward: the load steps of a workload with per-phase parameters theta (12:
E_inf, nu_inf, sigma0, eta_d, Gc, l0 of each phase); the converged state z_n and
the committed history entering step n are checkpointed on the device at every
load-step boundary.  Backward: pff_adjoint_step walks the steps in reverse,
recomputing each step's linearisation from its checkpoint, solving the
transposed system and propagating the history adjoint; the result is
dLoss/dtheta for dLoss/dF given by autograd."""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import pff
from .driver import LoadStepper
from .inputs import Workload, top_face_mask, with_params


class ReactionCurveRunner:
    def __init__(self, w: Workload, nsteps: int, levels=None, mixed: bool = False, newton_rtol: float = 1e-11,
                 krylov_rtol: float = 1e-8, adjoint_rtol: float = 1e-10):
        self.w = w
        self.nsteps = nsteps
        self.levels = levels
        self.mixed = mixed
        self.newton_rtol = newton_rtol
        self.krylov_rtol = krylov_rtol
        self.adjoint_rtol = adjoint_rtol
        self.lsp = None

    def forward(self, theta) -> np.ndarray:
        if self.lsp is not None:
            self.lsp.close()
        w = copy.copy(self.w)
        w.phases = with_params(self.w.phases, theta)
        self.lsp = LoadStepper(w, levels=self.levels, mixed=self.mixed, newton_rtol=self.newton_rtol,
                               krylov_rtol=self.krylov_rtol)
        s = self.lsp.s
        self.sel = torch.from_numpy(top_face_mask(w.mesh).ravel()).to(s.dev)
        self.z_ckpt, self.h_ckpt, F = [], [], []
        for n in range(1, self.nsteps + 1):
            self.h_ckpt.append(s.history(0).clone())
            st = self.lsp.step(n)
            if not st["converged"]:
                raise RuntimeError(f"load step {n} did not converge: {st}")
            self.z_ckpt.append(self.lsp.z.clone())
            F.append(st["reaction"])
        return np.array(F)

    def backward(self, dLdF) -> np.ndarray:
        s = self.lsp.s
        nq = self.w.mesh.nq
        grad = np.zeros(6 * len(self.w.phases))
        hbar = None
        hb_prev = torch.zeros(15 * nq, dtype=torch.float64, device=s.dev)
        self.adjoint_iters = []
        for n in range(self.nsteps, 0, -1):
            its = pff.pff_adjoint_step(self.lsp.solver, self.z_ckpt[n - 1], self.h_ckpt[n - 1], self.sel,
                                       float(dLdF[n - 1]), hbar, hb_prev, grad, self.adjoint_rtol, 400,
                                       s.stream)
            self.adjoint_iters.append(its)
            hbar = hb_prev.clone()
        return grad

    def close(self):
        if self.lsp is not None:
            self.lsp.close()
            self.lsp = None


class ReactionCurve(torch.autograd.Function):
    """F = ReactionCurve.apply(theta, runner): reaction per load step (CPU tensor);
    gradients flow to theta through the discrete adjoint."""

    @staticmethod
    def forward(ctx, theta, runner):
        ctx.runner = runner
        F = runner.forward(theta.detach().cpu().double().numpy())
        return torch.as_tensor(F, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, gF):
        g = ctx.runner.backward(gF.detach().cpu().double().numpy())
        return torch.as_tensor(g, dtype=gF.dtype), None
