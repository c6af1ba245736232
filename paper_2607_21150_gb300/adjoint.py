"""Differentiable reaction-force curve: load steps forward, discrete adjoint
backward, behind a torch.autograd.Function.

Forward: the load steps of a workload with per-phase parameters theta (12:
E_inf, nu_inf, sigma0, eta_d, Gc, l0 of each phase), each advanced with the
adaptive cut-back of LoadStepper.advance; the converged state and the committed
history entering every converged sub-step are checkpointed on the device with
the sub-step's time step.  Backward: pff_adjoint_step walks the sub-steps in
reverse, recomputing each one's linearisation from its checkpoint (with its
time step), solving the transposed system and propagating the history adjoint;
the reaction weights dLoss/dF enter at the sub-steps that end a load step.  The
result is dLoss/dtheta for the dLoss/dF given by autograd.  `schedule` replays
a recorded sub-step sequence (finite-difference checks must keep it fixed)."""
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

    def forward(self, theta, schedule=None) -> np.ndarray:
        if self.lsp is not None:
            self.lsp.close()
        w = copy.copy(self.w)
        w.phases = with_params(self.w.phases, theta)
        self.lsp = LoadStepper(w, levels=self.levels, mixed=self.mixed, newton_rtol=self.newton_rtol,
                               krylov_rtol=self.krylov_rtol)
        s = self.lsp.s
        self.sel = torch.from_numpy(top_face_mask(w.mesh).ravel()).to(s.dev)
        self.subs = []  # converged sub-steps: state after, history before, time step, end factor

        def record(f0, f1, dt, hist_before, stats):
            self.subs.append({"z": self.lsp.z.clone(), "h": hist_before, "dt": dt, "f1": f1})

        self.lsp.on_substep = record
        F, self.schedule = [], []
        for n in range(1, self.nsteps + 1):
            out = self.lsp.advance(n, None if schedule is None else schedule[n - 1])
            self.schedule.append([st["load"] for st in out])
            F.append(out[-1]["reaction"])
        return np.array(F)

    def backward(self, dLdF) -> np.ndarray:
        s = self.lsp.s
        nq = self.w.mesh.nq
        grad = np.zeros(6 * len(self.w.phases))
        hbar = None
        hb_prev = torch.zeros(15 * nq, dtype=torch.float64, device=s.dev)
        self.adjoint_iters = []
        for sub in reversed(self.subs):
            n = int(sub["f1"])
            wF = float(dLdF[n - 1]) if sub["f1"] == n else 0.0
            pff.pff_context_set_time_step(s.ctx, sub["dt"])
            its = pff.pff_adjoint_step(self.lsp.solver, sub["z"], sub["h"], self.sel, wF, hbar, hb_prev, grad,
                                       self.adjoint_rtol, 400, s.stream)
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
