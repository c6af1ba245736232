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


class StaleCheckpoints(RuntimeError):
    """backward() was asked for a forward run whose checkpoints were replaced."""


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
        self.generation = 0   # forward runs so far; the checkpoints belong to the last one

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
        self.generation += 1
        F, self.schedule = [], []
        for n in range(1, self.nsteps + 1):
            out = self.lsp.advance(n, None if schedule is None else schedule[n - 1])
            self.schedule.append([st["load"] for st in out])
            F.append(out[-1]["reaction"])
        return np.array(F)

    def backward(self, dLdF, generation: int | None = None) -> np.ndarray:
        """dLoss/dtheta of the last forward run; `generation` (the value of
        self.generation right after the forward run it belongs to) must be that
        run, else StaleCheckpoints."""
        if generation is not None and generation != self.generation:
            raise StaleCheckpoints(f"backward for forward run {generation}, but the runner holds the checkpoints "
                                   f"of run {self.generation}: repeat the forward run before differentiating it")
        if self.lsp is None:
            raise StaleCheckpoints("backward without a forward run (or after close())")
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
        self.generation += 1


class ReactionCurve(torch.autograd.Function):
    """F = ReactionCurve.apply(theta, runner): reaction per load step (CPU tensor);
    gradients flow to theta through the discrete adjoint.  The graph's backward
    needs the runner's checkpoints of this very forward run: if the runner ran
    forward again in between, backward raises StaleCheckpoints."""

    @staticmethod
    def forward(ctx, theta, runner):
        ctx.runner = runner
        F = runner.forward(theta.detach().cpu().double().numpy())
        ctx.generation = runner.generation
        return torch.as_tensor(F, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, gF):
        g = ctx.runner.backward(gF.detach().cpu().double().numpy(), ctx.generation)
        return torch.as_tensor(g, dtype=gF.dtype), None
