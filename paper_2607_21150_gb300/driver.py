"""Load stepping (Sec. 5): for every load step, impose the step's Dirichlet
values, solve the coupled system with Newton-FGMRES/p-multigrid, commit the
quadrature-point history (Box 1 step 4) and record the reaction on the loaded
face.  Host logic only; every numerical step is a libpff call."""
from __future__ import annotations

import time

import numpy as np
import torch

from . import pff
from .inputs import Workload, node_coords, top_face_mask
from .session import Session


class LoadStepper:
    def __init__(self, w: Workload, levels=None, mixed: bool = True, session: Session | None = None,
                 df: bool = False, **solver_params):
        """df: the fine-level action inside FGMRES in double-float arithmetic
        (PFF_DF64) instead of FP64."""
        m = w.mesh
        if levels is None:
            levels = {4: [4, 2, 1], 3: [3, 1], 2: [2, 1], 1: [1]}[m.p]
        self.levels = list(levels)
        self.s = session or Session(w, levels=[p for p in self.levels if p != m.p], f32=mixed, df=df)
        if df:
            solver_params.setdefault("outer_prec", pff.PFF_DF64)
        self.solver = self.s.solver(self.levels, mixed=int(mixed), **solver_params)
        self.w = w
        self.z = torch.from_numpy(np.ascontiguousarray(w.z, dtype=np.float64).ravel()).to(self.s.dev)
        self.unit = np.ascontiguousarray(w.dvals if w.dvals is not None else np.zeros((4, m.nn)), dtype=np.float64)
        self.top = torch.from_numpy(top_face_mask(m).ravel()).to(self.s.dev)
        self.history = []
        # predictor: the per-step Dirichlet increment of the loaded face spread
        # linearly over the height (the homogeneous solution of the uniaxial test)
        Z = node_coords(m)[:, 2] / m.L[2]
        ext = np.zeros((4, m.nn))
        top = top_face_mask(m).astype(bool)
        if np.any(top[2]):
            ext[2] = float(np.mean(self.unit[2][top[2]])) * Z
        self.extension = torch.from_numpy(ext.ravel()).to(self.s.dev)
        self.loaded = 0.0

    def set_load(self, factor: float):
        vals = torch.from_numpy((self.unit * factor).ravel()).to(self.s.dev)
        pff.pff_set_dirichlet(self.s.op, self.s.mask, vals, self.s.stream)
        self._vals = vals  # keep alive until the copy ran
        pff.pff_apply_dirichlet(self.s.op, self.z, self.s.stream)

    def step(self, k: int):
        """Load step k (Dirichlet values = k times the workload's per-step values)."""
        t0 = time.perf_counter()
        pff.pff_vec_axpby(pff.PFF_F64, self.z.numel(), float(k) - self.loaded, self.extension, 1.0, self.z,
                          self.s.stream)
        self.loaded = float(k)
        self.set_load(float(k))
        stats = pff.pff_newton_solve(self.solver, self.z, self.s.stream)
        pff.pff_commit_history(self.s.op, self.s.stream)
        reaction = pff.pff_reaction(self.s.op, self.top, self.s.stream)[2]
        stats["reaction"] = reaction
        stats["wall_s"] = time.perf_counter() - t0
        stats["step"] = k
        self.history.append(stats)
        return stats

    def close(self):
        if self.solver is not None:
            pff.pff_destroy_solver(self.solver)
            self.solver = None
        self.s.close()
