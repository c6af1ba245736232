"""Load stepping (Sec. 5): for every load step, impose the step's Dirichlet
values, solve the coupled system with Newton-FGMRES/p-multigrid, commit the
quadrature-point history (Box 1 step 4) and record the reaction on the loaded
face.  A step whose Newton solve fails is retried from the last converged state
with half the load increment and half the time step (adaptive cut-back), and
the increment grows again after successes.  Host logic only; every numerical
step is a libpff call."""
from __future__ import annotations

import time

import numpy as np
import torch

from . import pff
from .inputs import Workload, node_coords, top_face_mask
from .session import Session


class StepFailed(RuntimeError):
    pass


def _jsonable(x):
    """Plain Python numbers, lists and dicts of x (numpy scalars and arrays converted)."""
    if isinstance(x, dict):
        return {str(k): _jsonable(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_jsonable(v) for v in x]
    if isinstance(x, np.ndarray):
        return x.tolist()
    if isinstance(x, (np.floating, np.integer)):
        return x.item()
    return x


class StepController:
    """Adaptive sub-stepping of the load factor from `start` to `target`.

    attempt(f_from, f_to) -> bool runs one sub-step (load factor and time both
    advance by f_to - f_from in units of the nominal step) and reports whether
    it converged; a failed attempt must leave the state at f_from.  After a
    failure the increment is halved (at most `max_cuts` failures in a row);
    after `grow_after` successes in a row at the same increment it grows by
    `grow`, never past `target` (grow_after = 1: after every success; 2 keeps
    a halved increment for two sub-steps, which saves the attempts that fail
    when the softening regime needs the smaller increment for a while).
    Increments are dyadic fractions of the nominal step, so the sub-step ends
    are exact."""

    def __init__(self, max_cuts: int = 6, grow: float = 2.0, grow_after: int = 1):
        self.max_cuts = max_cuts
        self.grow = grow
        self.grow_after = max(1, int(grow_after))

    def run(self, start: float, target: float, attempt, first: float | None = None):
        f = float(start)
        inc = float(target - start) if first is None else float(first)
        done, cuts, wins = [], 0, 0
        while f < target:
            inc = min(inc, target - f)
            f_to = target if f + inc >= target else f + inc
            if attempt(f, f_to):
                done.append((f, f_to))
                f = f_to
                cuts = 0
                wins += 1
                if wins >= self.grow_after:
                    inc *= self.grow
                    wins = 0
            else:
                cuts += 1
                wins = 0
                if cuts > self.max_cuts:
                    raise StepFailed(f"no convergence from load factor {f} after {self.max_cuts} cuts")
                inc *= 0.5
        return done


class LoadStepper:
    def __init__(self, w: Workload, levels=None, mixed: bool = True, session: Session | None = None,
                 df: bool | None = None, max_cuts: int = 6, grow_after: int = 1, **solver_params):
        """df: the fine-level action inside FGMRES in double-float arithmetic
        (PFF_DF64) instead of FP64; by default on with mixed precision (same
        converged fields to ~1e-15, half the time of the FP64 action).
        max_cuts: consecutive halvings of a failing load increment before
        `advance` gives up; grow_after: successes in a row before a cut
        increment grows again (StepController).  solver_params: fields of pff_solver_params, e.g.
        level_words=16 for BF16 words in the FP32 levels."""
        if df is None:
            df = mixed
        m = w.mesh
        if levels is None:
            levels = {4: [4, 2, 1], 3: [3, 1], 2: [2, 1], 1: [1]}[m.p]
        self.levels = list(levels)
        bf16 = mixed and solver_params.get("level_words", 32) == 16
        self.s = session or Session(w, levels=[p for p in self.levels if p != m.p], f32=mixed, df=df, bf16=bf16)
        if df:
            solver_params.setdefault("outer_prec", pff.PFF_DF64)
        solver_params.setdefault("newton_stall", 6)  # a stagnating solve hands over to the cut-back early
        self.solver = self.s.solver(self.levels, mixed=int(mixed), **solver_params)
        self.w = w
        self.dt = float(w.glob[3])
        self.controller = StepController(max_cuts=max_cuts, grow_after=grow_after)
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
        # callback(f_from, f_to, dt, hist_before, stats) after every converged sub-step of `advance`
        self.on_substep = None
        # per committed sub-step: state summary (flag counts, phi extremes, ...) and the
        # lambda_max estimates of the levels
        self.diagnostics = False
        self.failures = []   # sub-steps that did not converge (undone), with their solver stats

    def set_load(self, factor: float):
        vals = torch.from_numpy((self.unit * factor).ravel()).to(self.s.dev)
        pff.pff_set_dirichlet(self.s.op, self.s.mask, vals, self.s.stream)
        self._vals = vals  # keep alive until the copy ran
        pff.pff_apply_dirichlet(self.s.op, self.z, self.s.stream)

    def _solve_to(self, factor: float, dt: float):
        """Predictor, Dirichlet values and Newton at load factor `factor` with time step dt."""
        pff.pff_context_set_time_step(self.s.ctx, dt)
        pff.pff_vec_axpby(pff.PFF_F64, self.z.numel(), factor - self.loaded, self.extension, 1.0, self.z,
                          self.s.stream)
        self.set_load(factor)
        return pff.pff_newton_solve(self.solver, self.z, self.s.stream)

    def _commit(self, factor: float, stats, t0: float):
        pff.pff_commit_history(self.s.op, self.s.stream)
        stats["reaction"] = pff.pff_reaction(self.s.op, self.top, self.s.stream)[2]
        if self.diagnostics:
            stats["state"] = pff.pff_state_summary(self.s.op, self.z, self.s.stream)
            stats["lambda_max"] = [pff.pff_solver_level_lambda(self.solver, l) for l in range(len(self.levels))]
        stats["wall_s"] = time.perf_counter() - t0
        stats["load"] = factor
        self.loaded = factor
        self.history.append(stats)
        return stats

    # ------------------------------------------------------------ checkpoints
    def state_dict(self):
        """Everything a later run needs to continue from the last committed
        load factor: the state z, the committed quadrature-point history, the
        phase map (to check that a resume uses the same microstructure), the
        load factor and the nominal time step (host arrays)."""
        if self.z.is_cuda:
            torch.cuda.synchronize()
        return {"z": self.z.cpu().numpy().copy(), "hist": self.s.history(0).cpu().numpy().copy(),
                "phase": np.ascontiguousarray(self.w.phase, dtype=np.uint8).copy(),
                "loaded": float(self.loaded), "dt": float(self.dt)}

    def load_state_dict(self, d):
        """Continue from a state_dict: z, committed history, load factor (and
        its Dirichlet values); refuses a different mesh or phase map."""
        if d["z"].size != self.z.numel() or d["hist"].shape != (15, self.w.mesh.nq):
            raise ValueError("checkpoint of a different mesh")
        if not np.array_equal(d["phase"], np.asarray(self.w.phase, dtype=np.uint8)):
            raise ValueError("checkpoint of a different microstructure (phase map)")
        self.dt = float(d["dt"])
        self.s.set_history(d["hist"])
        self.z.copy_(torch.from_numpy(np.ascontiguousarray(d["z"], dtype=np.float64).ravel()))
        self.loaded = float(d["loaded"])
        self.set_load(self.loaded)
        if self.z.is_cuda:
            torch.cuda.synchronize()

    def save_checkpoint(self, path: str, meta: dict | None = None):
        """Writes state_dict() to directory `path` (z.npy, hist.npy, phase.npy,
        meta.json with the load factor, time step, per-step log and `meta`);
        files are written under temporary names and renamed, so that an
        interrupted save leaves the previous checkpoint intact."""
        import json
        import os
        d = self.state_dict()
        os.makedirs(path, exist_ok=True)
        for k in ("z", "hist", "phase"):
            np.save(os.path.join(path, k + ".tmp.npy"), d[k])
        info = {"loaded": d["loaded"], "dt": d["dt"], "log": _jsonable(self.history), **(meta or {})}
        with open(os.path.join(path, "meta.tmp.json"), "w") as f:
            json.dump(info, f)
        for k in ("z", "hist", "phase"):
            os.replace(os.path.join(path, k + ".tmp.npy"), os.path.join(path, k + ".npy"))
        os.replace(os.path.join(path, "meta.tmp.json"), os.path.join(path, "meta.json"))

    def load_checkpoint(self, path: str) -> dict:
        """Continues from a checkpoint written by save_checkpoint; returns its meta."""
        import json
        import os
        with open(os.path.join(path, "meta.json")) as f:
            info = json.load(f)
        d = {k: np.load(os.path.join(path, k + ".npy")) for k in ("z", "hist", "phase")}
        d.update(loaded=info["loaded"], dt=info["dt"])
        self.load_state_dict(d)
        return info

    def step(self, k: float):
        """One Newton solve to load factor k from the current one, the time step
        being (k - loaded) nominal steps; commits and returns the stats whether
        or not it converged (no cut-back)."""
        t0 = time.perf_counter()
        k = float(k)
        stats = self._solve_to(k, self.dt * (k - self.loaded))
        stats["step"] = k
        return self._commit(k, stats, t0)

    def advance(self, k: float, schedule=None):
        """Advance to load factor k with adaptive cut-back, or along the given
        sub-step ends `schedule` (a replay: every sub-step must converge).
        Returns the stats of the converged sub-steps; the last one holds the
        reaction at k."""
        k = float(k)
        out = []

        def attempt(f0, f1):
            t0 = time.perf_counter()
            z_prev = self.z.clone()
            hist_before = self.s.history(0).clone() if self.on_substep else None
            dt = self.dt * (f1 - f0)
            try:
                stats = self._solve_to(f1, dt)
            except pff.PffError as e:  # kernel status or no admissible line-search step
                if e.code != pff.ERR_DEVICE:
                    raise
                stats = {"converged": 0, "status": -1}
            if not (stats["converged"] == 1 and stats["status"] == 0):
                # the committed history is untouched until a sub-step converges
                self.z.copy_(z_prev)
                self.loaded = f0
                self.failures.append({"from": f0, "to": f1, **{k: v for k, v in stats.items() if k != "res_history"}})
                return False
            stats["step"] = k
            stats["dt"] = dt
            self._commit(f1, stats, t0)
            out.append(stats)
            if self.on_substep:
                self.on_substep(f0, f1, dt, hist_before, stats)
            return True

        if schedule is None:
            self.controller.run(self.loaded, k, attempt)
        else:
            for f1 in schedule:
                if not attempt(self.loaded, float(f1)):
                    raise StepFailed(f"replayed sub-step to {f1} did not converge")
            if self.loaded != k:
                raise StepFailed(f"schedule ends at {self.loaded}, not {k}")
        return out

    def close(self):
        if self.solver is not None:
            pff.pff_destroy_solver(self.solver)
            self.solver = None
        self.s.close()
