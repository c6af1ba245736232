"""Load-stepping simulation of a workload: python -m paper_2607_21150_gb300.simulate
--workload notched_q3 --steps 40 [--fp64] [--max-cuts 6] [--verbose]
[--param NAME=VALUE ...] [--checkpoint DIR] [--resume DIR]
(NAME a field of pff_solver_params, e.g. cheb_degree, cheb_lo, krylov_rtol,
eig_every, coarse_maxit, level_words).

Runs LoadStepper.advance for load steps 1..steps (adaptive cut-back) and prints
one JSON line per load step: reaction on the loaded face, sub-steps, Newton,
FGMRES and coarse iterations, wall time, the state after the step (points
yielded / history-active, largest and smallest phase field, nodes with
phi > 0.9, largest plastic strain and history field) and the lambda_max
estimates of the multigrid levels; then a summary line.  --checkpoint DIR
saves the state after every completed load step (overwriting), --resume DIR
continues from such a checkpoint with the next load step."""
from __future__ import annotations

import argparse
import json
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="notched_q3",
                    choices=["notched_q3", "tension_q4", "compress_q4", "adjoint_q2"])
    ap.add_argument("--n", type=int, default=None, help="elements per direction (workload default if omitted)")
    ap.add_argument("--steps", type=int, default=None, help="load steps (workload default if omitted)")
    ap.add_argument("--fp64", action="store_true", help="FP64 multigrid levels instead of FP32")
    ap.add_argument("--max-cuts", type=int, default=6)
    ap.add_argument("--grow-after", type=int, default=2,
                    help="converged sub-steps in a row before a cut load increment doubles again")
    ap.add_argument("--verbose", action="store_true", help="the solver's per-iteration log on stderr")
    ap.add_argument("--param", action="append", default=[], metavar="NAME=VALUE",
                    help="solver parameter, a field of pff_solver_params (repeatable)")
    ap.add_argument("--checkpoint", default=None, metavar="DIR",
                    help="save the state to DIR after every completed load step")
    ap.add_argument("--resume", default=None, metavar="DIR", help="continue from the checkpoint in DIR")
    args = ap.parse_args(argv)
    import ctypes

    import torch
    from . import inputs, pff
    from .driver import LoadStepper, StepFailed
    fields = dict(pff.pff_solver_params._fields_)
    params = {}
    for kv in args.param:
        name, _, val = kv.partition("=")
        if name not in fields or not val:
            ap.error(f"--param {kv}: expected NAME=VALUE with NAME one of {', '.join(fields)}")
        params[name] = int(val) if fields[name] is ctypes.c_int else float(val)
    if args.verbose:
        params["verbose"] = 1
    make = getattr(inputs, args.workload)
    w = make() if args.n is None else make(n=args.n)
    steps = args.steps or int(w.meta.get("steps", 10))
    t0 = time.perf_counter()
    lsp = LoadStepper(w, mixed=not args.fp64, max_cuts=args.max_cuts, grow_after=args.grow_after, **params)
    lsp.diagnostics = True
    first = 1
    if args.resume:
        info = lsp.load_checkpoint(args.resume)
        first = int(round(info["loaded"])) + 1
    print(json.dumps({"workload": args.workload, "ndof": w.mesh.ndof, "nq": w.mesh.nq, "steps": steps,
                      "mixed": not args.fp64, "solver_params": params, "first_step": first,
                      "setup_s": time.perf_counter() - t0}), flush=True)
    t_all = time.perf_counter()
    status = "completed"
    for k in range(first, steps + 1):
        t1 = time.perf_counter()
        nf = len(lsp.failures)
        try:
            out = lsp.advance(k)
        except StepFailed as e:
            status = f"stopped at step {k}: {e}"
            break
        torch.cuda.synchronize()
        print(json.dumps({"step": k, "reaction": out[-1]["reaction"], "sub_steps": len(out),
                          "newton_iterations": sum(st["newton_iterations"] for st in out),
                          "krylov_iterations": sum(st["krylov_iterations"] for st in out),
                          "coarse_iterations": sum(st.get("coarse_iterations", 0) for st in out),
                          "line_search_cuts": sum(st.get("line_search_cuts", 0) for st in out),
                          "newton_res": out[-1].get("res_history"),
                          "failed_sub_steps": len(lsp.failures) - nf,
                          "state": out[-1].get("state"), "lambda_max": out[-1].get("lambda_max"),
                          "wall_s": time.perf_counter() - t1}), flush=True)
        if args.checkpoint:
            lsp.save_checkpoint(args.checkpoint, {"workload": args.workload, "step": k})
    print(json.dumps({"status": status, "wall_s": time.perf_counter() - t_all,
                      "attempts": len(lsp.history)}), flush=True)
    lsp.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
