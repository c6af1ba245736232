"""Benchmark of the matrix-free phase-field fracture operator on GB300.

Default workload: the Q4 compression microstructure (64^3 elements, 67.9 M
DoF, particle volume fraction 0.7, lognormal radii mean 0.04 / sd 0.015,
frictionless platens, Example 2 parameters, AT2), synthetic seeded state.
One timed step = one FP64 Jacobian action y = J x over the whole mesh (the
hottest call of the Newton-Krylov solve), inputs resident in HBM; the FP32
level action (p-multigrid smoother precision) and the residual are timed
beside it.  value = whole-job FP64 apply throughput in GDoF/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config compress_q4|tension_q4]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Q4 Jacobian-apply GDoF/s & %HBM roofline; Newton step time FP64 vs mixed p-MG"
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x max SM clock
# DRAM bytes (read + write) per element of one Jacobian action, Q4 (P = Q = 5),
# from one ncu capture of the same kernels on the 24^3 tension workload
# (python bench.py --config tension_q4 --n 24 ...): FP64 220.06 + 5.48 MB over
# a 3 040-element launch, FP32 words 495.72 + 3.87 MB and BF16 words 265.13 +
# 3.72 MB over 13 824 elements; scaled to a launch by the element count.  None
# where the kernel has changed since its counters were taken.
TRAFFIC_PER_ELEMENT = {"f64": (220.06e6 + 5.48e6) / 3040, "f32": (495.72e6 + 3.87e6) / 13824,
                       "bf16": (265.13e6 + 3.72e6) / 13824}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def pipe_rates(stream, iters: int = 20000):
    """FP64 FMA, FP64 tensor-core (mma.sync m8n8k4) and FP32 FMA throughput of
    this GPU at its current clocks, and the rate of the FP64 <-> FP32
    conversion instructions (G conversions/s), by the library's pipe-rate
    probe: best of three launches of 8 blocks of 256 threads per SM, CUDA events."""
    import torch
    from paper_2607_21150_gb300 import pff
    out = {}
    blocks, threads = 152 * 8, 256
    sink = torch.zeros(blocks * threads, dtype=torch.float64, device="cuda")
    for name, kind, it in (("dfma", pff.PFF_PROBE_DFMA, iters), ("dmma", pff.PFF_PROBE_DMMA, iters // 4),
                           ("ffma", pff.PFF_PROBE_FFMA, 8 * iters), ("cvt", pff.PFF_PROBE_CVT, iters // 2)):
        pff.pff_probe_pipe(kind, 64, blocks, threads, sink, stream)
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl = pff.pff_probe_pipe(kind, it, blocks, threads, sink, stream)
            b.record(stream)
            torch.cuda.synchronize()
            best = max(best, fl / (a.elapsed_time(b) / 1e3) / 1e12)
        if name == "cvt":
            out["cvt_gops"] = best * 1e3
        else:
            out[name + "_tflops"] = best
    return out


def make_workload(name: str, seed: int = 0, n: int | None = None):
    from paper_2607_21150_gb300 import inputs
    w = getattr(inputs, name)() if n is None else getattr(inputs, name)(n=n)
    rng = np.random.default_rng(seed + 100)
    m = w.mesh
    h = min(m.h) / m.p
    w.z = np.zeros((4, m.nn))
    w.z[:3] = rng.uniform(-1e-3 * h, 1e-3 * h, (3, m.nn))
    w.z[3] = rng.uniform(0.0, 0.3, m.nn)
    mk = w.mask.astype(bool)
    w.z[mk] = w.dvals[mk]
    w.hist[13] = np.maximum(w.hist[13], rng.uniform(0.0, 2e-3, m.nq))
    return w


def apply_counts(P: int, Q: int):
    """Algorithmic FP64/FP32 flops of one element of the fused Jacobian action:
    per field 2 (P^3 Q + P^2 Q^2 + P Q^3) + 6 Q^4 MACs of sum-factorised basis work
    (collocated gradient), plus 103 MACs of the stored-tangent map per point."""
    basis = 4 * (2 * (P ** 3 * Q + P ** 2 * Q ** 2 + P * Q ** 3) + 6 * Q ** 4)
    point = 103 * Q ** 3
    return 2 * (basis + point)


class ClockSampler:
    def __init__(self, period_ms=200):
        self.samples = []
        self.proc = None
        self.period = period_ms

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 8 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 8 and s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            if len(s) > 8:
                for k, nm in enumerate(names):
                    if s[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample(name: str = "compress_q4", seconds_budget: float = 20.0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the
    Q4 workload `name`: a 4x4x4-element box of the same generator and state recipe.
    Times the CSR assembly (element matrices by full quadrature) once and the
    CSR SpMV (the oracle's Jacobian action) repeatedly."""
    import oracle
    from paper_2607_21150_gb300 import inputs
    oracle.build()
    n = 4
    w = getattr(inputs, name)(n=n)
    rng = np.random.default_rng(7)
    m = w.mesh
    h = min(m.h) / m.p
    w.z = np.zeros((4, m.nn))
    w.z[:3] = rng.uniform(-1e-3 * h, 1e-3 * h, (3, m.nn))
    w.z[3] = rng.uniform(0.0, 0.3, m.nn)
    mk = w.mask.astype(bool)
    w.z[mk] = w.dvals[mk]
    t0 = time.perf_counter()
    out = oracle.assemble(w)
    t_asm = time.perf_counter() - t0
    K = out["K"]
    x = inputs.random_vector(m.ndof, 1)
    y_ref = K @ x
    assert np.linalg.norm(oracle.spmv(K, x) - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.spmv(K, x)
        reps += 1
        if time.perf_counter() - t0 > min(5.0, seconds_budget):
            break
    t_spmv = (time.perf_counter() - t0) / reps
    threads = oracle.num_threads()
    oracle.set_num_threads(1)  # the same loop on one core
    reps1 = 0
    t0 = time.perf_counter()
    while True:
        oracle.spmv(K, x)
        reps1 += 1
        if time.perf_counter() - t0 > min(2.0, seconds_budget):
            break
    t_spmv1 = (time.perf_counter() - t0) / reps1
    oracle.set_num_threads(threads)
    t0 = time.perf_counter()
    oracle.assemble(w, matrix=False)
    t_res = time.perf_counter() - t0
    # one load step from the unloaded state by Newton with direct solves, on a
    # 2x2x2-element sub-box (the 4^3 one takes minutes in the sparse direct solver)
    wn = getattr(inputs, name)(n=2)
    mkn = wn.mask.astype(bool)
    wn.z = np.zeros((4, wn.mesh.nn))
    wn.z[mkn] = wn.dvals[mkn]
    t0 = time.perf_counter()
    _, hres, _ = oracle.newton(wn, rtol=1e-8)
    t_newton = time.perf_counter() - t0
    return dict(ndof=m.ndof, nel=m.nel, t_assemble=t_asm, t_spmv=t_spmv, t_residual=t_res, t_newton=t_newton,
                newton_iterations=len(hres) - 1, threads=threads,
                gdofs=m.ndof / t_spmv / 1e9, gdofs_1core=m.ndof / t_spmv1 / 1e9,
                gdofs_incl_assembly=m.ndof / (t_spmv + t_asm) / 1e9)


def newton_compare(name: str, steps: int = 1, variants=("mixed", "mixed_df", "fp64")):
    """Load steps from the unloaded state with FP64 p-MG, with mixed p-MG (FP32
    levels and smoothers) and with mixed p-MG whose outer FGMRES operator is the
    double-float action, all to ||r||/||r0|| <= 1e-8 with inner rtol 1e-3.
    Returns per-variant timings (host clock around synchronised phases) and the
    relative difference of each converged field from the FP64 one."""
    import torch
    from paper_2607_21150_gb300 import inputs
    from paper_2607_21150_gb300.driver import LoadStepper
    out = {"workload": name, "load_steps": steps}
    fields = {}
    for label, mixed, df, extra in (("mixed", True, False, {}), ("mixed_df", True, True, {}),
                                    ("mixed_bf16", True, True, {"level_words": 16}), ("fp64", False, False, {})):
        if label not in variants:
            continue
        w = getattr(inputs, name)()
        lsp = LoadStepper(w, mixed=mixed, df=df, verbose=1, **extra)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = kr = 0
        res = []
        tr = ts = tk = 0.0
        for k in range(1, steps + 1):
            st = lsp.step(k)
            its += st["newton_iterations"]
            kr += st["krylov_iterations"]
            tr += st["t_residual"]
            ts += st["t_setup"]
            tk += st["t_krylov"]
            res.append(st["res_history"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        fields[label] = lsp.z.cpu().numpy()
        out[label] = {"wall_s": wall, "newton_iterations": its, "krylov_iterations": kr,
                      "ms_per_newton_iteration": 1e3 * wall / max(its, 1), "t_residual_s": tr, "t_setup_s": ts,
                      "t_krylov_s": tk, "reaction": st["reaction"], "res_history": res[-1],
                      "levels": lsp.levels}
        print(json.dumps({"newton_variant": label, **out[label]}), file=sys.stderr, flush=True)
        lsp.close()
        del lsp
        torch.cuda.empty_cache()
    if "fp64" in fields:
        a = fields["fp64"]
        for label in ("mixed", "mixed_df", "mixed_bf16"):
            if label in fields:
                sfx = "" if label == "mixed" else label[len("mixed"):]
                out["field_rel_diff" + sfx] = float(np.linalg.norm(a - fields[label]) / np.linalg.norm(a))
                out[f"speedup_{label}_vs_fp64"] = out["fp64"]["wall_s"] / out[label]["wall_s"]
    return out


# load steps per Newton-comparison workload beyond the first: the 16^3 Q4
# tension test runs its 10 load steps; the 48^3 Q3 notched bar (36 M DoF) one
# step (its 40-step crack-propagation run is a separate, longer measurement).
NEWTON_STEPS = {"tension_q4": 10, "notched_q3": 1, "compress_q4": 1}


def apply_config(name: str, steps: int, warmup: int, mapped: str | None = None):
    """FP64 and FP32 fine-level action, and the residual, on another workload
    (CUDA events); `mapped` = a mapped-mesh kind of inputs.mapped_coords."""
    import torch
    from paper_2607_21150_gb300 import inputs, pff
    from paper_2607_21150_gb300.session import Session
    w = make_workload(name, seed=0)
    m = w.mesh
    if mapped:
        w.X = inputs.mapped_coords(m, mapped, amp=0.15)
    s = Session(w, f32=True)
    stream = torch.cuda.current_stream()
    zt = torch.from_numpy(w.z.ravel()).cuda()
    s.residual(zt)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    s.residual(zt)
    b.record(stream)
    torch.cuda.synchronize()
    t_res = a.elapsed_time(b)
    status = s.status()
    L = s.levels[m.p]
    x = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, m.ndof)).cuda()
    y = torch.empty_like(x)
    x32, y32 = x.float(), torch.empty(m.ndof, dtype=torch.float32, device="cuda")
    out = {"workload": f"{name}: Q{m.p} {m.nx}x{m.ny}x{m.nz} elements, {m.ndof} DoF"
                       + (f", mapped mesh ({mapped}, amplitude 0.15 h)" if mapped else ""),
           "residual_ms": t_res, "kernel_status": status}
    for label, fn in (("fp64", lambda: pff.pff_jacobian_apply(L, pff.PFF_F64, x, y, stream)),
                      ("fp32", lambda: pff.pff_jacobian_apply(L, pff.PFF_F32, x32, y32, stream))):
        for _ in range(warmup):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[f"{label}_ms"] = ms
        out[f"{label}_gdofs"] = m.ndof / (ms / 1e3) / 1e9
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def adjoint_timing(steps: int = 10, fd_check: bool = True):
    """Gradient of the reaction-curve misfit (twin-experiment target) for the
    adjoint workload: forward load steps with checkpoints, then the discrete
    adjoint backward; plus one central difference of the loss as a check."""
    import torch
    from paper_2607_21150_gb300 import inputs
    from paper_2607_21150_gb300.adjoint import ReactionCurveRunner
    w = inputs.adjoint_q2()
    theta0 = inputs.params_of(w.phases)
    runner = ReactionCurveRunner(w, steps, newton_rtol=1e-10, krylov_rtol=1e-6, adjoint_rtol=1e-9)
    target = runner.forward(inputs.twin_target(theta0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F = runner.forward(theta0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g = runner.backward(2.0 * (F - target))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"workload": f"adjoint_q2: Q2 {w.mesh.nx}^3 elements, {w.mesh.ndof} DoF, {steps} load steps, 12 parameters",
           "forward_s": t1 - t0, "backward_s": t2 - t1, "adjoint_krylov_iterations": int(sum(runner.adjoint_iters)),
           "sub_steps": int(sum(len(x) for x in runner.schedule)),
           "loss": float(np.sum((F - target) ** 2)), "grad": g.tolist()}
    if fd_check:
        i = 4  # matrix Gc
        h = 1e-5 * theta0[i]
        tp, tm = theta0.copy(), theta0.copy()
        tp[i] += h
        tm[i] -= h
        sch = runner.schedule  # the perturbed runs replay the sub-steps of the gradient's run
        fd = (np.sum((runner.forward(tp, sch) - target) ** 2) - np.sum((runner.forward(tm, sch) - target) ** 2)) / (2 * h)
        out["fd_check"] = {"param": "Gc matrix", "adjoint": float(g[i]), "central_difference": float(fd),
                           "rel_err": float(abs(g[i] - fd) / abs(fd))}
    runner.close()
    return out


def workload_label(name: str) -> str:
    """The config label the native arm prints for a workload (a Q4 box of the
    generator's default size), from its mesh alone."""
    import inspect
    from paper_2607_21150_gb300 import inputs
    n = inspect.signature(getattr(inputs, name)).parameters["n"].default
    m = inputs.Mesh(n, n, n, 4, 5, (1.0, 1.0, 1.0))
    return f"{name}: Q{m.p} {m.nx}x{m.ny}x{m.nz} elements, {m.ndof} DoF, {m.nq} quadrature points"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2607_21150_gb300 import inputs
    oracle.build()
    w = getattr(inputs, args.config)(n=4)   # bounded sample: 4^3 elements of the same generator
    m = w.mesh
    rng = np.random.default_rng(7)
    h = min(m.h) / m.p
    w.z = np.zeros((4, m.nn))
    w.z[:3] = rng.uniform(-1e-3 * h, 1e-3 * h, (3, m.nn))
    w.z[3] = rng.uniform(0.0, 0.3, m.nn)
    x = inputs.random_vector(m.ndof, 1)
    K = oracle.assemble(w)["K"]
    for _ in range(args.warmup):
        oracle.spmv(K, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv(K, x)
    dt = (time.perf_counter() - t0) / args.steps
    value = m.ndof / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(args.config), "parallelism": f"replicas x{args.gpus}",
                       "sample": f"4x4x4-element Q4 box of the same generator ({m.ndof} DoF)"},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"4x4x4-element Q4 box of the {args.config} generator ({m.ndof} DoF); "
                                       "CSR SpMV of the oracle's assembled Jacobian, GDoF/s of that box"},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def max_over_ranks(values, world: int):
    """Element-wise maximum of per-rank timings over all ranks: one all-reduce,
    on a CUDA tensor under NCCL and a CPU tensor under gloo."""
    vals = [float(v) for v in values]
    if world <= 1:
        return vals
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def whole_job_rate(world: int, units_per_rank: float, steps: int, t_ms: float) -> float:
    """Units of all ranks per second, in 1e9, for `steps` steps on every rank
    whose slowest rank took t_ms (weak scaling: every rank holds its own units)."""
    return world * units_per_rank * steps / (t_ms / 1e3) / 1e9


# --------------------------------------------------------------------------- GPU
def run_native(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_21150_gb300 import pff
    from paper_2607_21150_gb300.session import Session

    w = make_workload(args.config, seed=rank, n=args.n)
    m = w.mesh
    s = Session(w, levels=(2, 1) if m.p == 4 else (), f32=True, df=True, bf16=True)
    stream = torch.cuda.current_stream()
    z = torch.from_numpy(w.z.ravel()).cuda()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # residual (stores the linearisation used by every action), timed separately
    s.residual(z)
    torch.cuda.synchronize()
    t0.record(stream)
    r = s.residual(z)
    t1.record(stream)
    torch.cuda.synchronize()
    t_res = t0.elapsed_time(t1)
    # the residual alone, without the level copies of the words (FP32 / double-
    # float planes, BF16) that the mixed-precision solvers read; then restored
    pff.pff_op_enable_bf16(s.op, False)
    pff.pff_op_enable_f32(s.op, False)
    s.residual(z)
    torch.cuda.synchronize()
    t0.record(stream)
    s.residual(z)
    t1.record(stream)
    torch.cuda.synchronize()
    t_res64 = t0.elapsed_time(t1)
    pff.pff_op_enable_f32(s.op, True)
    pff.pff_op_enable_df(s.op, True)
    pff.pff_op_enable_bf16(s.op, True)
    r = s.residual(z)
    torch.cuda.synchronize()
    status = s.status()
    ndof = m.ndof
    L = s.levels[m.p]
    x64 = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, ndof)).cuda()
    y64 = torch.empty_like(x64)
    x32 = x64.float()
    y32 = torch.empty_like(x32)

    def apply64():
        pff.pff_jacobian_apply(L, pff.PFF_F64, x64, y64, stream)

    def apply32():
        pff.pff_jacobian_apply(L, pff.PFF_F32, x32, y32, stream)

    ydf = torch.empty_like(x64)

    def applydf():
        pff.pff_jacobian_apply(L, pff.PFF_DF64, x64, ydf, stream)

    launches = {}

    def timed(fn, K, W, label=None):
        """W untimed calls, then K calls bracketed by CUDA events on the launching
        stream (barrier and synchronize on both sides); also counts the
        library's kernel launches inside the timed calls."""
        for _ in range(W):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        n0 = pff.pff_kernel_launches()
        wall0 = time.perf_counter()
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - wall0
        if label:
            launches[label] = pff.pff_kernel_launches() - n0
        per = [a.elapsed_time(b) for a, b in evs]
        return sum(per), per, wall

    with ClockSampler() as clk:
        tot64, per64, wall64 = timed(apply64, args.steps, args.warmup, "fp64")
    with ClockSampler() as clk_probe:
        rates = pipe_rates(stream)
    tot32, per32, _ = timed(apply32, args.steps, args.warmup)
    totdf, _, _ = timed(applydf, args.steps, args.warmup)
    df_rel = float(torch.linalg.norm(ydf - y64) / torch.linalg.norm(y64))

    # end to end through the C ABI with host buffers: pff_jacobian_apply_host
    # uploads x from pinned host memory, applies and downloads y, the copies of
    # one chunk of node layers overlapping the computation of another
    xh = x64.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()

    def e2e_step():
        pff.pff_jacobian_apply_host(L, pff.PFF_F64, xh, yh, args.e2e_chunks, stream)

    tot_e2e, _, _ = timed(e2e_step, args.steps, 3, "e2e")
    apply64()
    torch.cuda.synchronize()
    e2e_rel = float(torch.linalg.norm(yh.cuda() - y64) / torch.linalg.norm(y64))

    # level action with BF16 stored words (FP32 vectors and arithmetic)
    y16 = torch.empty_like(x32)
    tot16, _, _ = timed(lambda: pff.pff_jacobian_apply(L, pff.PFF_F32_BF16, x32, y16, stream), args.steps,
                        args.warmup)
    bf16_rel = float(torch.linalg.norm(y16.double() - y64) / torch.linalg.norm(y64))

    # p-multigrid level actions on the same quadrature points (Galerkin levels)
    levels = {}
    for pl in sorted((p for p in s.levels if p != m.p), reverse=True):
        nl = 4 * s.nn(pl)
        Ll = s.levels[pl]
        xl = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, nl)).cuda()
        yl = torch.empty_like(xl)
        xl32, yl32 = xl.float(), torch.empty(nl, dtype=torch.float32, device="cuda")
        t64l, _, _ = timed(lambda: pff.pff_jacobian_apply(Ll, pff.PFF_F64, xl, yl, stream), args.steps, args.warmup)
        t32l, _, _ = timed(lambda: pff.pff_jacobian_apply(Ll, pff.PFF_F32, xl32, yl32, stream), args.steps,
                           args.warmup)
        t16l, _, _ = timed(lambda: pff.pff_jacobian_apply(Ll, pff.PFF_F32_BF16, xl32, yl32, stream), args.steps,
                           args.warmup)
        b32 = 4 * nl * 2 + nl + 67 * 4 * m.nq
        b16 = 4 * nl * 2 + nl + 67 * 2 * m.nq
        levels[f"Q{pl}"] = {"ndof": nl, "fp64_ms": t64l / args.steps, "fp32_ms": t32l / args.steps,
                            "bf16_words_ms": t16l / args.steps,
                            "fp64_gdofs": nl / (t64l / args.steps / 1e3) / 1e9,
                            "fp32_gdofs": nl / (t32l / args.steps / 1e3) / 1e9,
                            "fp32_hbm_frac": b32 / (t32l / args.steps / 1e3) / 1e9 / peaks()[0],
                            "bf16_words_hbm_frac": b16 / (t16l / args.steps / 1e3) / 1e9 / peaks()[0]}

    # every timed leg: the slowest rank's time
    tot64, tot32, totdf, tot_e2e = max_over_ranks([tot64, tot32, totdf, tot_e2e], world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    P, Q = m.p + 1, m.Q
    flops_el = apply_counts(P, Q)
    t_apply = tot64 / args.steps / 1e3
    value = whole_job_rate(world, ndof, args.steps, tot64)
    achieved_flops = flops_el * m.nel / t_apply / 1e12
    hbm_peak, src = peaks()
    bytes64 = 8 * ndof * 2 + ndof + 67 * 8 * m.nq
    bytes32 = 4 * ndof * 2 + ndof + 67 * 4 * m.nq
    bytes16 = 4 * ndof * 2 + ndof + 67 * 2 * m.nq
    t32 = tot32 / args.steps / 1e3
    q4 = (P, Q) == (5, 5)
    traffic64 = TRAFFIC_PER_ELEMENT["f64"] * m.nel if q4 else None
    traffic32 = TRAFFIC_PER_ELEMENT["f32"] * m.nel if q4 and TRAFFIC_PER_ELEMENT["f32"] else None
    traffic16 = TRAFFIC_PER_ELEMENT["bf16"] * m.nel if q4 and TRAFFIC_PER_ELEMENT["bf16"] else None
    s.close()
    del s
    torch.cuda.empty_cache()
    newton, newton_configs = None, {}
    for k, name in enumerate([] if args.newton == "none" else args.newton.split(",")):
        steps = args.newton_steps if k == 0 else NEWTON_STEPS.get(name, 1)
        res = newton_compare(name, steps, args.newton_variants.split(","))
        if k == 0:
            newton = res
        else:
            newton_configs[name] = res
    apply_small = apply_config("tension_q4", args.steps, args.warmup) if args.newton != "none" else None
    apply_mapped = (apply_config(args.config, args.steps, args.warmup, mapped="smooth")
                    if args.newton != "none" else None)
    adjoint = adjoint_timing(args.adjoint_steps) if args.adjoint_steps > 0 else None
    cpu = oracle_sample(args.config)
    line = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.config}: Q{m.p} {m.nx}x{m.ny}x{m.nz} elements, {ndof} DoF, "
                               f"{m.nq} quadrature points", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (stored linearisation %.1f GB)" % (67 * 8 * m.nq / 1e9),
                   "microstructure": w.meta},
        "roofline": {"bound": "alu", "achieved": achieved_flops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_flops / FP64_PEAK_TFLOPS, "traffic": traffic64,
                     "traffic_source": "ncu dram bytes per element at 24^3 Q4 x elements" if traffic64 else None,
                     "algorithmic_bytes": bytes64,
                     "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (derived from unit "
                                    "counts and the maximum clock; pipe_rates has the live probe)",
                     "pipe_rates": {**rates, "clocks": clk_probe.summary(),
                                    "frac_of_probe_dfma": achieved_flops / rates["dfma_tflops"]},
                     "hbm_frac": bytes64 / t_apply / 1e9 / hbm_peak, "hbm_peak_gbs": hbm_peak,
                     "hbm_peak_source": src},
        "fp32_level_apply": {"gdofs": ndof / t32 / 1e9, "ms": t32 * 1e3, "traffic": traffic32,
                             "algorithmic_bytes": bytes32,
                             "achieved_gbs": bytes32 / t32 / 1e9, "hbm_frac": bytes32 / t32 / 1e9 / hbm_peak,
                             "bound": "hbm", "peak_gbs": hbm_peak, "peak_source": src},
        "bf16_words_level_apply": {"gdofs": ndof / (tot16 / args.steps / 1e3) / 1e9, "ms": tot16 / args.steps,
                                   "algorithmic_bytes": bytes16, "traffic": traffic16, "achieved_gbs": bytes16 / (tot16 / args.steps / 1e3) / 1e9,
                                   "hbm_frac": bytes16 / (tot16 / args.steps / 1e3) / 1e9 / hbm_peak,
                                   "rel_l2_vs_fp64": bf16_rel,
                                   "note": "FP32 vectors and arithmetic, stored words as BF16 staged through shared "
                                           "memory by bulk copies (the p-multigrid level precision PFF_F32_BF16)"},
        "df64_apply": {"gdofs": ndof / (totdf / args.steps / 1e3) / 1e9, "ms": totdf / args.steps,
                       "rel_l2_vs_fp64": df_rel,
                       "note": "double-float action (FP32-pair arithmetic, FP64 vectors); not the headline"},
        "residual_ms": t_res, "residual_without_level_copies_ms": t_res64, "kernel_status": status,
        "newton_step": newton,
        "newton_configs": newton_configs,
        "level_applies": levels,
        "apply_tension_q4": apply_small,
        "apply_mapped_mesh": apply_mapped,
        "adjoint": adjoint,
        "e2e": {"value": whole_job_rate(world, ndof, args.steps, tot_e2e), "unit": "GDoF/s",
                "h2d_bytes_per_step": 8 * ndof, "d2h_bytes_per_step": 8 * ndof,
                "call": f"pff_jacobian_apply_host(PFF_F64, pinned x, pinned y, {args.e2e_chunks} chunks)",
                "rel_l2_vs_device_buffers": e2e_rel},
        "gpu_launches": launches["fp64"],
        "gpu_launches_note": "libpff kernels launched inside the timed FP64-action region (pff_kernel_launches "
                             "before and after it); per action: the y initialisation and the fused element kernel",
        "cpu_baseline": {"value": cpu["gdofs"], "unit": "GDoF/s", "cores": cpu["threads"], "kind": "oracle",
                         "sample": f"{cpu['nel']}-element Q4 sub-box ({cpu['ndof']} DoF) of the same workload; "
                                   f"CSR SpMV of the oracle's assembled Jacobian "
                                   f"(assembly {cpu['t_assemble']:.2f} s not included)",
                         "value_1core": cpu["gdofs_1core"],
                         "residual_s": cpu["t_residual"], "assembly_s": cpu["t_assemble"],
                         "newton_step_s_2x2x2": cpu["t_newton"], "newton_iterations": cpu["newton_iterations"]},
        "clocks": clk.summary(),
        "wall_s_timed": wall64,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="compress_q4", choices=["compress_q4", "tension_q4"])
    ap.add_argument("--n", type=int, default=None,
                    help="elements per direction of the --config workload (its default size if omitted; smaller "
                         "sizes serve ncu captures, the bench line is for the default)")
    ap.add_argument("--newton", default="compress_q4,tension_q4,notched_q3",
                    help="comma list of workloads (compress_q4, tension_q4, notched_q3) of the FP64-vs-mixed "
                         "Newton comparison, the first one reported as newton_step; or none")
    ap.add_argument("--newton-steps", type=int, default=1, help="load steps of the first --newton workload")
    ap.add_argument("--newton-variants", default="mixed,mixed_df,mixed_bf16,fp64",
                    help="comma list of mixed, mixed_df (double-float outer action), mixed_bf16 (double-float "
                         "outer action, BF16 level words), fp64")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="chunks of the end-to-end action through host buffers (pff_jacobian_apply_host)")
    ap.add_argument("--adjoint-steps", type=int, default=10, help="load steps of the adjoint timing (0 = skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
