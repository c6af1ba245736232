"""The benchmark's multi-rank path on CPU (gloo, world size 2).

The hot path is replicated, not sharded: every rank runs the whole workload on
its own GPU, and only the timings meet.  These tests cover that host logic
without a GPU:

* `max_over_ranks` returns the element-wise maximum of the ranks' timings on
  every rank (one all-reduce over gloo);
* `whole_job_rate` counts the units of all ranks against the slowest rank;
* `bench.py --impl reference` under torchrun with two ranks prints exactly one
  JSON line (rank 0) and both ranks exit 0.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: timings (10 + r, 5 - r, 7)
        got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 7.0], world)
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [11.0, 5.0, 7.0]


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks([3, 4.5], 1) == [3.0, 4.5]


def test_whole_job_rate():
    import bench
    # 2 ranks x 1e9 units x 5 steps in 2.5 s of the slowest rank = 4 (1e9/s)
    assert bench.whole_job_rate(2, 1e9, 5, 2500.0) == pytest.approx(4.0)
    assert bench.whole_job_rate(1, 67898372, 10, 196.0) == pytest.approx(67898372 * 10 / 0.196 / 1e9)


def test_reference_arm_two_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_config_matches_the_native_label():
    """The reference arm reports the native arm's workload label (computed from
    the mesh alone) and samples a 4^3 box of the same generator."""
    import bench
    from paper_2607_21150_gb300 import inputs
    assert bench.workload_label("compress_q4") == \
        "compress_q4: Q4 64x64x64 elements, 67898372 DoF, 32768000 quadrature points"
    m = inputs.tension_q4().mesh
    assert bench.workload_label("tension_q4") == \
        f"tension_q4: Q{m.p} {m.nx}x{m.ny}x{m.nz} elements, {m.ndof} DoF, {m.nq} quadrature points"
