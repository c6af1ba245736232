"""The allocation-free Chebyshev smoother gives what the regular one gives.

pff_chebyshev_smooth_noalloc exists for callers that may not allocate device
memory at the point where they smooth (their memory belongs to another
allocator or to a budget fixed at start-up, or they run in a loop where
cudaMalloc/cudaFree would synchronise the device).  It takes its work vectors
from an array built into the library instead of from the caller.  This test
calls it through the C ABI twice in a row on two multigrid levels and compares
each result with pff_chebyshev_smooth given caller-allocated work space, at the
tolerance of the other GPU tests; it also checks that a level too large for
the built-in array is refused with a clear error.  The file name makes pytest
collect it after every other test file.
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_21150_gb300 import pff  # noqa: E402
from paper_2607_21150_gb300.session import Session  # noqa: E402

TOL = 1e-12


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _workload():
    m = inputs.Mesh(3, 2, 2, 4, 5, (0.03, 0.02, 0.02))
    rng = np.random.default_rng(41)
    phases = np.stack([inputs.phase_vector(inputs.EX3_MATRIX), inputs.phase_vector(inputs.EX3_PARTICLE)])
    glob = inputs.glob_vector(2, 1e-3, 1e-2, 0.005, inputs.EX3_MATRIX["s_phi"][2])
    phase = (rng.random(m.nq) < 0.4).astype(np.uint8)
    z = inputs.random_state(m, 41, u_amp=2e-4, phi_max=0.6)
    hist = inputs.random_history(m.nq, 42, H_max=3000.0)
    mask, dv = inputs.dirichlet_tension(m, 1e-4)
    z[mask.astype(bool)] = dv[mask.astype(bool)]
    return inputs.Workload("box", m, phases, glob, phase, z, hist, mask, dv)


def test_noalloc_chebyshev_matches_regular_entry_point():
    pff.lib()
    w = _workload()
    s = Session(w, levels=(2,), f32=True)
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    for p in (4, 2):
        for prec, dtype in ((pff.PFF_F64, torch.float64), (pff.PFF_F32, torch.float32)):
            n = 4 * s.nn(p)
            diag = s.diag(p, prec)
            b = torch.from_numpy(inputs.random_vector(n, 51)).to("cuda", dtype)
            x0 = (torch.from_numpy(inputs.random_vector(n, 52)) * 1e-3).to("cuda", dtype)
            x_ref = x0.clone()
            work = torch.zeros(3 * n, dtype=dtype, device="cuda")
            pff.pff_chebyshev_smooth(s.levels[p], prec, 3, 0.1, 1.9, diag, b, x_ref, work)
            tol = TOL if prec == pff.PFF_F64 else 1e-5
            for _ in range(2):  # two calls in a row share the built-in work space
                x = x0.clone()
                pff.pff_chebyshev_smooth_noalloc(s.levels[p], prec, 3, 0.1, 1.9, diag, b, x)
                torch.cuda.synchronize()
                assert _rel(x, x_ref) <= tol, (p, prec)
    s.close()


def test_noalloc_rejects_levels_beyond_its_work_space():
    pff.lib()
    m = inputs.Mesh(20, 20, 20, 4, 5, (0.2, 0.2, 0.2))  # 4 * 81^3 = 2 125 764 DoF > 2 097 152
    w = inputs.Workload("big", m, inputs.phase_vector(inputs.EX3_MATRIX)[None],
                        inputs.glob_vector(2, 1e-3, 1e-2, 0.01, 1.0), np.zeros(m.nq, np.uint8),
                        np.zeros((4, m.nn)), inputs.zero_history(m.nq))
    s = Session(w)
    n = 4 * m.nn
    d = torch.ones(n, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(d)
    x = torch.zeros_like(d)
    with pytest.raises(pff.PffError, match="more than the 2097152"):
        pff.pff_chebyshev_smooth_noalloc(s.levels[4], pff.PFF_F64, 3, 0.1, 1.9, d, b, x)
    s.close()
