"""The Jacobian action on host buffers (pff_jacobian_apply_host: chunks of
element blocks, uploads and downloads of node layers on their own streams)
against the oracle, element by element.

A 6 x 5 x 12 Q2 box (360 elements, 13 blocks of 28) cut into 1 to 13 chunks
puts chunk boundaries in the middle of element layers, at layer boundaries and
between single blocks; every precision is held to its bar against the
oracle's K x (FP64 and double-float 1e-12, FP32 2e-5, BF16 words 4e-3).  At
full size (64^3 Q4, the bench's e2e call), sampled rows against the oracle at
1e-12 and the whole vector against the device-buffer action (same kernels,
only the scatter order of the atomics differs: 1e-14)."""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_21150_gb300 import pff  # noqa: E402
from paper_2607_21150_gb300.session import Session  # noqa: E402

import test_gpu_parity as tp  # noqa: E402

BARS = {pff.PFF_F64: (1e-12, 0.0), pff.PFF_DF64: (1e-12, 0.0), pff.PFF_F32: (2e-5, 0.0),
        pff.PFF_F32_BF16: (4e-3, 2e-5)}


@pytest.fixture(scope="module")
def box(orc):
    w = tp._two_phase(6, 5, 12, 2, 71)
    ref = orc.assemble(w)
    s = Session(w, f32=True, df=True, bf16=True)
    s.residual(w.z)
    torch.cuda.synchronize()
    yield w, ref, s
    s.close()


@pytest.mark.parametrize("nchunks", [1, 2, 5, 13])
@pytest.mark.parametrize("prec", [pff.PFF_F64, pff.PFF_DF64, pff.PFF_F32, pff.PFF_F32_BF16])
def test_apply_host_matches_oracle(box, nchunks, prec):
    w, ref, s = box
    v = inputs.random_vector(w.mesh.ndof, 9)
    dt = torch.float64 if prec in (pff.PFF_F64, pff.PFF_DF64) else torch.float32
    xh = torch.from_numpy(v).to(dt).pin_memory()
    yh = torch.full_like(xh, float("nan")).pin_memory()
    pff.pff_jacobian_apply_host(s.levels[w.mesh.p], prec, xh, yh, nchunks)
    torch.cuda.synchronize()
    hi, lo = BARS[prec]
    e = tp.rel(yh.double().numpy(), ref["K"] @ xh.double().numpy())
    assert lo <= e <= hi, (prec, nchunks, e)


def test_apply_host_full_size(orc):
    import bench
    w = bench.make_workload("compress_q4", seed=0)
    m = w.mesh
    s = Session(w, levels=(2, 1), f32=True, df=True)
    s.residual(w.z)
    x = inputs.random_vector(m.ndof, 8)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    pff.pff_jacobian_apply_host(s.levels[m.p], pff.PFF_F64, xh, yh, 8)
    yd = tp.np_(s.apply(torch.from_numpy(x).cuda()))
    torch.cuda.synchronize()
    s.close()
    y = yh.numpy()
    assert tp.rel(y, yd) <= 1e-14
    rng = np.random.default_rng(5)
    dofs = np.sort(rng.choice(m.ndof, 40, replace=False))
    dofs = np.concatenate([dofs, [0, m.ndof - 1, 3 * m.nn + m.nn // 2, 2 * m.nn + m.nn - 1]])
    ref = orc.sample_rows(w, dofs, x)
    assert tp.rel(y[dofs], ref["jx"]) <= 1e-12
