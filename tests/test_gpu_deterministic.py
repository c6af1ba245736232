"""Deterministic transposed contractions (pff_op_set_deterministic): element
values plus one fixed-order sum per node instead of the atomic scatter-add.

Every quantity that goes through it stays at its parity bar against the
oracle (residual, FP64 / double-float / FP32 / BF16-word actions and
transposes, diagonal, p-level operators and the restriction) and two calls
give bitwise identical results; the host-buffer action equals the
device-buffer one bit for bit; a whole Newton solve (mixed p-multigrid, h-multigrid
coarse solve) repeated from the same start ends in the same bits."""
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


def _twice(fn):
    a = fn().clone()
    b = fn().clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    return tp.np_(a).astype(np.float64)


@pytest.mark.parametrize("name", ["box_q4_ragged", "box_q3_ragged", "box_q4_curved"])
def test_deterministic_operator(orc, name):
    w = tp.CASES[name]()
    ref = orc.assemble(w)
    s = Session(w, f32=True, df=True, bf16=True)
    pff.pff_op_set_deterministic(s.op, True)
    zt = torch.from_numpy(w.z.ravel()).cuda()
    r = _twice(lambda: s.residual(zt))
    assert tp.rel(r, ref["r"]) <= 1e-12
    v = inputs.random_vector(w.mesh.ndof, 4)
    v64 = torch.from_numpy(v).cuda()
    v32 = v64.float()
    K = ref["K"]
    for prec, x, bar in ((pff.PFF_F64, v64, 1e-12), (pff.PFF_DF64, v64, 1e-12), (pff.PFF_F32, v32, 2e-5),
                         (pff.PFF_F32_BF16, v32, 4e-3)):
        y = _twice(lambda: s.apply(x, prec=prec))
        yt = _twice(lambda: s.apply(x, prec=prec, transpose=True))
        assert tp.rel(y, K @ v) <= bar, prec
        assert tp.rel(yt, K.T @ v) <= bar, prec
    d = _twice(lambda: s.diag())
    assert tp.rel(d, K.diagonal()) <= 1e-12
    # host buffers, chunked: the same bits as the device-buffer action
    xh = v64.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    pff.pff_jacobian_apply_host(s.levels[w.mesh.p], pff.PFF_F64, xh, yh, 2)
    yd = s.apply(v64)
    torch.cuda.synchronize()
    assert torch.equal(yh, yd.cpu())
    s.close()


def test_deterministic_levels_and_restriction(orc):
    w = tp._two_phase(2, 3, 2, 4, 21)
    ref = orc.assemble(w)
    s = Session(w, levels=(2, 1))
    pff.pff_op_set_deterministic(s.op, True)
    s.residual(w.z)
    for pc in (2, 1):
        P = orc.prolongation(w.mesh, pc)
        mc = inputs.coarsen_mask(w.mesh, w.mask, pc)
        Pm = orc.masked_prolongation(P, w.mask, mc)
        Kc = orc.coarse_operator(ref["K"], Pm, mc)
        xc = torch.from_numpy(inputs.random_vector(Pm.shape[1], 21)).cuda()
        yc = _twice(lambda: s.apply(xc, p=pc))
        assert tp.rel(yc, Kc @ tp.np_(xc)) <= 1e-12
        rf = inputs.random_vector(Pm.shape[0], 22)
        rc = _twice(lambda: s.restrict(torch.from_numpy(rf).cuda(), pc, 4))
        assert tp.rel(rc, Pm.T @ rf) <= 1e-14
    s.close()


def test_deterministic_newton_solve_repeats_bitwise(orc):
    import test_gpu_solver as ts
    w = ts._box(4, 4, 4, 2, 33, state=False)   # a tension step from the unloaded state
    z0 = torch.from_numpy(w.z.ravel().copy()).cuda()
    s = Session(w, levels=(1,), f32=True, df=True)
    pff.pff_op_set_deterministic(s.op, True)
    solver = s.solver([2, 1], mixed=1, newton_rtol=1e-10, krylov_rtol=1e-6, outer_prec=pff.PFF_DF64)
    out = []
    for _ in range(2):
        z = z0.clone()
        st = pff.pff_newton_solve(solver, z)
        assert st["converged"] == 1
        out.append((z, st["krylov_iterations"]))
    torch.cuda.synchronize()
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])
    pff.pff_destroy_solver(solver)
    s.close()
