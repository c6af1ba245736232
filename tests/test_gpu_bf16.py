"""Level actions with BF16 stored words (PFF_F32_BF16) against the oracle.

Tolerance, from the arithmetic: every stored word is rounded to 8 significant
bits (relative error <= u = 2^-9, round to nearest even), and each output of
the action is a sum of products of such words with FP32 gradients.  The
rounding errors of different words are independent, so the relative L2 error
of the action is about u / sqrt(3) = 1.1e-3 (the FP32 arithmetic adds ~1e-6);
the bound is 4e-3 (two u).  The error must also exceed the FP32 level
(> 2e-5): the words really are 16-bit.  The level operators of the p-levels
are held to the same bound against the oracle's Galerkin product P^T K P,
and the Newton solution with BF16 words in every V-cycle level must still
equal the oracle's to 1e-9 (the preconditioner's precision does not change the
FP64 solution).
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

import test_gpu_parity as tp  # noqa: E402

BF16_TOL = 4e-3


def _check(y, ref, what):
    e = tp.rel(y, ref)
    assert 2e-5 < e <= BF16_TOL, (what, e)


@pytest.mark.parametrize("name", ["box_q4_ragged", "box_q3_ragged", "box_q1", "box_q4_curved", "box_q2_distorted",
                                  "box_q4_single"])
def test_bf16_apply_matches_oracle(orc, name):
    """Fine-level action and its transpose with BF16 words: ragged blocks, every
    Q, a single element, curved and distorted (mapped) meshes."""
    w = tp.CASES[name]()
    ref = orc.assemble(w)
    s = Session(w, f32=True, bf16=True)
    s.residual(w.z)
    v = inputs.random_vector(w.mesh.ndof, 4)
    v32 = torch.from_numpy(v.astype(np.float32)).cuda()
    y = tp.np_(s.apply(v32, prec=pff.PFF_F32_BF16)).astype(np.float64)
    yt = tp.np_(s.apply(v32, prec=pff.PFF_F32_BF16, transpose=True)).astype(np.float64)
    assert s.status() == 0
    _check(y, ref["K"] @ v, "apply")
    _check(yt, ref["K"].T @ v, "transpose")
    s.close()


@pytest.mark.parametrize("pf,levels", [(4, (2, 1)), (3, (1,))])
def test_bf16_level_operators(orc, pf, levels):
    """p-levels at the fine Gauss points with BF16 words = P^T K_f P."""
    w = tp._two_phase(2, 3, 2, pf, 17 + pf)
    ref = orc.assemble(w)
    s = Session(w, levels=levels, f32=True, bf16=True)
    s.residual(w.z)
    for pc in levels:
        P = orc.prolongation(w.mesh, pc)
        mc = inputs.coarsen_mask(w.mesh, w.mask, pc)
        Pm = orc.masked_prolongation(P, w.mask, mc)
        Kc = orc.coarse_operator(ref["K"], Pm, mc)
        xc = inputs.random_vector(Pm.shape[1], 21)
        x32 = torch.from_numpy(xc.astype(np.float32)).cuda()
        _check(tp.np_(s.apply(x32, p=pc, prec=pff.PFF_F32_BF16)), Kc @ xc, pc)
        _check(tp.np_(s.apply(x32, p=pc, prec=pff.PFF_F32_BF16, transpose=True)), Kc.T @ xc, pc)
    s.close()


def test_bf16_chebyshev_smoother(orc):
    """Chebyshev-Jacobi smoothing with the BF16-word action against the oracle's
    Chebyshev iteration on the assembled K and its diagonal (same interval and
    degree)."""
    w = tp._two_phase(3, 2, 2, 4, 61)
    ref = orc.assemble(w)
    s = Session(w, f32=True, bf16=True)
    s.residual(w.z)
    d = s.diag(prec=pff.PFF_F32)
    b = inputs.random_vector(w.mesh.ndof, 5)
    x0 = np.zeros(w.mesh.ndof)
    lmax = 2.0
    x = s.chebyshev(torch.from_numpy(b.astype(np.float32)).cuda(), torch.zeros(w.mesh.ndof, device="cuda"),
                    d, 3, 0.1 * lmax, 1.1 * lmax, prec=pff.PFF_F32_BF16)
    xr = orc.chebyshev(ref["K"], ref["K"].diagonal(), b, x0, 3, 0.1 * lmax, 1.1 * lmax)
    _check(tp.np_(x).astype(np.float64), xr, "chebyshev")
    s.close()


def test_full_size_bf16_sampled_rows(orc):
    """The 64^3 Q4 compression workload (67.9 M DoF) in the bench's launch
    configuration: the BF16-word action at sampled rows against the oracle's
    element rows (relative L2 over the rows; the bound allows for the
    fluctuation of a 44-row sample: 1e-2)."""
    import bench
    w = bench.make_workload("compress_q4", seed=0)
    m = w.mesh
    s = Session(w, levels=(2, 1), f32=True, df=True, bf16=True)
    s.residual(w.z)
    x = inputs.random_vector(m.ndof, 8)
    y = tp.np_(s.apply(torch.from_numpy(x.astype(np.float32)).cuda(), prec=pff.PFF_F32_BF16)).astype(np.float64)
    assert s.status() == 0
    s.close()
    rng = np.random.default_rng(5)
    dofs = np.sort(rng.choice(m.ndof, 40, replace=False))
    dofs = np.concatenate([dofs, [0, m.ndof - 1, 3 * m.nn + m.nn // 2, 2 * m.nn + m.nn - 1]])
    ref = orc.sample_rows(w, dofs, x)
    e = tp.rel(y[dofs], ref["jx"])
    assert 2e-5 < e <= 1e-2, e
