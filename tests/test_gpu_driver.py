"""Load stepping and the reaction force on the GPU vs the oracle.

* pff_reaction = the oracle's internal force summed over the top-face u_z DoFs;
* three load steps of the tension box (Newton to 1e-11, history committed after
  every step; FP64 levels, or FP32 levels with the double-float outer action)
  reproduce the oracle's trajectory (Newton with direct solves, commit of its
  own trial history) to 1e-9 in the fields and the reactions.
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2607_21150_gb300 import pff  # noqa: E402
from paper_2607_21150_gb300.driver import LoadStepper  # noqa: E402
from paper_2607_21150_gb300.session import Session  # noqa: E402


def _tension_box(at=2):
    m = inputs.Mesh(2, 2, 3, 2, 3, (0.02, 0.02, 0.03))
    rng = np.random.default_rng(5)
    phases = np.stack([inputs.phase_vector(inputs.EX3_MATRIX), inputs.phase_vector(inputs.EX3_PARTICLE)])
    glob = inputs.glob_vector(at, 1e-3, 1e-2, 0.002 / 0.4, inputs.EX3_MATRIX["s_phi"][at])
    phase = (rng.random(m.nq) < 0.3).astype(np.uint8)
    mask, dv = inputs.dirichlet_tension(m, 0.002 * m.L[2])
    hist = inputs.zero_history(m.nq)
    if at == 1:
        for pid, d in ((0, inputs.EX3_MATRIX), (1, inputs.EX3_PARTICLE)):
            hist[13, phase == pid] = d["psi_c"]
    return inputs.Workload("tension", m, phases, glob, phase, np.zeros((4, m.nn)), hist, mask, dv)


def test_reaction_matches_oracle_internal_force(orc):
    w = _tension_box()
    rng = np.random.default_rng(2)
    w.z = inputs.random_state(w.mesh, 3, u_amp=1e-4, phi_max=0.2)
    s = Session(w)
    s.residual(torch.from_numpy(w.z.ravel()).cuda())
    top = inputs.top_face_mask(w.mesh)
    got = pff.pff_reaction(s.op, torch.from_numpy(top.ravel()).cuda())
    fint = orc.assemble(w, matrix=False, mask=None, dvals=None)["r"]
    ref = [float(fint[f][top[f].astype(bool)].sum()) for f in range(4)]
    assert abs(got[2] - ref[2]) <= 1e-12 * np.abs(fint).max() * top.sum()
    assert got[0] == 0.0 and got[3] == 0.0


@pytest.mark.parametrize("at,mixed", [(1, False), (2, False), (2, True)])
def test_load_steps_match_oracle(orc, at, mixed):
    """mixed: FP32 levels and the default double-float outer action."""
    w = _tension_box(at)
    lsp = LoadStepper(w, levels=[2, 1], mixed=mixed, newton_rtol=1e-11, krylov_rtol=1e-8)
    # oracle trajectory
    z = w.z.copy()
    hist = w.hist.copy()
    mk = w.mask.astype(bool)
    top = inputs.top_face_mask(w.mesh).astype(bool)
    for k in (1, 2, 3):
        wk = inputs.Workload("t", w.mesh, w.phases, w.glob, w.phase, z, hist, w.mask, w.dvals * k)
        z = z.copy()
        z[mk] = (w.dvals * k)[mk]
        wk.z = z
        z, hres, out = orc.newton(wk, rtol=1e-13)
        hist = out["hist_new"]
        fint = orc.assemble(inputs.Workload("t", w.mesh, w.phases, w.glob, w.phase, z, wk.hist, None, None),
                            matrix=False, mask=None, dvals=None)["r"]
        react = float(fint[2][top[2]].sum())
        st = lsp.step(k)
        assert st["converged"] == 1
        zg = lsp.z.cpu().numpy().reshape(4, -1)
        assert np.linalg.norm(zg - z) <= 1e-9 * np.linalg.norm(z)
        assert abs(st["reaction"] - react) <= 1e-8 * abs(react)
        hg = lsp.s.history(0).cpu().numpy()
        assert np.linalg.norm(hg - hist) <= 1e-9 * np.linalg.norm(hist)
    assert lsp.history[-1]["reaction"] > lsp.history[0]["reaction"] > 0
    lsp.close()


def test_substeps_match_oracle(orc):
    """Sub-steps (load factor and time step halved) against the oracle's Newton
    with the same time steps: 0 -> 0.5 -> 1 (dt/2 each), then 1 -> 2 (dt)."""
    w = _tension_box(2)
    lsp = LoadStepper(w, levels=[2, 1], mixed=False, newton_rtol=1e-11, krylov_rtol=1e-8)
    out = lsp.advance(1, schedule=[0.5, 1.0]) + lsp.advance(2, schedule=[2.0])
    assert [st["load"] for st in out] == [0.5, 1.0, 2.0]
    dt0 = float(w.glob[3])
    assert [st["dt"] for st in out] == [0.5 * dt0, 0.5 * dt0, dt0]
    z = w.z.copy()
    hist = w.hist.copy()
    mk = w.mask.astype(bool)
    top = inputs.top_face_mask(w.mesh).astype(bool)
    for st, (f, dt) in zip(out, ((0.5, 0.5 * dt0), (1.0, 0.5 * dt0), (2.0, dt0))):
        glob = w.glob.copy()
        glob[3] = dt
        z = z.copy()
        z[mk] = (w.dvals * f)[mk]
        wk = inputs.Workload("t", w.mesh, w.phases, glob, w.phase, z, hist, w.mask, w.dvals * f)
        z, _, res = orc.newton(wk, rtol=1e-13)
        fint = orc.assemble(inputs.Workload("t", w.mesh, w.phases, glob, w.phase, z, hist, None, None),
                            matrix=False, mask=None, dvals=None)["r"]
        hist = res["hist_new"]
        react = float(fint[2][top[2]].sum())
        assert abs(st["reaction"] - react) <= 1e-8 * abs(react)
    zg = lsp.z.cpu().numpy().reshape(4, -1)
    assert np.linalg.norm(zg - z) <= 1e-9 * np.linalg.norm(z)
    assert np.linalg.norm(lsp.s.history(0).cpu().numpy() - hist) <= 1e-9 * np.linalg.norm(hist)
    lsp.close()


def test_state_summary_and_checkpoint_resume(orc, tmp_path):
    """Per-step diagnostics and checkpoint/resume of the load stepper.

    The state summary's flag counts equal the counts of the oracle's flags at
    the converged state (up to points whose decision margin is below 1e-10);
    its extremes equal those of the state and history it summarises.  A
    stepper resumed from the checkpoint after step 1 reproduces step 2 of the
    uninterrupted run (fields and reaction to 1e-9, the trajectory tolerance:
    both runs stop Newton at 1e-11 and the atomic scatter orders sums
    differently from run to run)."""
    w = _tension_box(1)
    lsp = LoadStepper(w, levels=[2, 1], mixed=False, newton_rtol=1e-11, krylov_rtol=1e-8)
    lsp.diagnostics = True
    h0 = w.hist.copy()
    st1 = lsp.advance(1)[-1]
    z1 = lsp.z.cpu().numpy().reshape(4, -1)
    summ = st1["state"]
    ref = orc.assemble(w, z=z1, hist=h0, matrix=False)
    margins = ref["margins"]
    unsafe = int(np.sum(np.any(np.abs(margins) <= 1e-10, axis=1)))
    for bit, key in ((1, "n_yield"), (2, "n_active"), (4, "n_tension")):
        assert abs(summ[key] - np.count_nonzero(ref["flags"] & bit)) <= unsafe, key
    assert summ["phi_max"] == z1[3].max() and summ["phi_min"] == z1[3].min()
    assert summ["n_phi_above_0.9"] == np.count_nonzero(z1[3] > 0.9)
    hc = lsp.s.history(0).cpu().numpy()
    assert summ["eps_p_max"] == hc[12].max() and summ["H_max"] == hc[13].max()
    assert len(st1["lambda_max"]) == 2 and all(v > 0 for v in st1["lambda_max"])
    lsp.save_checkpoint(str(tmp_path / "ck"), {"step": 1})
    st2 = lsp.advance(2)[-1]
    z2 = lsp.z.cpu().numpy()
    lsp.close()
    lsp2 = LoadStepper(w, levels=[2, 1], mixed=False, newton_rtol=1e-11, krylov_rtol=1e-8)
    info = lsp2.load_checkpoint(str(tmp_path / "ck"))
    assert info["step"] == 1 and lsp2.loaded == 1.0
    st2b = lsp2.advance(2)[-1]
    z2b = lsp2.z.cpu().numpy()
    lsp2.close()
    assert np.linalg.norm(z2b - z2) <= 1e-9 * np.linalg.norm(z2)
    assert abs(st2b["reaction"] - st2["reaction"]) <= 1e-9 * abs(st2["reaction"])
