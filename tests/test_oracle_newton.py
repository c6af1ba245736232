"""Pin of the oracle's consistent tangent by Newton's convergence rate (the
quadratic stage I of the paper's Newton iterations, Table 3): from the linear
predictor of a uniaxial tension step on the unit cube, Newton with direct
solves reaches ||r|| <= 1e-13 ||r_0|| within 8 iterations, and once the
residual is small every step squares it, e_{k+1} <= C e_k^2 with e = ||r|| /
||r_0||.  A tangent with a wrong or missing term converges linearly and fails
the bound.  Cases: a Hooke-only phase at 3 % strain, and the Example 3 matrix
(Hooke, Maxwell and Prandtl branches) at 1 %.
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs


def _tension_cube(delta, hooke_only):
    w = inputs.cube(nx=2, p=2)
    if hooke_only:
        w.phases = np.stack([inputs.phase_vector(dict(Gc=0.8, l0=0.05, E0=1000.0, nu0=0.3))])
    w.hist = inputs.zero_history(w.mesh.nq)
    w.mask, w.dvals = inputs.dirichlet_tension(w.mesh, delta)
    m = w.mesh
    X = inputs.node_coords(m)
    z = np.zeros((4, m.nn))
    z[2] = delta * X[:, 2] / m.L[2]   # linear predictor, exact on the Dirichlet faces
    w.z = z
    return w


@pytest.mark.parametrize("delta,hooke_only", [(0.03, True), (0.01, False)])
def test_newton_converges_quadratically(orc, delta, hooke_only):
    w = _tension_cube(delta, hooke_only)
    _, hist, _ = orc.newton(w, rtol=1e-15, maxit=12)
    e = np.array(hist) / hist[0]
    assert np.all(np.isfinite(e))
    k_end = int(np.argmax(e <= 1e-13))
    assert e[k_end] <= 1e-13 and k_end <= 8, e
    # steps from a small residual to one still above the rounding level
    pairs = [(e[k], e[k + 1]) for k in range(len(e) - 1) if e[k] <= 1e-2 and e[k + 1] >= 1e-14]
    assert pairs, e
    for a, b in pairs:
        assert b <= 10.0 * a * a, (a, b, e)
