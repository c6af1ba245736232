"""Pin of the oracle's reaction force (`load_steps`), the quantity the adjoint's
loss is built from: a Hooke-only box in homogeneous uniaxial strain.

With u_x = u_y = 0 everywhere, phi = 0 everywhere (Dirichlet), u_z = 0 on the
bottom face and u_z = n delta on the top face, Newton finds the homogeneous
state F = diag(1, 1, lam), lam = 1 + n delta / L_z, exactly (patch test).  The
Hencky stress is then closed-form (Sec. 2, Eqs. hencky-tau): tau_33 = (4/3) mu
ln lam + kappa ln lam, with the Amor split of Sec. 3 degrading the whole stress
in tension (theta = ln lam >= 0) and the deviatoric part only in compression,
g = (1 - phi)^2 + eta = 1 + eta.  The first Piola stress is P_33 = tau_33 / lam
(P = tau F^-T), and the sum of the internal force over the top-face u_z DoFs
is P_33 L_x L_y: the top layer's basis functions sum to a function of z that is
1 on the top face and 0 at the bottom of its element layer, so the sum is the
integral of P_33 d/dz of it over the box.  A wrong face, component, sign,
degradation or missing F^-T fails this test."""
import numpy as np

from paper_2607_21150_gb300 import inputs


def _uniaxial_box(delta):
    L = (0.5, 0.75, 1.0)
    m = inputs.Mesh(2, 2, 2, 2, 3, L)
    row = inputs.phase_vector(dict(Gc=0.8, l0=0.05, E0=1000.0, nu0=0.3))   # Hooke only
    eta = 1e-3
    glob = inputs.glob_vector(2, eta, 1e-2, 0.01, 1.0)
    mask = np.zeros((4, m.nnz, m.nny, m.nnx), dtype=np.uint8)
    vals = np.zeros((4, m.nnz, m.nny, m.nnx))
    mask[0:2] = 1          # u_x = u_y = 0 everywhere
    mask[3] = 1            # phi = 0 everywhere
    mask[2, 0] = 1         # bottom u_z = 0
    mask[2, -1] = 1        # top u_z = n delta at step n
    vals[2, -1] = delta
    w = inputs.Workload("uniaxial", m, row[None], glob, np.zeros(m.nq, np.uint8), np.zeros((4, m.nn)),
                        inputs.zero_history(m.nq), mask.reshape(4, -1), vals.reshape(4, -1))
    return w, row, eta


def _closed_form(row, eta, lam, area):
    E, nu = row[2], row[3]
    mu, kap = E / (2 * (1 + nu)), E / (3 * (1 - 2 * nu))
    g = 1.0 + eta
    t_d, t_v = 4.0 / 3.0 * mu * np.log(lam), kap * np.log(lam)
    tau33 = g * (t_d + t_v) if lam >= 1.0 else g * t_d + t_v
    return tau33 / lam * area


def test_reaction_of_homogeneous_uniaxial_strain(orc):
    for delta in (0.02, -0.02):   # tension, then compression
        w, row, eta = _uniaxial_box(delta)
        top = inputs.top_face_mask(w.mesh)
        F, zs, _ = orc.load_steps(w, orc.get_params(w.phases), 3, top)
        Lx, Ly, Lz = w.mesh.L
        for n in range(1, 4):
            lam = 1.0 + n * delta / Lz
            # the state is the homogeneous one
            assert np.allclose(zs[n - 1][2], (lam - 1.0) * inputs.node_coords(w.mesh)[:, 2], rtol=0, atol=1e-13)
            want = _closed_form(row, eta, lam, Lx * Ly)
            assert abs(F[n - 1] - want) <= 1e-11 * abs(want), (delta, n, F[n - 1], want)
