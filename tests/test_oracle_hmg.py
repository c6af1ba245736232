"""Pins of the oracle's geometric h-coarsening (structured order-1 grid):

* the prolongation is the coarse hat functions at the fine vertices: rows sum
  to one, the 1D matrix of one coarse element is [[1, 0], [1/2, 1/2], [0, 1]],
  and trilinear coarse functions are reproduced exactly at the fine vertices;
* for a homogeneous material at the undeformed state (constant tangent, the
  Q1 integrands exact with 2 Gauss points) the Galerkin operator P^T K_h P
  equals the operator assembled directly on the coarse grid;
* the coarse mask is the mask of the coincident fine vertices.
"""
import numpy as np

from paper_2607_21150_gb300 import inputs


def test_prolongation_partition_of_unity_and_entries(orc):
    P = orc.h_prolongation(2, 1, 1)
    n_f = 5 * 3 * 3
    n_c = 3 * 2 * 2
    assert P.shape == (4 * n_f, 4 * n_c)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=0, rtol=0)
    P1 = orc.h_prolongation(1, 1, 1)[:27, :8].toarray()
    one_d = np.array([[1.0, 0.0], [0.5, 0.5], [0.0, 1.0]])
    assert np.array_equal(P1, np.kron(one_d, np.kron(one_d, one_d)))


def test_prolongation_reproduces_trilinear_functions(orc):
    nx, ny, nz = 3, 2, 2
    P = orc.h_prolongation(nx, ny, nz)
    Xc = np.stack(np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij"), -1)
    Xf = np.stack(np.meshgrid(np.arange(2 * nx + 1), np.arange(2 * ny + 1), np.arange(2 * nz + 1),
                              indexing="ij"), -1) / 2.0

    def field(X, f):  # four trilinear fields, node order x fastest
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        vals = [1 + 2 * x - y + 0.5 * z, x * y * z, 3 * x * z - y, 0.25 + x * y]
        return np.transpose(vals[f], (2, 1, 0)).ravel()

    uc = np.concatenate([field(Xc, f) for f in range(4)])
    uf = np.concatenate([field(Xf, f) for f in range(4)])
    assert np.allclose(P @ uc, uf, rtol=0, atol=1e-14)


def test_galerkin_equals_rediscretisation(orc):
    L = (0.04, 0.04, 0.02)
    mf = inputs.Mesh(4, 4, 2, 1, 2, L)
    mc = inputs.Mesh(2, 2, 1, 1, 2, L)
    phases = inputs.phase_vector(inputs.EX3_MATRIX)[None]
    glob = inputs.glob_vector(2, 1e-3, 1e-2, 0.005, inputs.EX3_MATRIX["s_phi"][2])

    def K_of(m):
        w = inputs.Workload("h", m, phases, glob, np.zeros(m.nq, np.uint8), np.zeros((4, m.nn)),
                            inputs.zero_history(m.nq), None, None)
        return orc.assemble(w)["K"]

    Kf, Kc = K_of(mf), K_of(mc)
    P = orc.h_prolongation(2, 2, 1)
    G = (P.T @ Kf @ P).toarray()
    assert np.linalg.norm(G - Kc.toarray()) <= 1e-12 * np.linalg.norm(Kc.toarray())


def test_coarse_mask_takes_coincident_vertices(orc):
    m = inputs.Mesh(4, 2, 2, 1, 2, (0.04, 0.02, 0.02))
    mask, _ = inputs.dirichlet_tension(m, 1e-4)
    mc = orc.h_coarse_mask(mask, 2, 1, 1)
    assert mc.shape == (4, 3 * 2 * 2)
    full = mask.reshape(4, 3, 3, 5)
    for f in range(4):
        for K in range(2):
            for J in range(2):
                for I in range(3):
                    assert mc[f, I + 3 * (J + 2 * K)] == full[f, 2 * K, 2 * J, 2 * I]
