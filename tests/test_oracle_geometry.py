"""Pins of the oracle on mapped meshes (isoparametric geometry from nodal
coordinates, the general-geometry extension of Sec. 4's element maps):

* the box's own nodal coordinates reproduce the affine-box path;
* an affine map scales the quadrature weights by det M (total volume);
* patch test on straight-edged distorted hexahedra (trilinear element maps,
  integrands polynomial and integrated exactly): an affine displacement field
  gives a zero interior displacement residual;
* a rigid rotation of the mesh with the displacement field rotates the
  displacement residual and leaves the phase-field residual unchanged;
* on curved elements the assembled Jacobian equals central differences of the
  residual;
* cylinder and dogbone specimens built as mapped boxes keep w det J > 0 at
  every Gauss point, and their discrete volumes converge to the exact ones at
  high order.
"""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs


def _hooke_cube(nx=3, p=2):
    w = inputs.cube(nx=nx, p=p)
    w.phases = np.stack([inputs.phase_vector(dict(Gc=0.8, l0=0.005, E0=1000.0, nu0=0.3))])
    w.hist = inputs.zero_history(w.mesh.nq)
    return w


def test_box_coordinates_reproduce_the_box(orc):
    w = inputs.cube(nx=2, p=2, hist_seed=2, H_max=80.0)
    ref = orc.assemble(w)
    w.X = inputs.node_coords(w.mesh).T.copy()
    out = orc.assemble(w)
    assert np.linalg.norm(out["r"] - ref["r"]) <= 1e-13 * np.linalg.norm(ref["r"])
    assert abs(out["K"] - ref["K"]).max() <= 1e-13 * abs(ref["K"]).max()


def test_affine_map_scales_the_volume(orc):
    m = inputs.Mesh(3, 2, 2, 3, 4, (0.3, 0.2, 0.25))
    M = np.array([[1.1, 0.2, 0.0], [0.05, 0.9, 0.1], [0.0, -0.1, 1.2]])
    X = inputs.mapped_coords(m, "affine", M=M)
    _, wq = orc.qpoint_inputs(m, np.zeros((4, m.nn)), X)
    assert np.isclose(wq.sum(), np.linalg.det(M) * 0.3 * 0.2 * 0.25, rtol=1e-13)


def test_patch_test_distorted_hexahedra(orc):
    w = _hooke_cube(nx=3, p=2)
    m = w.mesh
    w.X = inputs.mapped_coords(m, "vertices", amp=0.15, seed=3)
    A = np.array([[2e-3, 1e-3, 0], [0, -1e-3, 5e-4], [3e-4, 0, 1.5e-3]])
    w.z = np.zeros((4, m.nn))
    w.z[:3] = A @ w.X
    w.z[3] = 0.2
    r = orc.assemble(w, matrix=False)["r"].reshape(4, m.nnz, m.nny, m.nnx)
    assert np.abs(r[:3, 1:-1, 1:-1, 1:-1]).max() <= 1e-12 * np.abs(r[:3]).max()


def test_rigid_rotation_of_the_mesh(orc):
    w = inputs.cube(nx=2, p=2, hist_seed=2, H_max=80.0)
    m = w.mesh
    w.X = inputs.mapped_coords(m, "smooth", amp=0.2)
    a = 0.7
    R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    R = R @ np.array([[1.0, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    ref = orc.assemble(w, matrix=False)
    wr = inputs.Workload("rot", m, w.phases, w.glob, w.phase, w.z.copy(), w.hist, None, None)
    wr.X = R @ w.X
    wr.z[:3] = R @ w.z[:3]
    # history: C_in^-1 is a reference-frame tensor; rotate it with the frame
    H = w.hist.copy()
    for off in (0, 6):
        C = np.zeros((3, 3, m.nq))
        for v, (i, j) in enumerate([(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]):
            C[i, j] = C[j, i] = w.hist[off + v]
        Cr = np.einsum("ia,abq,jb->ijq", R, C, R)
        for v, (i, j) in enumerate([(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]):
            H[off + v] = Cr[i, j]
    wr.hist = H
    out = orc.assemble(wr, matrix=False)
    r, rr = ref["r"], out["r"]
    assert np.linalg.norm(rr[:3] - R @ r[:3]) <= 1e-12 * np.linalg.norm(r[:3])
    assert np.linalg.norm(rr[3] - r[3]) <= 1e-12 * np.linalg.norm(r[3])


def test_fd_of_residual_on_curved_elements(orc):
    w = inputs.cube(nx=2, p=2, hist_seed=2, H_max=80.0)
    w.X = inputs.mapped_coords(w.mesh, "smooth", amp=0.2)
    out = orc.assemble(w, matrix=True)
    K = out["K"]
    v = inputs.random_vector(w.mesh.ndof, 1)
    eps = 1e-6 * np.linalg.norm(w.z) / np.linalg.norm(v)
    op = orc.assemble(w, z=w.z + eps * v.reshape(4, -1), matrix=False)
    om = orc.assemble(w, z=w.z - eps * v.reshape(4, -1), matrix=False)
    assert np.array_equal(op["flags"], out["flags"]) and np.array_equal(om["flags"], out["flags"])
    fd = (op["r"] - om["r"]).ravel() / (2 * eps)
    Kv = K @ v
    assert np.linalg.norm(Kv - fd) <= 1e-7 * np.linalg.norm(Kv)


@pytest.mark.parametrize("kind,p", [("cylinder", 2), ("cylinder", 4), ("dogbone", 2), ("dogbone", 4)])
def test_specimen_volumes_converge(orc, kind, p):
    """Cylinder (cross-sections mapped onto the inscribed disk) and dogbone
    (smooth neck) specimens as mapped boxes: every Gauss point keeps
    w det J > 0, and the discrete volume converges to the exact one
    (pi R^2 Lz; Lx Ly Lz (1 - a + 3 a^2 / 8)) at about order p + 2 in h."""
    L = (1.0, 1.0, 2.0)
    exact = np.pi * 0.25 * L[2] if kind == "cylinder" else L[0] * L[1] * L[2] * (1 - 0.3 + 3 * 0.09 / 8)
    errs = []
    for n in (2, 4):
        m = inputs.Mesh(n, n, n, p, p + 1, L)
        X = inputs.mapped_coords(m, kind, amp=0.3)
        _, wq = orc.qpoint_inputs(m, np.zeros((4, m.nn)), X)
        assert wq.min() > 0
        errs.append(abs(wq.sum() - exact) / exact)
    assert errs[1] < errs[0] / 2 ** (p + 1)
    assert errs[1] < (2e-4 if p == 2 else 1e-7)
