"""The seeded synthetic inputs (their recipe is part of the benchmark's
definition): determinism, the microstructure statistics the workloads are
specified by, agreement of the two phase rasterisers, the history generator's
invariants, the mapped-mesh coordinates, the coarse Dirichlet masks and the
explicit element map."""
import numpy as np
import pytest

from paper_2607_21150_gb300 import inputs as I


def test_spheres_seeded_and_on_target():
    a = I.place_spheres(0, 0.06, 0.02, 0.6)
    b = I.place_spheres(0, 0.06, 0.02, 0.6)
    assert np.array_equal(a.centers, b.centers) and np.array_equal(a.radii, b.radii)
    vol = (4.0 / 3.0 * np.pi * a.radii ** 3).sum()
    assert 0.6 <= vol <= 0.6 + 4.0 / 3.0 * np.pi * a.radii.max() ** 3   # stops at the target
    # lognormal radii with the requested mean and standard deviation (~500 samples)
    assert abs(a.radii.mean() / 0.06 - 1.0) < 0.05
    assert abs(a.radii.std() / 0.02 - 1.0) < 0.15
    assert np.all(a.centers >= 0.0) and np.all(a.centers < 1.0)
    assert a.max_overlap < 0.05
    c = I.place_spheres(1, 0.06, 0.02, 0.6)
    assert not np.array_equal(a.centers[:10], c.centers[:10])


def test_fast_phase_map_equals_point_test():
    sph = I.place_spheres(0, 0.06, 0.02, 0.6)
    m = I.Mesh(6, 5, 4, 2, 3, (0.06, 0.05, 0.04))
    scale = np.array([0.06] * 3)
    fast = I.phase_map_fast(m, sph, scale)
    slow = I.phase_map(I.qpoint_coords(m) / scale, sph)
    assert np.array_equal(fast, slow)
    assert 0.3 < fast.mean() < 0.9


def test_random_history_invariants():
    h = I.random_history(500, seed=2, c_amp=0.05, ep_max=0.01, H_max=3.0)
    for off in (0, 6):
        C = np.empty((500, 3, 3))
        C[:, 0, 0], C[:, 1, 1], C[:, 2, 2] = h[off], h[off + 1], h[off + 2]
        C[:, 1, 2] = C[:, 2, 1] = h[off + 3]
        C[:, 0, 2] = C[:, 2, 0] = h[off + 4]
        C[:, 0, 1] = C[:, 1, 0] = h[off + 5]
        assert np.allclose(np.linalg.det(C), 1.0, atol=1e-13)          # isochoric
        lam = np.linalg.eigvalsh(C)
        assert np.all(lam > 0) and np.abs(np.log(lam)).max() <= 0.05 + 1e-12
    assert h[12].min() >= 0 and h[12].max() <= 0.01
    assert h[13].min() >= 0 and h[13].max() <= 3.0
    assert np.array_equal(h, I.random_history(500, seed=2, c_amp=0.05, ep_max=0.01, H_max=3.0))
    z = I.zero_history(7, H0=0.5)
    assert np.all(z[0:3] == 1) and np.all(z[6:9] == 1) and np.all(z[13] == 0.5) and np.all(z[[3, 4, 5, 12, 14]] == 0)


def test_mapped_coords():
    m = I.Mesh(3, 2, 2, 2, 3, (0.3, 0.2, 0.2))
    X = I.node_coords(m)
    assert np.array_equal(I.mapped_coords(m, "affine", M=np.eye(3)), X.T)
    M = np.array([[1.1, 0.1, 0.0], [0.0, 0.9, 0.2], [0.05, 0.0, 1.0]])
    assert np.allclose(I.mapped_coords(m, "affine", M=M), M @ X.T)
    # straight-edged hexahedra: every element's GLL nodes are the trilinear map of its vertices,
    # so the middle node of each element edge is the mean of the edge's end vertices
    Y = I.mapped_coords(m, "vertices", amp=0.15, seed=3).T.reshape(m.nnz, m.nny, m.nnx, 3)
    assert np.allclose(Y[:, :, 1::2], 0.5 * (Y[:, :, 0:-1:2] + Y[:, :, 2::2]))
    assert np.allclose(Y[:, 1::2], 0.5 * (Y[:, 0:-1:2] + Y[:, 2::2]))
    assert np.abs(Y - X.reshape(m.nnz, m.nny, m.nnx, 3)).max() <= 0.15 * max(m.h) + 1e-15
    S = I.mapped_coords(m, "smooth", amp=0.2).T
    assert np.abs(S - X).max() <= 0.2 * max(m.h) + 1e-15 and np.abs(S - X).max() > 0


@pytest.mark.parametrize("pc", [1, 2])
def test_coarsen_mask_matches_coincident_nodes(pc):
    m = I.Mesh(2, 3, 2, 4, 5, (0.2, 0.3, 0.2))
    for mask, _ in (I.dirichlet_tension(m, 1e-3), I.dirichlet_compression(m, 1e-3)):
        mc = I.coarsen_mask(m, mask, pc).reshape(4, pc * m.nz + 1, pc * m.ny + 1, pc * m.nx + 1)
        mf = mask.reshape(4, m.nnz, m.nny, m.nnx)
        r = m.p // pc
        assert np.array_equal(mc, mf[:, ::r, ::r, ::r])


def test_element_offsets_structured_map():
    m = I.Mesh(3, 2, 2, 2, 3, (0.3, 0.2, 0.2))
    off = I.element_offsets(m)
    assert off.shape == (m.nel, 27) and off.dtype == np.int32
    counts = np.bincount(off.ravel(), minlength=m.nn)
    assert np.all(counts >= 1) and counts.max() == 8          # interior vertices shared by 8 elements
    X = I.node_coords(m)
    for e in (0, 5, m.nel - 1):
        pts = X[off[e]]
        assert np.allclose(pts.max(0) - pts.min(0), m.h)       # one element's box


def test_adjoint_parameter_vector_layout():
    """theta = (E_inf, nu_inf, sigma0, eta_d, Gc, l0) per phase: the slots name
    the Table 2 entries they claim, with_params inverts params_of, and the
    oracle's own copy of the layout agrees."""
    import oracle
    ph = np.stack([I.phase_vector(I.EX3_MATRIX), I.phase_vector(I.EX3_PARTICLE_ADJ)])
    th = I.params_of(ph)
    d = I.EX3_MATRIX
    assert list(th[:6]) == [d["E0"], d["nu0"], d["prandtl"][2], d["maxwell"][2], d["Gc"], d["l0"]]
    assert np.array_equal(I.with_params(ph, th), ph)
    th2 = th * np.arange(1, 13)
    assert np.array_equal(I.params_of(I.with_params(ph, th2)), th2)
    assert np.array_equal(oracle.get_params(ph), th)
    assert np.array_equal(oracle.set_params(ph, th2), I.with_params(ph, th2))


def test_twin_target_and_hardening_rows():
    th = np.arange(1.0, 13.0)
    a, b = I.twin_target(th), I.twin_target(th)
    assert np.array_equal(a, b) and not np.array_equal(a, th)
    f = a / th
    assert np.all(f > np.exp(-0.5)) and np.all(f < np.exp(0.5))      # lognormal, sigma 0.1
    ph = np.stack([I.phase_vector(I.EX3_MATRIX), I.phase_vector(I.EX3_PARTICLE)])
    hr = I.harden(ph, 2000.0, 800.0, 40.0)
    assert hr.shape == (2, 15) and np.array_equal(hr[:, :12], ph)
    assert list(hr[0, 12:]) == [2000.0, 800.0, 40.0]                  # the phase with a Prandtl branch
    assert list(hr[1, 12:]) == [0.0, ph[1, 11], 0.0]                  # perfect plasticity row otherwise
