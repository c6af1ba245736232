"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds NO arithmetic of the method: it only draws random numbers,
lays out a structured box mesh, places particles and writes parameter tables.
Everything it returns is plain numpy data that both sides consume.

Workloads (units mm, MPa, s):

* ``cube``     -- unit cube, 4^3 Q2 elements, homogeneous matrix material
                  (Hooke + Maxwell + perfectly plastic Prandtl, Table 2,
                  Example 3 column), AT2, random nodal fields, zero history.
* ``cube_b``   -- the same mesh with a seeded random committed history so that
                  both yield states and both history states occur.
* ``tension_q4``   -- Q4, 16^3 elements, two-phase particle/matrix
                  microstructure (spheres, lognormal radii, volume fraction
                  0.6), uniaxial tension, AT1, Example 3 parameters.
* ``notched_q3``   -- Q3, 48x48x144 elements, notched bar (aspect 1:1:3).
* ``adjoint_q2``   -- Q2, 24^3 elements, tension, AT2.
* ``compress_q4``  -- Q4, 64^3 elements (~67.9 M DoF), volume fraction 0.7,
                  uniaxial compression with frictionless platens, AT2,
                  Example 2 parameters.

The paper's own microstructures (microstructpy seed lists, Gmsh meshes) are not
available; these generators stand in for them with the same statistics.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Material parameters (Table 2), converted to mm / MPa / s.
# Phase parameter vector layout (12 doubles):
#   Gc, l0, E_inf, nu_inf, hasMaxwell, E1, nu1, eta_d, hasPrandtl, E2, nu2, sigma0
# Global parameter vector (5 doubles): AT (1|2), eta (residual stiffness),
#   zeta (damage viscosity), dt, s_phi.
# ---------------------------------------------------------------------------
GPA = 1.0e3  # MPa per GPa

# Two constants of each workload are derived from these parameters by the
# method: the phase-field residual scale s_phi = E_inf c0 / (2 l0 Gc) of the
# matrix phase (Eq. damage-residual-scaling; c0 = 8/3 for AT1, 2 for AT2) and
# the AT1 threshold psi_c = 3 Gc / (16 l0) of every phase (Sec. 3.1), from
# which AT1 runs start their crack-driving history.  They are stored here as
# explicit numbers, worked out by hand from Table 2 (the arithmetic is printed
# beside each), so that this module computes neither formula; the oracle
# derives both itself and the tests pin the two against each other.
EX3_PARTICLE = dict(Gc=8.0, l0=0.005, E0=400 * GPA, nu0=0.25,
                    psi_c=300.0)                       # 3 * 8 / (16 * 0.005)
EX3_MATRIX = dict(Gc=0.8, l0=0.005, E0=1.0 * GPA, nu0=0.3,
                  maxwell=(1.0 * GPA, 0.3, 0.01 * GPA),
                  prandtl=(198 * GPA, 0.30, 500.0),
                  psi_c=30.0,                          # 3 * 0.8 / (16 * 0.005)
                  s_phi={1: 333333.3333333333,          # 1000 * (8/3) / (2 * 0.005 * 0.8)
                         2: 250000.0})                 # 1000 * 2 / (2 * 0.005 * 0.8)
EX2_PARTICLE = dict(Gc=0.1, l0=0.01, E0=10 * GPA, nu0=0.3,
                    psi_c=1.875)                       # 3 * 0.1 / (16 * 0.01)
# Adjoint workload: the Example 3 particle phase with a Maxwell (eta_d = 1 GPa s)
# and a perfectly plastic Prandtl branch (sigma0 = 5 GPa, E2 = E_inf) so that
# none of the twelve parameter gradients is structurally zero.
EX3_PARTICLE_ADJ = dict(Gc=8.0, l0=0.005, E0=400 * GPA, nu0=0.25,
                        maxwell=(400 * GPA, 0.25, 1.0 * GPA),
                        prandtl=(400 * GPA, 0.25, 5000.0),
                        psi_c=300.0)                   # 3 * 8 / (16 * 0.005)
EX2_MATRIX = dict(Gc=0.01, l0=0.01, E0=1.0 * GPA, nu0=0.4,
                  maxwell=(1.0 * GPA, 0.4, 0.1 * GPA),
                  psi_c=0.1875,                        # 3 * 0.01 / (16 * 0.01)
                  s_phi={1: 13333333.333333334,         # 1000 * (8/3) / (2 * 0.01 * 0.01)
                         2: 10000000.0})               # 1000 * 2 / (2 * 0.01 * 0.01)


def phase_vector(d: dict) -> np.ndarray:
    """Pack one phase's parameters into the 12-double layout above."""
    v = np.zeros(12)
    v[0], v[1], v[2], v[3] = d["Gc"], d["l0"], d["E0"], d["nu0"]
    if "maxwell" in d:
        v[4] = 1.0
        v[5], v[6], v[7] = d["maxwell"]
    if "prandtl" in d:
        v[8] = 1.0
        v[9], v[10], v[11] = d["prandtl"]
    return v


def harden(phases, H_lin: float, sigma_inf: float, beta: float) -> np.ndarray:
    """Phase rows widened to 15 doubles with the linear + Voce hardening law of
    the Prandtl branch (Eq. plasticity-strain-hardening-law): H_lin, sigma_inf,
    beta for every phase that has a Prandtl branch, (0, sigma0, 0) = perfect
    plasticity for the others.  The paper's examples are perfectly plastic; the
    values used with this are test inputs, not Table 2 data."""
    ph = np.atleast_2d(np.asarray(phases, dtype=np.float64))
    out = np.zeros((ph.shape[0], 15))
    out[:, :12] = ph[:, :12]
    out[:, 13] = ph[:, 11]
    for k in range(ph.shape[0]):
        if ph[k, 8]:
            out[k, 12:15] = (H_lin, sigma_inf, beta)
    return out


def glob_vector(at: int, eta: float, zeta: float, dt: float, s_phi: float) -> np.ndarray:
    return np.array([float(at), eta, zeta, dt, s_phi])


# ---------------------------------------------------------------------------
# Structured box mesh
# ---------------------------------------------------------------------------
@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    p: int
    Q: int
    L: tuple  # side lengths (Lx, Ly, Lz)

    @property
    def h(self):
        return (self.L[0] / self.nx, self.L[1] / self.ny, self.L[2] / self.nz)

    @property
    def dims(self):
        return np.array([self.nx, self.ny, self.nz, self.p, self.Q], dtype=np.int32)

    @property
    def nnx(self):
        return self.p * self.nx + 1

    @property
    def nny(self):
        return self.p * self.ny + 1

    @property
    def nnz(self):
        return self.p * self.nz + 1

    @property
    def nn(self):
        return self.nnx * self.nny * self.nnz

    @property
    def nel(self):
        return self.nx * self.ny * self.nz

    @property
    def nq(self):
        return self.nel * self.Q ** 3

    @property
    def ndof(self):
        return 4 * self.nn


def gll_points(p: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre points on [-1, 1] (numpy's Legendre roots)."""
    if p == 1:
        return np.array([-1.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def gauss_points(Q: int) -> np.ndarray:
    return np.polynomial.legendre.leggauss(Q)[0]


def node_coords(m: Mesh) -> np.ndarray:
    """Reference coordinates of every node, shape [nn, 3] (node id = I + nnx (J + nny K))."""
    xs = []
    g = gll_points(m.p)
    for d, (n, Ld) in enumerate(zip((m.nx, m.ny, m.nz), m.L)):
        h = Ld / n
        pts = np.empty(m.p * n + 1)
        for e in range(n):
            pts[m.p * e: m.p * e + m.p + 1] = e * h + (g + 1.0) * 0.5 * h
        xs.append(pts)
    X, Y, Z = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
    # node id = I + nnx*(J + nny*K): flatten with K slowest, I fastest
    return np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                     Z.transpose(2, 1, 0).ravel()], axis=1)


def mapped_coords(m: Mesh, kind: str = "smooth", amp: float = 0.1, seed: int = 0, M=None) -> np.ndarray:
    """Nodal coordinates [3][nn] of a mapped mesh on the box of ``m``:

    * ``affine``: X' = M X (M given, det M > 0);
    * ``vertices``: every element vertex moved by U[-amp, amp] h per direction
      (seeded), the element's GLL nodes placed by trilinear interpolation of
      its eight vertices (straight-edged hexahedra, conforming faces);
    * ``smooth``: X'_d = X_d + amp h_d sin(2 pi X_{d+1} / L_{d+1}) sin(pi X_{d+2} / L_{d+2}),
      evaluated at every node (curved elements);
    * ``cylinder``: every cross-section square mapped onto its inscribed disk
      (radius min(Lx, Ly) / 2) by the elliptical grid map
      x' = u sqrt(1 - v^2 / 2), y' = v sqrt(1 - u^2 / 2) of u, v in [-1, 1]
      (a single patch: the corner angles open to 180 degrees, so the Jacobian
      vanishes at the four corner lines and only Gauss points see it positive);
    * ``dogbone``: the cross-section scaled about its centre by
      s(z) = 1 - amp (1 + cos(2 pi (z / Lz - 1/2))) / 2, a smooth neck of
      relative depth amp at mid-length (exact volume Lx Ly Lz (1 - amp + 3 amp^2 / 8))."""
    X = node_coords(m)
    if kind == "affine":
        return np.ascontiguousarray((X @ np.asarray(M, dtype=float).T).T)
    if kind in ("cylinder", "dogbone"):
        Lx, Ly, Lz = m.L
        cx, cy = 0.5 * Lx, 0.5 * Ly
        Y = X.copy()
        if kind == "cylinder":
            R = 0.5 * min(Lx, Ly)
            u, v = 2.0 * X[:, 0] / Lx - 1.0, 2.0 * X[:, 1] / Ly - 1.0
            Y[:, 0] = cx + R * u * np.sqrt(1.0 - 0.5 * v * v)
            Y[:, 1] = cy + R * v * np.sqrt(1.0 - 0.5 * u * u)
        else:
            sz = 1.0 - amp * 0.5 * (1.0 + np.cos(2.0 * np.pi * (X[:, 2] / Lz - 0.5)))
            Y[:, 0] = cx + sz * (X[:, 0] - cx)
            Y[:, 1] = cy + sz * (X[:, 1] - cy)
        return np.ascontiguousarray(Y.T)
    h = np.array(m.h)
    L = np.array(m.L)
    if kind == "smooth":
        Y = X.copy()
        for d in range(3):
            d1, d2 = (d + 1) % 3, (d + 2) % 3
            Y[:, d] += amp * h[d] * np.sin(2 * np.pi * X[:, d1] / L[d1]) * np.sin(np.pi * X[:, d2] / L[d2])
        return np.ascontiguousarray(Y.T)
    if kind != "vertices":
        raise ValueError(kind)
    rng = np.random.default_rng(seed)
    V = np.stack(np.meshgrid(np.arange(m.nx + 1) * h[0], np.arange(m.ny + 1) * h[1], np.arange(m.nz + 1) * h[2],
                             indexing="ij"), -1)
    V = V + rng.uniform(-amp, amp, V.shape) * h
    g = (gll_points(m.p) + 1.0) * 0.5
    out = np.zeros((3, m.nn))
    for ez in range(m.nz):
        for ey in range(m.ny):
            for ex in range(m.nx):
                for c in range(m.p + 1):
                    for b in range(m.p + 1):
                        for a in range(m.p + 1):
                            t = (g[a], g[b], g[c])
                            x = np.zeros(3)
                            for k in range(8):
                                i, j, l = k & 1, (k >> 1) & 1, k >> 2
                                wgt = (t[0] if i else 1 - t[0]) * (t[1] if j else 1 - t[1]) * (t[2] if l else 1 - t[2])
                                x += wgt * V[ex + i, ey + j, ez + l]
                            n = (m.p * ex + a) + m.nnx * ((m.p * ey + b) + m.nny * (m.p * ez + c))
                            out[:, n] = x
    return out


def qpoint_coords(m: Mesh) -> np.ndarray:
    """Reference coordinates of every Gauss point, shape [nq, 3] (q = e Q^3 + i + Q (j + Q k))."""
    g = gauss_points(m.Q)
    hx, hy, hz = m.h
    ex = np.arange(m.nx)
    ey = np.arange(m.ny)
    ez = np.arange(m.nz)
    # element-major, then k, j, i (i fastest)
    EZ, EY, EX, K, J, I = np.meshgrid(ez, ey, ex, np.arange(m.Q), np.arange(m.Q), np.arange(m.Q), indexing="ij")
    x = EX * hx + (g[I] + 1) * 0.5 * hx
    y = EY * hy + (g[J] + 1) * 0.5 * hy
    z = EZ * hz + (g[K] + 1) * 0.5 * hz
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


# ---------------------------------------------------------------------------
# Microstructure: seeded spheres, lognormal radii, force-biased relaxation
# ---------------------------------------------------------------------------
@dataclass
class Spheres:
    centers: np.ndarray
    radii: np.ndarray
    max_overlap: float
    sweeps: int


def place_spheres(seed: int, mean: float, sd: float, vf: float, max_sweeps: int = 300) -> Spheres:
    """Spheres in the unit cube (periodic), radii lognormal(mean, sd), until their
    summed volume reaches ``vf``; overlaps pushed apart pairwise until the largest
    relative overlap is below 1e-3 or ``max_sweeps`` is reached."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    s2 = math.log(1.0 + (sd / mean) ** 2)
    mu = math.log(mean) - 0.5 * s2
    radii = []
    vol = 0.0
    while vol < vf:
        r = float(rng.lognormal(mu, math.sqrt(s2)))
        r = min(r, 0.45)
        radii.append(r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    radii = np.array(sorted(radii, reverse=True))
    centers = rng.random((len(radii), 3))
    rmax = radii.max()
    worst = 0.0
    sweep = 0
    for sweep in range(1, max_sweeps + 1):
        tree = cKDTree(centers, boxsize=1.0)
        pairs = tree.query_pairs(2.0 * rmax, output_type="ndarray")
        if len(pairs) == 0:
            worst = 0.0
            break
        d = centers[pairs[:, 1]] - centers[pairs[:, 0]]
        d -= np.round(d)
        dist = np.linalg.norm(d, axis=1)
        rs = radii[pairs[:, 0]] + radii[pairs[:, 1]]
        ov = rs - dist
        sel = ov > 0
        if not np.any(sel):
            worst = 0.0
            break
        worst = float(np.max(ov[sel] / rs[sel]))
        if worst < 1e-3:
            break
        pr, d, dist, ov = pairs[sel], d[sel], np.maximum(dist[sel], 1e-12), ov[sel]
        push = (0.5 * ov / dist)[:, None] * d
        np.add.at(centers, pr[:, 0], -push)
        np.add.at(centers, pr[:, 1], push)
        centers %= 1.0
    return Spheres(centers, radii, worst, sweep)


def phase_map(points_unit: np.ndarray, sph: Spheres, chunk: int = 1 << 20) -> np.ndarray:
    """uint8 phase per point: 1 inside any (periodic) sphere = particle, 0 = matrix.
    ``points_unit`` are coordinates scaled to the unit cube."""
    from scipy.spatial import cKDTree

    tree = cKDTree(sph.centers, boxsize=1.0)
    rmax = sph.radii.max()
    out = np.zeros(len(points_unit), dtype=np.uint8)
    pts = np.mod(points_unit, 1.0)
    for s in range(0, len(pts), chunk):
        p = pts[s:s + chunk]
        near = tree.query_ball_point(p, rmax)
        for i, lst in enumerate(near):
            if not lst:
                continue
            d = sph.centers[lst] - p[i]
            d -= np.round(d)
            if np.any(np.einsum("ij,ij->i", d, d) < sph.radii[lst] ** 2):
                out[s + i] = 1
    return out


def phase_map_fast(m: Mesh, sph: Spheres, scale: np.ndarray) -> np.ndarray:
    """Phase per Gauss point by rasterising each sphere's bounding box on the
    structured grid of Gauss points (same result as ``phase_map``)."""
    g = gauss_points(m.Q)
    h = np.array(m.h)
    n = np.array([m.nx, m.ny, m.nz])
    # 1D Gauss coordinates along each axis, in unit-cube coordinates
    axes = []
    for d in range(3):
        e = np.arange(n[d])[:, None]
        axes.append(((e * h[d] + (g[None, :] + 1) * 0.5 * h[d]) / scale[d]).ravel())
    nqx, nqy, nqz = len(axes[0]), len(axes[1]), len(axes[2])
    grid = np.zeros((nqz, nqy, nqx), dtype=np.uint8)
    for c, r in zip(sph.centers, sph.radii):
        for sx in (-1, 0, 1):
            for sy in (-1, 0, 1):
                for sz in (-1, 0, 1):
                    cc = c + np.array([sx, sy, sz])
                    lo = cc - r
                    hi = cc + r
                    if np.any(hi < 0) or np.any(lo > 1):
                        continue
                    ix = np.nonzero((axes[0] >= lo[0]) & (axes[0] <= hi[0]))[0]
                    iy = np.nonzero((axes[1] >= lo[1]) & (axes[1] <= hi[1]))[0]
                    iz = np.nonzero((axes[2] >= lo[2]) & (axes[2] <= hi[2]))[0]
                    if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
                        continue
                    dx = (axes[0][ix] - cc[0]) ** 2
                    dy = (axes[1][iy] - cc[1]) ** 2
                    dz = (axes[2][iz] - cc[2]) ** 2
                    inside = (dz[:, None, None] + dy[None, :, None] + dx[None, None, :]) < r * r
                    sub = grid[np.ix_(iz, iy, ix)]
                    grid[np.ix_(iz, iy, ix)] = sub | inside.astype(np.uint8)
    # reorder from the (z,y,x) Gauss grid to element-major q = e Q^3 + i + Q (j + Q k)
    Q = m.Q
    g6 = grid.reshape(m.nz, Q, m.ny, Q, m.nx, Q)  # ez, k, ey, j, ex, i
    return np.ascontiguousarray(g6.transpose(0, 2, 4, 1, 3, 5)).ravel()


# ---------------------------------------------------------------------------
# Dirichlet data
# ---------------------------------------------------------------------------
def dirichlet_tension(m: Mesh, delta: float):
    """Bottom face z = 0 clamped; top face z = Lz: u_x = u_y = 0, u_z = delta."""
    mask = np.zeros((4, m.nnz, m.nny, m.nnx), dtype=np.uint8)
    vals = np.zeros((4, m.nnz, m.nny, m.nnx))
    mask[0:3, 0] = 1
    mask[0:3, -1] = 1
    vals[2, -1] = delta
    return mask.reshape(4, -1), vals.reshape(4, -1)


def dirichlet_compression(m: Mesh, delta: float):
    """Frictionless platens: u_z = 0 at z = 0, u_z = -delta at z = Lz, u_x = 0 on
    x = 0, u_y = 0 on y = 0."""
    mask = np.zeros((4, m.nnz, m.nny, m.nnx), dtype=np.uint8)
    vals = np.zeros((4, m.nnz, m.nny, m.nnx))
    mask[2, 0] = 1
    mask[2, -1] = 1
    vals[2, -1] = -delta
    mask[0, :, :, 0] = 1
    mask[1, :, 0, :] = 1
    return mask.reshape(4, -1), vals.reshape(4, -1)


def top_face_mask(m: Mesh) -> np.ndarray:
    """uint8 [4][nn] selecting the u_z DoFs of the top face (reaction force)."""
    mask = np.zeros((4, m.nnz, m.nny, m.nnx), dtype=np.uint8)
    mask[2, -1] = 1
    return mask.reshape(4, -1)


# ---------------------------------------------------------------------------
# Random fields and histories
# ---------------------------------------------------------------------------
def random_state(m: Mesh, seed: int = 0, u_amp: float = 1e-3, phi_max: float = 0.3) -> np.ndarray:
    """Nodal z [4][nn]: u ~ U[-u_amp, u_amp] (mm), phi ~ U[0, phi_max]; PCG64(seed),
    drawn in the order u_x, u_y, u_z, phi over nodes in lexicographic order."""
    rng = np.random.default_rng(seed)
    z = np.empty((4, m.nn))
    for f in range(3):
        z[f] = rng.uniform(-u_amp, u_amp, m.nn)
    z[3] = rng.uniform(0.0, phi_max, m.nn)
    return z


def random_vector(n: int, seed: int = 1) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def zero_history(nq: int, H0: float = 0.0) -> np.ndarray:
    """Committed history [15][nq]: C_M = C_P = I (Voigt), eps_p = 0, H = H0, phi_n = 0."""
    h = np.zeros((15, nq))
    h[0:3] = 1.0
    h[6:9] = 1.0
    h[13] = H0
    return h


def _sym_from_voigt(v):
    A = np.empty(v.shape[:-1] + (3, 3))
    A[..., 0, 0], A[..., 1, 1], A[..., 2, 2] = v[..., 0], v[..., 1], v[..., 2]
    A[..., 1, 2] = A[..., 2, 1] = v[..., 3]
    A[..., 0, 2] = A[..., 2, 0] = v[..., 4]
    A[..., 0, 1] = A[..., 1, 0] = v[..., 5]
    return A


def random_history(nq: int, seed: int = 2, c_amp: float = 0.05, ep_max: float = 0.01,
                   H_max: float = 1.0, phi_n_max: float = 0.3) -> np.ndarray:
    """Committed history [15][nq] with isochoric C_M, C_P = exp(S), S symmetric
    traceless with |S|_F <= c_amp, eps_p ~ U[0, ep_max], H ~ U[0, H_max],
    phi_n ~ U[0, phi_n_max]."""
    rng = np.random.default_rng(seed)
    h = np.zeros((15, nq))
    for off in (0, 6):
        v = rng.uniform(-1.0, 1.0, (nq, 6))
        S = _sym_from_voigt(v)
        tr = np.trace(S, axis1=1, axis2=2)
        S -= tr[:, None, None] / 3.0 * np.eye(3)
        nrm = np.linalg.norm(S, axis=(1, 2))
        S *= (c_amp * rng.uniform(0.0, 1.0, nq) / np.maximum(nrm, 1e-300))[:, None, None]
        w, V = np.linalg.eigh(S)
        C = np.einsum("nij,nj,nkj->nik", V, np.exp(w), V)
        h[off + 0], h[off + 1], h[off + 2] = C[:, 0, 0], C[:, 1, 1], C[:, 2, 2]
        h[off + 3], h[off + 4], h[off + 5] = C[:, 1, 2], C[:, 0, 2], C[:, 0, 1]
    h[12] = rng.uniform(0.0, ep_max, nq)
    h[13] = rng.uniform(0.0, H_max, nq)
    h[14] = rng.uniform(0.0, phi_n_max, nq)
    return h


# ---------------------------------------------------------------------------
# Workload definitions
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mesh: Mesh
    phases: np.ndarray            # [nphase][12]
    glob: np.ndarray              # [5]
    phase: np.ndarray             # uint8 [nq]
    z: np.ndarray                 # [4][nn] state
    hist: np.ndarray              # [15][nq]
    mask: np.ndarray | None = None
    dvals: np.ndarray | None = None
    meta: dict = field(default_factory=dict)
    X: np.ndarray | None = None   # nodal coordinates [3][nn] of a mapped mesh (None: the box of `mesh`)


def cube(nx: int = 4, p: int = 2, seed_state: int = 0, hist_seed: int | None = None,
         H_max: float = 1.0, u_amp: float = 1e-3) -> Workload:
    """Homogeneous unit cube (Table 2, Example 3 matrix), AT2, dt = 0.01 s,
    eta = 1e-3, zeta = 1e-2 MPa s, no Dirichlet conditions."""
    m = Mesh(nx, nx, nx, p, p + 1, (1.0, 1.0, 1.0))
    at = 2
    glob = glob_vector(at, 1e-3, 1e-2, 0.01, EX3_MATRIX["s_phi"][at])
    phases = np.stack([phase_vector(EX3_MATRIX)])
    phase = np.zeros(m.nq, dtype=np.uint8)
    z = random_state(m, seed_state, u_amp=u_amp)
    hist = zero_history(m.nq) if hist_seed is None else random_history(m.nq, hist_seed, H_max=H_max)
    return Workload("cube" if hist_seed is None else "cube_b", m, phases, glob, phase, z, hist)


def two_phase_box(nx, ny, nz, p, L, sph_mean, sph_sd, vf, seed, at, example, bc, delta,
                  dt, eta=1e-3, zeta=1e-2, notch=False) -> Workload:
    m = Mesh(nx, ny, nz, p, p + 1, L)
    if example == "3adj":
        matrix, particle = EX3_MATRIX, EX3_PARTICLE_ADJ
    elif example == 3:
        matrix, particle = EX3_MATRIX, EX3_PARTICLE
    else:
        matrix, particle = EX2_MATRIX, EX2_PARTICLE
    phases = np.stack([phase_vector(matrix), phase_vector(particle)])
    glob = glob_vector(at, eta, zeta, dt, matrix["s_phi"][at])
    sph = place_spheres(seed, sph_mean, sph_sd, vf)
    scale = np.array(L) / max(L)
    phase = phase_map_fast(m, sph, np.array([max(L)] * 3))
    H0 = np.zeros(m.nq)
    if at == 1:  # AT1 runs start from the threshold psi_c of each phase
        for ph_id, d in ((0, matrix), (1, particle)):
            H0[phase == ph_id] = d["psi_c"]
    hist = zero_history(m.nq)
    hist[13] = H0
    z = np.zeros((4, m.nn))
    if notch:
        xq = qpoint_coords(m)
        sel = (xq[:, 0] < 0.2 * L[0]) & (np.abs(xq[:, 2] - 0.5 * L[2]) < 0.01 * L[2])
        hist[13, sel] = 1e4 * hist[13, sel]
        X = node_coords(m)
        nsel = (X[:, 0] < 0.2 * L[0]) & (np.abs(X[:, 2] - 0.5 * L[2]) < 0.01 * L[2])
        z[3, nsel] = 1.0
    mask, dvals = (dirichlet_tension if bc == "tension" else dirichlet_compression)(m, delta)
    z[mask.astype(bool)] = dvals[mask.astype(bool)]
    meta = dict(spheres=len(sph.radii), max_overlap=sph.max_overlap, sweeps=sph.sweeps,
                vf_points=float(phase.mean()), scale=scale.tolist())
    return Workload("box", m, phases, glob, phase, z, hist, mask, dvals, meta)


def tension_q4(n: int = 16, seed: int = 0) -> Workload:
    """Q4, n^3 elements on L = 0.16 mm (h = 2 l0), spheres mean 0.06 L / sd 0.02 L,
    vf 0.6, tension at 0.4 /s, AT1, Example 3; 10 steps to 2 % strain."""
    L = 0.16 * n / 16.0
    strain_per_step = 0.002
    dt = strain_per_step / 0.4
    w = two_phase_box(n, n, n, 4, (L, L, L), 0.06, 0.02, 0.6, seed, 1, 3, "tension",
                      strain_per_step * L, dt)
    w.name = "tension_q4"
    w.meta.update(steps=10, strain_per_step=strain_per_step)
    return w


def notched_q3(n: int = 48, seed: int = 0) -> Workload:
    L = (0.01 * n, 0.01 * n, 0.03 * n)
    strain_per_step = 0.001
    w = two_phase_box(n, n, 3 * n, 3, L, 0.06, 0.02, 0.6, seed, 1, 3, "tension",
                      strain_per_step * L[2], strain_per_step / 0.4, notch=True)
    w.name = "notched_q3"
    w.meta.update(steps=40, strain_per_step=strain_per_step)
    return w


def adjoint_q2(n: int = 24, seed: int = 0) -> Workload:
    L = 0.01 * n
    strain_per_step = 0.001
    w = two_phase_box(n, n, n, 2, (L, L, L), 0.06, 0.02, 0.6, seed, 2, "3adj", "tension",
                      strain_per_step * L, strain_per_step / 0.4)
    w.name = "adjoint_q2"
    w.meta.update(steps=20, strain_per_step=strain_per_step)
    return w


def compress_q4(n: int = 64, seed: int = 0) -> Workload:
    L = 0.01 * n
    strain_per_step = 0.001
    w = two_phase_box(n, n, n, 4, (L, L, L), 0.04, 0.015, 0.7, seed, 2, 2, "compression",
                      strain_per_step * L, strain_per_step / 0.05, eta=1e-2)
    w.name = "compress_q4"
    w.meta.update(steps=30, strain_per_step=strain_per_step)
    return w


def coarsen_mask(m: Mesh, mask: np.ndarray, pc: int) -> np.ndarray:
    """Dirichlet mask of the order-pc level on the same element grid, for masks
    that are constant on each boundary class (face, edge, corner, interior):
    a coarse node is prescribed iff the fine nodes of its class are."""
    mf = np.asarray(mask, dtype=np.uint8).reshape(4, m.nnz, m.nny, m.nnx)
    sizes_f = (m.nnx, m.nny, m.nnz)
    sizes_c = (pc * m.nx + 1, pc * m.ny + 1, pc * m.nz + 1)

    def cls(n):
        c = np.ones(n, dtype=np.int64)
        c[0] = 0
        c[-1] = 2
        return c

    out = np.zeros((4, sizes_c[2], sizes_c[1], sizes_c[0]), dtype=np.uint8)
    cf = [cls(s) for s in sizes_f]
    cc = [cls(s) for s in sizes_c]
    for f in range(4):
        table = np.zeros((3, 3, 3), dtype=np.uint8)
        for kz in range(3):
            for ky in range(3):
                for kx in range(3):
                    sel = mf[f][np.ix_(cf[2] == kz, cf[1] == ky, cf[0] == kx)]
                    if sel.size:
                        if sel.min() != sel.max():
                            raise ValueError("mask is not constant on a boundary class")
                        table[kz, ky, kx] = sel.flat[0]
        out[f] = table[np.ix_(cc[2], cc[1], cc[0])]
    return out.reshape(4, -1)


def element_offsets(m: Mesh) -> np.ndarray:
    """Explicit element -> node map int32 [nel][P^3] of the structured box (for
    exercising the general restriction)."""
    P = m.p + 1
    e = np.arange(m.nel)
    ex, ey, ez = e % m.nx, (e // m.nx) % m.ny, e // (m.nx * m.ny)
    a = np.arange(P)
    C, B, A = np.meshgrid(a, a, a, indexing="ij")
    I = m.p * ex[:, None] + A.ravel()[None, :]
    J = m.p * ey[:, None] + B.ravel()[None, :]
    K = m.p * ez[:, None] + C.ravel()[None, :]
    return (I + m.nnx * (J + m.nny * K)).astype(np.int32)


def twin_target(theta, seed: int = 1, sigma: float = 0.1):
    """Parameters of the twin experiment that generates the target reaction
    curve: theta scaled by seeded lognormal factors (sigma 0.1)."""
    rng = np.random.default_rng(seed)
    return np.asarray(theta) * np.exp(rng.normal(0.0, sigma, len(theta)))


# Parameter vector theta of the adjoint (12 entries): for phase k in (0, 1) the six
# entries E_inf, nu_inf, sigma0, eta_d, Gc, l0 at 6 k + (0..5).
PARAM_SLOTS = (2, 3, 11, 7, 0, 1)   # their positions in the 12-double phase row


def with_params(phases, theta):
    ph = np.array(phases, dtype=np.float64, copy=True)
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 6)
    for k in range(min(len(ph), len(th))):
        for j, slot in enumerate(PARAM_SLOTS):
            ph[k, slot] = th[k, j]
    return ph


def params_of(phases):
    return np.array([[p[s] for s in PARAM_SLOTS] for p in phases]).ravel()
