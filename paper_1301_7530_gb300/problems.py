"""Seeded synthetic workloads: Q1 hexahedral linear elasticity on the unit cube.

This module builds the inputs of the solver sequences, A^(k) x^(k) = b^(k) (Eq. 1 of the
paper, Section 1): a 3x3 block-CSR stiffness matrix over the free nodes and right-hand
sides made of surface tractions.  It contains none of the solver's arithmetic (no CG, no
projection, no recycling) and is shared, as an input generator only, by the CUDA path,
the CPU oracle, the tests and the benchmark.

Mesh and discretisation
  * Unit cube, N^3 cubic Q1 elements of side h = 1/N, trilinear shape functions,
    2x2x2 Gauss quadrature, isotropic material (Young's modulus E per element, Poisson
    ratio nu shared by all elements).
  * Nodes (i, j, k), i the x index (0..N), j the y index, k the z index.  Nodes with
    i = 0 are clamped (u = 0) and eliminated; the free nodes (i >= 1) are numbered
    f(i, j, k) = (i - 1) + N*j + N*(N+1)*k, so block row f holds node (i, j, k).
  * Block columns of a row are sorted ascending; the diagonal block is always present.
  * Free node count N*(N+1)^2, free dofs n = 3*N*(N+1)^2,
    stored blocks nb = (3N-2)*(3N+1)^2.

Loads
  * A nodal traction field t on the x = 1 face, drawn i.i.d. U[-1, 1] per face node and
    component, is integrated against the bilinear face shape functions (consistent
    nodal forces f = h^2 (M1 (x) M1) t with the 1D mass matrix M1 of the face grid).

Random numbers come from numpy.random.Generator(PCG64(seed)); the draw order of each
generator is stated in its docstring so that the inputs can be regenerated elsewhere.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "BSR3",
    "element_stiffness_unit",
    "assemble",
    "traction_rhs",
    "uniform_modulus",
    "ellipsoid_mask",
    "sphere_inclusions_mask",
    "elasticity_sequence_fixed",
    "elasticity_sequence_damage",
    "elasticity_inclusions",
    "damage_parts",
    "damage_matrix",
    "batch_sizes",
    "sizes",
]


@dataclasses.dataclass
class BSR3:
    """3x3 block-CSR matrix (int32 indices, float64 blocks, row-major 3x3 blocks)."""

    row_ptr: np.ndarray  # int32[nbr + 1]
    col_idx: np.ndarray  # int32[nb]
    vals: np.ndarray     # float64[nb, 3, 3]

    @property
    def n_block_rows(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n(self) -> int:
        return 3 * self.n_block_rows

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    def to_dense(self) -> np.ndarray:
        """Dense copy (tests on tiny meshes only)."""
        n = self.n
        out = np.zeros((n, n))
        for i in range(self.n_block_rows):
            for k in range(self.row_ptr[i], self.row_ptr[i + 1]):
                c = self.col_idx[k]
                out[3 * i:3 * i + 3, 3 * c:3 * c + 3] = self.vals[k]
        return out

    def to_scipy(self):
        """scipy.sparse.bsr_matrix view (tests only)."""
        import scipy.sparse as sp
        return sp.bsr_matrix((self.vals, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def sizes(N: int) -> dict:
    """Closed-form sizes of the clamped N^3 cube."""
    nodes = N * (N + 1) ** 2
    return {"N": N, "free_nodes": nodes, "n": 3 * nodes, "nb": (3 * N - 2) * (3 * N + 1) ** 2}


# ----------------------------------------------------------------------------------------
# Element stiffness
# ----------------------------------------------------------------------------------------

def _local_offsets() -> np.ndarray:
    """Local node a = ax + 2*ay + 4*az -> (ax, ay, az)."""
    return np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)


def _hooke(E: float, nu: float) -> np.ndarray:
    """Isotropic Hooke matrix, Voigt order (xx, yy, zz, yz, xz, xy), engineering shears."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def element_stiffness_unit(nu: float) -> np.ndarray:
    """24x24 stiffness of the unit cube Q1 element with E = 1 (2x2x2 Gauss rule).

    The element of side h and modulus E has stiffness E * h * K (B scales as 1/h and the
    volume as h^3).  Dof order: 3*a + component, local node a as in _local_offsets().
    """
    off = _local_offsets()
    D = _hooke(1.0, nu)
    g = [0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)]
    K = np.zeros((24, 24))
    for gx in g:
        for gy in g:
            for gz in g:
                xi = (gx, gy, gz)
                dN = np.zeros((8, 3))
                for a in range(8):
                    f = [xi[d] if off[a, d] else 1.0 - xi[d] for d in range(3)]
                    s = [1.0 if off[a, d] else -1.0 for d in range(3)]
                    dN[a, 0] = s[0] * f[1] * f[2]
                    dN[a, 1] = f[0] * s[1] * f[2]
                    dN[a, 2] = f[0] * f[1] * s[2]
                B = np.zeros((6, 24))
                for a in range(8):
                    dx, dy, dz = dN[a]
                    B[0, 3 * a + 0] = dx
                    B[1, 3 * a + 1] = dy
                    B[2, 3 * a + 2] = dz
                    B[3, 3 * a + 1] = dz
                    B[3, 3 * a + 2] = dy
                    B[4, 3 * a + 0] = dz
                    B[4, 3 * a + 2] = dx
                    B[5, 3 * a + 0] = dy
                    B[5, 3 * a + 1] = dx
                K += 0.125 * B.T @ D @ B
    return K


# ----------------------------------------------------------------------------------------
# Assembly
# ----------------------------------------------------------------------------------------

def _slot(d: np.ndarray) -> int:
    """Neighbour slot of the offset (dx, dy, dz) in {-1, 0, 1}^3; ascending in column."""
    return int((d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1))


def assemble(N: int, E_elem: np.ndarray, nu: float = 0.3, clamp: bool = True) -> BSR3:
    """Assemble the Q1 stiffness of the N^3 cube into 3x3 BSR.

    E_elem: float64[N, N, N] indexed [ez, ey, ex] (element Young's moduli).
    clamp=True eliminates the nodes at x = 0 (the solver's matrices); clamp=False keeps
    every node (singular: the 6 rigid-body modes span its null space; tests only).
    """
    E_elem = np.asarray(E_elem, dtype=np.float64)
    assert E_elem.shape == (N, N, N)
    h = 1.0 / N
    K = element_stiffness_unit(nu)
    off = _local_offsets()
    M = N + 1
    # dense slot array over all nodes: [k, j, i, slot, 3, 3]
    blocks = np.zeros((M, M, M, 27, 3, 3))
    Eh = E_elem * h
    for a in range(8):
        ax, ay, az = off[a]
        for b in range(8):
            s = _slot(off[b] - off[a])
            kab = K[3 * a:3 * a + 3, 3 * b:3 * b + 3]
            blocks[az:az + N, ay:ay + N, ax:ax + N, s] += Eh[:, :, :, None, None] * kab
    i0 = 1 if clamp else 0
    nx = M - i0  # free nodes along x
    kk, jj, ii = np.meshgrid(np.arange(M), np.arange(M), np.arange(i0, M), indexing="ij")
    valid = np.zeros((M, M, nx, 27), dtype=bool)
    ncol = np.zeros((M, M, nx, 27), dtype=np.int64)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                s = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                ci, cj, ck = ii + dx, jj + dy, kk + dz
                ok = (ci >= i0) & (ci < M) & (cj >= 0) & (cj < M) & (ck >= 0) & (ck < M)
                valid[..., s] = ok
                ncol[..., s] = (ci - i0) + nx * cj + nx * M * ck
    sub = blocks[:, :, i0:, :, :, :]
    counts = valid.reshape(-1, 27).sum(axis=1)
    row_ptr = np.zeros(counts.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    vmask = valid.reshape(-1)
    col_idx = ncol.reshape(-1)[vmask]
    vals = sub.reshape(-1, 3, 3)[vmask]
    return BSR3(row_ptr.astype(np.int32), col_idx.astype(np.int32), np.ascontiguousarray(vals))


# ----------------------------------------------------------------------------------------
# Right-hand sides
# ----------------------------------------------------------------------------------------

def _mass_1d(M: int, h: float) -> np.ndarray:
    """Assembled 1D linear-element mass matrix on M nodes (spacing h), dense."""
    m = np.zeros((M, M))
    for e in range(M - 1):
        m[e:e + 2, e:e + 2] += h * np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
    return m


def traction_rhs(N: int, traction: np.ndarray) -> np.ndarray:
    """Consistent nodal forces of a nodal traction field on the x = 1 face.

    traction: float64[N+1, N+1, 3] indexed [k, j, component] (face node (N, j, k)).
    Returns b: float64[n] over the free dofs (zero away from the loaded face).
    """
    M = N + 1
    h = 1.0 / N
    t = np.asarray(traction, dtype=np.float64)
    assert t.shape == (M, M, 3)
    m1 = _mass_1d(M, h)
    f = np.einsum("kK,jJ,KJc->kjc", m1, m1, t)
    b = np.zeros((M, M, N, 3))  # [k, j, i-1, c]
    b[:, :, N - 1, :] = f
    return b.reshape(-1)


def random_traction(N: int, seed: int) -> np.ndarray:
    """i.i.d. U[-1, 1] nodal tractions: one draw rng.uniform(-1, 1, (N+1, N+1, 3))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(N + 1, N + 1, 3))


# ----------------------------------------------------------------------------------------
# Material fields
# ----------------------------------------------------------------------------------------

def _centroids(N: int):
    c = (np.arange(N) + 0.5) / N
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    return cx, cy, cz


def uniform_modulus(N: int, E: float = 1.0) -> np.ndarray:
    return np.full((N, N, N), float(E))


def ellipsoid_mask(N: int, seed: int):
    """Axis-aligned ellipsoid: centre U[0.3, 0.7]^3 then semi-axes U[0.1, 0.25]^3.

    Draw order: rng.uniform(0.3, 0.7, 3), then rng.uniform(0.1, 0.25, 3).
    An element is inside when its centroid is.  Returns (mask[N,N,N], centre, axes).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = rng.uniform(0.3, 0.7, size=3)
    axes = rng.uniform(0.1, 0.25, size=3)
    cx, cy, cz = _centroids(N)
    r = ((cx - centre[0]) / axes[0]) ** 2 + ((cy - centre[1]) / axes[1]) ** 2 \
        + ((cz - centre[2]) / axes[2]) ** 2
    return r <= 1.0, centre, axes


def sphere_inclusions_mask(N: int, seed: int, fraction: float = 0.05):
    """Spheres added until at least `fraction` of the elements (by centroid) are inside.

    Each sphere draws rng.uniform(0, 1, 3) (centre) then rng.uniform(0.04, 0.08) (radius).
    Returns (mask[N,N,N], list of (centre, radius)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cx, cy, cz = _centroids(N)
    mask = np.zeros((N, N, N), dtype=bool)
    spheres = []
    while mask.mean() < fraction:
        c = rng.uniform(0.0, 1.0, size=3)
        rad = rng.uniform(0.04, 0.08)
        spheres.append((c, rad))
        mask |= (cx - c[0]) ** 2 + (cy - c[1]) ** 2 + (cz - c[2]) ** 2 <= rad * rad
    return mask, spheres


# ----------------------------------------------------------------------------------------
# Sequences
# ----------------------------------------------------------------------------------------

def elasticity_sequence_fixed(N: int, n_systems: int, seed0: int, E: float = 1.0,
                              nu: float = 0.3):
    """Fixed A, one random traction field per system (system k uses seed seed0 + k).

    Returns (A, [b_0, ..., b_{p-1}]).
    """
    A = assemble(N, uniform_modulus(N, E), nu)
    bs = [traction_rhs(N, random_traction(N, seed0 + k)) for k in range(n_systems)]
    return A, bs


def damage_factors(n_systems: int, d_final: float = 0.05) -> np.ndarray:
    """d_k = d_final^(k / (p - 1)), k = 0..p-1: falls geometrically from 1 to d_final."""
    if n_systems == 1:
        return np.ones(1)
    return d_final ** (np.arange(n_systems) / (n_systems - 1))


def elasticity_sequence_damage(N: int, n_systems: int, seed_geom: int, seed_rhs: int,
                               E: float = 1.0, nu: float = 0.3, d_final: float = 0.05):
    """Secant damage sequence: elements in a seeded ellipsoid get E * d_k.

    The right-hand side is fixed (tractions drawn with seed_rhs).  Yields a generator of
    (k, A^(k)) pairs (assembled lazily) and returns (mask, b, generator).
    """
    mask, _, _ = ellipsoid_mask(N, seed_geom)
    b = traction_rhs(N, random_traction(N, seed_rhs))
    d = damage_factors(n_systems, d_final)

    def gen():
        for k in range(n_systems):
            Ee = np.where(mask, E * d[k], E)
            yield k, assemble(N, Ee, nu)

    return mask, b, gen()


def elasticity_inclusions(N: int, seed_geom: int, E: float = 1.0, E_incl: float = 1.0e3,
                          nu: float = 0.3, fraction: float = 0.05) -> BSR3:
    """Heterogeneous cube: matrix modulus E, seeded spherical inclusions of modulus E_incl."""
    mask, _ = sphere_inclusions_mask(N, seed_geom, fraction)
    return assemble(N, np.where(mask, E_incl, E), nu)


# ----------------------------------------------------------------------------------------
# Many sequences (batched and served workloads)
# ----------------------------------------------------------------------------------------

def damage_parts(N: int, seed_geom: int, seed_rhs: int, E: float = 1.0, nu: float = 0.3):
    """Damage sequence in split form.  The stiffness is linear in the element moduli, so
    A^(k) = A_out + d_k * A_in, with A_out assembled from the elements outside the seeded
    ellipsoid (modulus E) and A_in from those inside (modulus E); both have the full
    27-neighbour pattern.  Returns (A_out: BSR3, vals_in: float64[nb, 3, 3], b)."""
    mask, _, _ = ellipsoid_mask(N, seed_geom)
    A_out = assemble(N, np.where(mask, 0.0, E), nu)
    A_in = assemble(N, np.where(mask, E, 0.0), nu)
    assert np.array_equal(A_out.col_idx, A_in.col_idx)
    b = traction_rhs(N, random_traction(N, seed_rhs))
    return A_out, A_in.vals, b


def damage_matrix(A_out: BSR3, vals_in: np.ndarray, d: float) -> BSR3:
    """A_out + d * A_in (host)."""
    return BSR3(A_out.row_ptr, A_out.col_idx, A_out.vals + d * vals_in)


def batch_sizes(n_seq: int, n_min: int, n_max: int, seed: int) -> np.ndarray:
    """Cube sizes N ~ U{n_min, ..., n_max}, one per sequence (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(n_min, n_max + 1, size=n_seq)
