"""Pins of the input generator (Q1 elasticity): closed-form sizes, symmetry, rigid-body
null space of the unclamped operator, patch test, positive definiteness once clamped,
load resultant, seeded reproducibility."""
import numpy as np
import pytest

from paper_1301_7530_gb300 import problems as P


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_sizes_closed_form(N):
    A = P.assemble(N, P.uniform_modulus(N))
    s = P.sizes(N)
    assert A.n == s["n"] and A.nnzb == s["nb"]
    assert A.row_ptr.dtype == np.int32 and A.col_idx.dtype == np.int32
    # sorted columns, diagonal present
    for i in range(A.n_block_rows):
        cols = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols


@pytest.mark.parametrize("N", [2, 3])
def test_symmetric_and_spd_when_clamped(N):
    rng = np.random.default_rng(0)
    E = rng.uniform(0.5, 2.0, size=(N, N, N))
    K = P.assemble(N, E).to_dense()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0
    np.linalg.cholesky(K)


def _node_coords(N, i0=0):
    M = N + 1
    kk, jj, ii = np.meshgrid(np.arange(M), np.arange(M), np.arange(i0, M), indexing="ij")
    return np.stack([ii, jj, kk], -1).reshape(-1, 3) / N


def test_rigid_body_modes_in_null_space():
    N = 3
    rng = np.random.default_rng(1)
    K = P.assemble(N, rng.uniform(0.5, 2.0, size=(N, N, N)), clamp=False).to_dense()
    X = _node_coords(N)
    modes = []
    for c in range(3):
        u = np.zeros_like(X)
        u[:, c] = 1.0
        modes.append(u.reshape(-1))
    for a, b in ((0, 1), (1, 2), (0, 2)):
        u = np.zeros_like(X)
        u[:, a] = -X[:, b]
        u[:, b] = X[:, a]
        modes.append(u.reshape(-1))
    for u in modes:
        assert np.abs(K @ u).max() <= 1e-13 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-12 * ev.max()) == 6


def test_patch_test_linear_field():
    """A linear displacement field gives zero nodal forces at interior nodes."""
    N = 4
    K = P.assemble(N, P.uniform_modulus(N, 3.0), nu=0.25, clamp=False).to_dense()
    X = _node_coords(N)
    G = np.array([[0.3, -0.1, 0.2], [0.05, 0.4, -0.2], [0.1, 0.2, -0.3]])
    u = (X @ G.T).reshape(-1)
    f = (K @ u).reshape(-1, 3)
    M = N + 1
    idx = np.arange(M ** 3).reshape(M, M, M)  # [k, j, i]
    interior = idx[1:-1, 1:-1, 1:-1].reshape(-1)
    assert np.abs(f[interior]).max() <= 1e-12 * np.abs(K).max()
    assert np.abs(f).max() > 1e-3  # boundary forces are not zero


def test_element_stiffness_properties():
    K = P.element_stiffness_unit(0.3)
    assert np.abs(K - K.T).max() < 1e-15
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-12) == 6 and ev.min() > -1e-12


def test_traction_resultant():
    """A uniform unit traction on the unit face integrates to a unit resultant force."""
    N = 5
    t = np.zeros((N + 1, N + 1, 3))
    t[..., 0] = 1.0
    t[..., 2] = -2.0
    b = P.traction_rhs(N, t).reshape(-1, 3)
    assert abs(b[:, 0].sum() - 1.0) < 1e-14
    assert abs(b[:, 2].sum() + 2.0) < 1e-14
    # only the x = 1 face is loaded: nodes (i=N) have free index (N-1) + N*j + ...
    nz = np.nonzero(np.abs(b).sum(axis=1))[0]
    assert np.all(nz % N == N - 1)


def test_seeded_reproducible():
    a = P.random_traction(4, 1003)
    b = P.random_traction(4, 1003)
    assert np.array_equal(a, b) and a.min() >= -1 and a.max() <= 1
    m1, c1, ax1 = P.ellipsoid_mask(8, 7)
    m2, c2, ax2 = P.ellipsoid_mask(8, 7)
    assert np.array_equal(m1, m2) and np.all((c1 >= 0.3) & (c1 <= 0.7)) and np.all((ax1 >= 0.1) & (ax1 <= 0.25))
    mk, sph = P.sphere_inclusions_mask(16, 3)
    assert mk.mean() >= 0.05 and all(0.04 <= r <= 0.08 for _, r in sph)


def test_damage_factors():
    d = P.damage_factors(20)
    assert d[0] == 1.0 and abs(d[-1] - 0.05) < 1e-15
    assert np.allclose(d[1:] / d[:-1], 0.05 ** (1 / 19))
