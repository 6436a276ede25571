"""Pins of the FP64 oracle against things other than itself: closed forms, textbook
CG/PCG and Lanczos written here, numpy/LAPACK routines, hand-derived selection sets,
and the exact relations and equivalences the paper states (Section 2.1 relations (7),
Propositions 1-2, Corollary 1; Section 4.1 Lanczos/Ritz properties)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_1301_7530_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------------
# helpers written independently of the oracle
# ----------------------------------------------------------------------------------------

def dense_bsr(Ad):
    """Every 3x3 block of a dense matrix stored (so any dense operator can be fed in)."""
    n = Ad.shape[0]
    nbr = n // 3
    rp = (np.arange(nbr + 1) * nbr).astype(np.int32)
    ci = np.tile(np.arange(nbr), nbr).astype(np.int32)
    vals = Ad.reshape(nbr, 3, nbr, 3).transpose(0, 2, 1, 3).reshape(-1, 3, 3).copy()
    return P.BSR3(rp, ci, vals)


def textbook_pcg(A, b, Minv, tol, maxit, reorth=False):
    """Hestenes-Stiefel PCG with the (r, M^-1 r) formulas; optional full A-reorth of p."""
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv @ r
    p = z.copy()
    rz = r @ z
    ps, Aps = [], []
    it = 0
    bb = b @ b
    while r @ r > tol * tol * bb and it < maxit:
        Ap = A @ p
        a = rz / (p @ Ap)
        x = x + a * p
        r = r - a * Ap
        ps.append(p.copy())
        Aps.append(Ap.copy())
        it += 1
        if r @ r <= tol * tol * bb:
            break
        z = Minv @ r
        rz_new = r @ z
        if reorth:
            p = z.copy()
            for pi, Api in zip(ps, Aps):
                p = p - (Api @ z) / (pi @ Api) * pi
        else:
            p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def lanczos_process(A, v0, m):
    """Symmetric Lanczos with full reorthogonalisation: diagonal a, off-diagonal b > 0."""
    Q = [v0 / np.linalg.norm(v0)]
    a, bs = [], []
    for j in range(m):
        w = A @ Q[j]
        a.append(Q[j] @ w)
        for q in Q:
            w = w - (q @ w) * q
        for q in Q:
            w = w - (q @ w) * q
        if j < m - 1:
            bs.append(np.linalg.norm(w))
            Q.append(w / bs[-1])
    return np.array(a), np.array(bs)


def small_problem(N=2, seed=5, hetero=True):
    rng = np.random.default_rng(seed)
    E = rng.uniform(0.5, 3.0, size=(N, N, N)) if hetero else P.uniform_modulus(N)
    A = P.assemble(N, E)
    b = P.traction_rhs(N, P.random_traction(N, 1000 + seed))
    return A, b


def block_jacobi_dense(A):
    Ad = A.to_dense()
    M = np.zeros_like(Ad)
    for i in range(A.n_block_rows):
        M[3 * i:3 * i + 3, 3 * i:3 * i + 3] = Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3]
    return M


def run(A, b, tol, C=None, **kw):
    s = O.Sequence(A.n)
    if C is not None:
        s.set_C(C)
    x, st = s.solve(A, b, tol, O.make_policy(**kw))
    return s, x, st


# ----------------------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------------------

def test_spmv_matches_dense():
    A, b = small_problem(3)
    Ad = A.to_dense()
    x = np.random.default_rng(0).standard_normal(A.n)
    assert np.abs(O.spmv(A, x) - Ad @ x).max() <= 1e-14 * np.abs(Ad).max() * np.abs(x).max() * 30


def test_precond_inverse_blocks_and_jacobi():
    A, _ = small_problem(2)
    Ad = A.to_dense()
    mb = O.precond_setup(A, "block_jacobi3").reshape(-1, 3, 3)
    for i in range(A.n_block_rows):
        assert np.allclose(mb[i] @ Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3], np.eye(3), atol=1e-13)
    mj = O.precond_setup(A, "jacobi")[:A.n]
    assert np.allclose(mj * np.diag(Ad), 1.0, atol=1e-15)
    r = np.random.default_rng(1).standard_normal(A.n)
    Mbd = block_jacobi_dense(A)
    assert np.allclose(O.precond_apply("block_jacobi3", A.n_block_rows, mb.reshape(-1), r),
                       np.linalg.solve(Mbd, r), rtol=1e-12, atol=1e-12)


def test_cholesky_and_solve_vs_numpy():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((30, 30))
    G = X @ X.T + 30 * np.eye(30)
    L = O.cholesky(G)
    assert np.allclose(L, np.linalg.cholesky(G), rtol=1e-12, atol=1e-12)
    y = rng.standard_normal(30)
    assert np.allclose(O.chol_solve(L, y), np.linalg.solve(G, y), rtol=1e-11, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_tridiag_eig_closed_form():
    """tridiag(1, 2, 1) of order m: eigenvalues 2 + 2 cos(k pi/(m+1)) with eigenvectors
    sin(j k pi/(m+1)), since sin((j-1)f) + sin((j+1)f) = 2 cos(f) sin(j f)."""
    for m in (1, 2, 7, 40):
        th, Q = O.tridiag_eig(np.full(m, 2.0), np.ones(m - 1))
        k = np.arange(1, m + 1)
        exact = 2.0 + 2.0 * np.cos(k * np.pi / (m + 1))  # already descending
        assert np.allclose(th, exact, atol=1e-13)
        j = np.arange(1, m + 1)
        for c in range(m):
            v = np.sin(j * (c + 1) * np.pi / (m + 1))
            v /= np.linalg.norm(v)
            assert abs(abs(v @ Q[:, c]) - 1.0) < 1e-12


def test_sym_eig_vs_lapack():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((25, 25))
    S = X + X.T
    th, Q = O.sym_eig(S)
    ref = np.linalg.eigvalsh(S)[::-1]
    assert np.allclose(th, ref, atol=1e-12)
    assert np.allclose(Q.T @ Q, np.eye(25), atol=1e-12)
    assert np.allclose(S @ Q, Q * th, atol=1e-11)


def test_srks_selection_golden():
    with open(os.path.join(GOLDEN, "srks_selection.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        got = O.srks_select(np.array(c["theta_m"], float), np.array(c["theta_m1"], float),
                            c["eps"], c["theta_frac"], c["room"])
        assert list(got) == c["expected"], c["name"]


def test_lanczos_formula_matches_lanczos_process():
    """C = 0, M = I: the tridiagonal built from alpha/rho equals the one of the symmetric
    Lanczos process started from b (Section 4.1)."""
    A, b = small_problem(2, seed=7)
    Ad = A.to_dense()
    s, x, st = run(A, b, 1e-11, precond="identity")
    alpha, rho, gamma = s.coeffs()
    m = st["m"]
    delta, eta = O.lanczos(alpha, rho)
    a, bb = lanczos_process(Ad, b, m)
    assert np.allclose(delta, a, rtol=1e-9)
    assert np.allclose(eta, bb, rtol=1e-8)


@pytest.mark.parametrize("with_C", [False, True])
def test_lanczos_identity_VtAV(with_C):
    """V^T A V = H_m with V = [(-1)^j z_j / sqrt(rho_j)] (Eq. 17), with and without C."""
    A, b = small_problem(2, seed=8)
    Ad = A.to_dense()
    C = None
    if with_C:
        C = np.random.default_rng(4).standard_normal((A.n, 5))
    s, x, st = run(A, b, 1e-10, C=C, precond="block_jacobi3")
    m = st["m"]
    alpha, rho, gamma = s.coeffs()
    Z = s.Z
    V = Z * ((-1.0) ** np.arange(m) / np.sqrt(rho))
    H = V.T @ Ad @ V
    delta, eta = O.lanczos(alpha, rho)
    # On the band an index or sign slip in delta / eta / (-1)^j is an O(1) error.  With
    # alpha = (r, w)/(Aw, w) as printed, alpha differs from rho/(Aw, w) by about
    # eps ||r_0|| / ||r_j||, so the band is tight while ||r_j|| is large and loosens
    # towards the end of the solve.
    scale = np.abs(delta).max()
    h = m // 2
    assert np.abs(np.diag(H)[:h] - delta[:h]).max() <= 1e-10 * scale
    assert np.abs(np.diag(H, 1)[:h] - eta[:h]).max() <= 1e-10 * scale
    assert np.abs(np.diag(H) - delta).max() <= 1e-5 * scale
    assert np.abs(np.diag(H, 1) - eta).max() <= 1e-5 * scale
    assert np.all(eta > 0)
    # away from the band only the rounding-level loss of A-conjugacy of the z's remains
    # (full reorthogonalisation acts on the w's, not on the z's)
    T = np.diag(delta) + np.diag(eta, 1) + np.diag(eta, -1)
    assert np.abs(H - T).max() <= 1e-3 * scale


# ----------------------------------------------------------------------------------------
# APCG solve
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("precond", ["identity", "jacobi", "block_jacobi3"])
def test_solution_vs_dense_cholesky(precond):
    A, b = small_problem(3)
    Ad = A.to_dense()
    xe = sla.cho_solve(sla.cho_factor(Ad), b)
    tol = 1e-12
    s, x, st = run(A, b, tol, precond=precond)
    assert st["status"] == 0
    kappa = np.linalg.cond(Ad)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= kappa * tol
    assert st["true_rel_res"] <= 10 * tol


def test_cg_equals_textbook_cg():
    """C = 0, M = I, no reorthogonalisation: APCG is CG (Section 2.1)."""
    A, b = small_problem(2, seed=11)
    Ad = A.to_dense()
    s, x, st = run(A, b, 1e-9, precond="identity", reorth="none")
    xt, it = textbook_pcg(Ad, b, np.eye(A.n), 1e-9, 1000)
    assert abs(st["m"] - it) <= 1
    assert np.linalg.norm(x - xt) <= 1e-8 * np.linalg.norm(xt)


def test_pcg_equals_textbook_pcg_with_reorth():
    """C = 0: APCG(A, M, 0, b) with full reorthogonalisation is PCG."""
    A, b = small_problem(3, seed=12)
    Ad = A.to_dense()
    Minv = np.linalg.inv(block_jacobi_dense(A))
    s, x, st = run(A, b, 1e-10, precond="block_jacobi3")
    xt, it = textbook_pcg(Ad, b, Minv, 1e-10, 2000, reorth=True)
    assert st["m"] == it
    assert np.linalg.norm(x - xt) <= 1e-9 * np.linalg.norm(xt)
    xj, itj = textbook_pcg(Ad, b, np.diag(1 / np.diag(Ad)), 1e-10, 2000, reorth=True)
    s2, x2, st2 = run(A, b, 1e-10, precond="jacobi")
    assert st2["m"] == itj and np.linalg.norm(x2 - xj) <= 1e-9 * np.linalg.norm(xj)


def test_exact_relations_Ct_r_and_conjugacy():
    """C^T r_j = 0, C^T A w_j = 0, (w_i, A w_j) = 0 for i != j (Eq. 5, relations (7))."""
    A, b = small_problem(3, seed=13)
    Ad = A.to_dense()
    C = np.random.default_rng(5).standard_normal((A.n, 8))
    s, x, st = run(A, b, 1e-9, C=C, precond="jacobi")
    r = b - Ad @ x
    assert np.abs(C.T @ r).max() <= 1e-11 * np.linalg.norm(C, 2) * np.linalg.norm(b)
    W, AW = s.W, s.AW
    assert np.allclose(AW, Ad @ W, atol=1e-13 * np.abs(AW).max())
    CtAW = C.T @ AW
    assert np.abs(CtAW).max() <= 1e-10 * np.linalg.norm(C, 2) * np.abs(AW).max() * math.sqrt(A.n)
    G = W.T @ AW
    d = np.sqrt(np.diag(G))
    Gn = G / np.outer(d, d)
    assert np.abs(Gn - np.eye(G.shape[0])).max() <= 1e-10


def test_finite_termination():
    """Exact arithmetic: at most n - n_c iterations (FP64 with full reorth: small slack)."""
    A, b = small_problem(2, seed=14)
    for nc in (0, 6, 20):
        C = np.random.default_rng(nc).standard_normal((A.n, nc)) if nc else None
        s, x, st = run(A, b, 1e-13, C=C, precond="identity")
        assert st["status"] == 0 and st["m"] <= A.n - nc + 2


def test_convergence_bound():
    """m <= ceil(ln(tol / (2 sqrt(kappa(A)))) / ln sigma), sigma from kappa(M^-1 A) (Eq. 10)."""
    A, b = small_problem(3, seed=15)
    Ad = A.to_dense()
    ev = sla.eigh(Ad, np.diag(np.diag(Ad)), eigvals_only=True)
    kap = ev.max() / ev.min()
    sig = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    ka = np.linalg.cond(Ad)
    for tol in (1e-4, 1e-8):
        s, x, st = run(A, b, tol, precond="jacobi")
        assert st["m"] <= math.ceil(math.log(tol / (2 * math.sqrt(ka))) / math.log(sig))


def _projector(Ad, C):
    G = C.T @ Ad @ C
    return np.eye(Ad.shape[0]) - C @ np.linalg.solve(G, C.T @ Ad)


def test_proposition1_residuals_equal_cg_on_projected():
    """APCG(A, I, C, b) has the residuals of CG(P^T A P, P^T b) and x_i = x_0 + P y_i."""
    A, b = small_problem(2, seed=16)
    Ad = A.to_dense()
    C = np.random.default_rng(6).standard_normal((A.n, 4))
    Pm = _projector(Ad, C)
    B = Pm.T @ Ad @ Pm
    x0 = C @ np.linalg.solve(C.T @ Ad @ C, C.T @ b)
    for k in (1, 3, 6):
        s = O.Sequence(A.n)
        s.set_C(C)
        x, st = s.solve(A, b, 0.0, O.make_policy(precond="identity", max_iter=k))
        assert st["m"] == k
        yk, it = textbook_pcg(B, Pm.T @ b, np.eye(A.n), 0.0, k, reorth=True)
        assert it == k
        r_apcg = b - Ad @ x
        r_cg = Pm.T @ b - B @ yk
        assert np.linalg.norm(r_apcg - r_cg) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(x - (x0 + Pm @ yk)) <= 1e-9 * np.linalg.norm(x)


def test_corollary1_nested_augmentation():
    """APCG(A, I, [C, D], b) == APCG(P^T A P, I, D, P^T b): same alphas and m."""
    A, b = small_problem(2, seed=17)
    Ad = A.to_dense()
    rng = np.random.default_rng(7)
    C = rng.standard_normal((A.n, 3))
    D = rng.standard_normal((A.n, 4))
    Pm = _projector(Ad, C)
    s1, x1, st1 = run(A, b, 1e-9, C=np.hstack([C, D]), precond="identity")
    B = Pm.T @ Ad @ Pm
    s2, x2, st2 = run(dense_bsr(B), Pm.T @ b, 1e-9 * np.linalg.norm(b) / np.linalg.norm(Pm.T @ b),
                      C=D, precond="identity")
    assert abs(st1["m"] - st2["m"]) <= 1
    m = min(st1["m"], st2["m"])
    a1 = s1.coeffs()[0][:m]
    a2 = s2.coeffs()[0][:m]
    assert np.allclose(a1, a2, rtol=1e-7)
    x0 = C @ np.linalg.solve(C.T @ Ad @ C, C.T @ b)
    if st1["m"] == st2["m"]:
        assert np.linalg.norm(x1 - (x0 + Pm @ x2)) <= 1e-8 * np.linalg.norm(x1)


def test_proposition2_preconditioned_equivalence():
    """APCG(A, M, C, b) and APCG(L^-1 A L^-T, I, L^T C, L^-1 b) share alpha and m."""
    A, b = small_problem(2, seed=18)
    Ad = A.to_dense()
    M = block_jacobi_dense(A)
    L = np.linalg.cholesky(M)
    Li = np.linalg.inv(L)
    Ah = Li @ Ad @ Li.T
    C = np.random.default_rng(8).standard_normal((A.n, 3))
    s1, x1, st1 = run(A, b, 1e-9, C=C, precond="block_jacobi3")
    bh = Li @ b
    s2, x2, st2 = run(dense_bsr(Ah), bh, 1e-9 * np.linalg.norm(b) / np.linalg.norm(bh),
                      C=L.T @ C, precond="identity")
    m = min(st1["m"], st2["m"])
    assert m >= 5
    assert np.allclose(s1.coeffs()[0][:m], s2.coeffs()[0][:m], rtol=1e-7)
    # rho = (r, z) is the same quantity in both systems
    assert np.allclose(s1.coeffs()[1][:m], s2.coeffs()[1][:m], rtol=1e-7)


def test_deflation_closed_form():
    """Diagonal A, C = eigenvectors of the n_c smallest eigenvalues: APCG is CG on the
    remaining spectrum (Section 2.2; condition number lambda_n / lambda_{n_c+1})."""
    n, nc = 60, 6
    lam = np.geomspace(1e-3, 1.0, n)
    Ad = np.diag(lam)
    A = dense_bsr(Ad)
    b = np.random.default_rng(9).standard_normal(n)
    C = np.eye(n)[:, :nc]
    s, x, st = run(A, b, 1e-10, C=C, precond="identity")
    rest = np.arange(nc, n)
    xr, it = textbook_pcg(np.diag(lam[rest]), b[rest], np.eye(n - nc),
                          1e-10 * np.linalg.norm(b) / np.linalg.norm(b[rest]), 1000, reorth=True)
    assert st["m"] == it
    assert np.allclose(x[:nc], b[:nc] / lam[:nc], rtol=1e-12)
    assert np.allclose(x[rest], xr, rtol=1e-8)


def test_trks_repeated_rhs_needs_no_iteration():
    """Fixed A, TRKS: a right-hand side already in the span of previous ones converges at
    initialisation, to within sqrt(kappa) of the previous tolerance (Algorithm 2)."""
    A, b0 = small_problem(3, seed=19)
    b1 = P.traction_rhs(3, P.random_traction(3, 4242))
    Ad = A.to_dense()
    ka = np.linalg.cond(Ad)
    tol = 1e-10
    s = O.Sequence(A.n)
    pol = O.make_policy("trks", "jacobi")
    s.solve(A, b0, tol, pol)
    s.solve(A, b1, tol, pol)
    b2 = 2.0 * b0 - 0.5 * b1
    tol2 = tol * math.sqrt(ka) * (2 * np.linalg.norm(b0) + 0.5 * np.linalg.norm(b1)) / np.linalg.norm(b2)
    x, st = s.solve(A, b2, tol2, pol)
    assert st["m"] == 0 and st["n_selected"] == 0
    assert st["true_rel_res"] <= tol2


def test_trks_concatenates_directions():
    A, b = small_problem(2, seed=20)
    s = O.Sequence(A.n)
    pol = O.make_policy("trks", "jacobi")
    x, st = s.solve(A, b, 1e-8, pol)
    W = s.W
    assert s.nc == st["m"] and np.array_equal(s.C, W)
    b2 = P.traction_rhs(2, P.random_traction(2, 77))
    x2, st2 = s.solve(A, b2, 1e-8, pol)
    assert st2["n_c"] == st["m"] and s.nc == st["m"] + st2["m"]
    capped = O.Sequence(A.n)
    pol_c = O.make_policy("trks", "jacobi", max_aug=10)
    capped.solve(A, b, 1e-8, pol_c)
    assert capped.nc == 10 and np.array_equal(capped.C, W[:, :10])


def test_srks_ritz_properties_no_augmentation():
    """C = 0: scaled Ritz vectors satisfy Y^T A Y = I and Y^T M Y = Theta^-1 (Section 4.1,
    Eq. 18 with the 1/sqrt(theta) scaling of Algorithm 3); theta_m interlaces theta_{m-1};
    theta_m matches LAPACK on H_m."""
    A, b = small_problem(3, seed=21)
    Ad = A.to_dense()
    M = block_jacobi_dense(A)
    s = O.Sequence(A.n)
    x, st = s.solve(A, b, 1e-10, O.make_policy("srks", "block_jacobi3", ritz_eps=1e-8))
    tm, tm1, sel, Y = s.ritz()
    m = st["m"]
    assert len(sel) >= 2 and s.nc == len(sel)
    YAY = Y.T @ Ad @ Y
    assert np.abs(YAY - np.eye(len(sel))).max() <= 1e-8
    YMY = Y.T @ M @ Y
    assert np.allclose(np.diag(YMY), 1.0 / tm[sel], rtol=1e-7)
    alpha, rho, _ = s.coeffs()
    delta, eta = O.lanczos(alpha, rho)
    ref = sla.eigh_tridiagonal(delta, eta, eigvals_only=True)[::-1]
    assert np.allclose(tm, ref, atol=1e-12 * ref.max())
    ref1 = sla.eigh_tridiagonal(delta[:-1], eta[:-1], eigvals_only=True)[::-1]
    assert np.allclose(tm1, ref1, atol=1e-12 * ref.max())
    tol_i = 1e-12 * tm[0]
    for j in range(m - 1):
        assert tm[j] + tol_i >= tm1[j] >= tm[j + 1] - tol_i
    # ascending theta order of the appended columns
    assert np.all(np.diff(tm[sel]) > 0)


def test_srks_ritz_values_at_termination():
    """Run to termination: the Ritz values are the eigenvalues of M^-1 A."""
    A, b = small_problem(1, seed=22)  # n = 12
    Ad = A.to_dense()
    M = block_jacobi_dense(A)
    s = O.Sequence(A.n)
    x, st = s.solve(A, b, 1e-15, O.make_policy("srks", "block_jacobi3", ritz_eps=1e-10, max_iter=A.n))
    assert st["status"] in (0, 3)
    alpha, rho, _ = s.coeffs()
    delta, eta = O.lanczos(alpha, rho)
    th = O.tridiag_eig(delta, eta, vectors=False)
    ev = sla.eigh(Ad, M, eigvals_only=True)[::-1]
    distinct = [ev[0]]
    for e in ev[1:]:
        if abs(e - distinct[-1]) > 1e-8 * ev[0]:
            distinct.append(e)
    # CG terminates after as many steps as M^-1 A has distinct eigenvalues (the clamped
    # one-element cube has three double eigenvalues), and the Ritz values are those values
    assert s.m == len(distinct)
    assert np.allclose(th, distinct, rtol=1e-8)


def test_srks_diagonal_selects_scaled_eigenvectors():
    """Diagonal A, M = I, distinct eigenvalues: each selected vector is +-e_k / sqrt(lambda_k)."""
    n = 30
    lam = np.concatenate([[0.01, 0.02, 0.05], np.linspace(1.0, 2.0, n - 6), [20.0, 40.0, 80.0]])
    A = dense_bsr(np.diag(lam))
    b = np.ones(n)
    s = O.Sequence(n)
    x, st = s.solve(A, b, 1e-12, O.make_policy("srks", "identity", ritz_eps=1e-12))
    tm, tm1, sel, Y = s.ritz()
    assert len(sel) >= 3
    for c in range(len(sel)):
        y = Y[:, c]
        k = int(np.argmax(np.abs(y)))
        assert abs(tm[sel[c]] - lam[k]) <= 1e-9 * lam[k]
        e = np.zeros(n)
        e[k] = np.sign(y[k]) / math.sqrt(lam[k])
        assert np.linalg.norm(y - e) <= 1e-5 * np.linalg.norm(e)


def test_srks_theta_frac_and_cap():
    A, b = small_problem(3, seed=23)
    s = O.Sequence(A.n)
    x, st = s.solve(A, b, 1e-10, O.make_policy("srks", "block_jacobi3", ritz_eps=1e-8, theta_frac=0.1))
    tm, tm1, sel, Y = s.ritz()
    assert np.all(tm[sel] < 0.1 * tm[0])
    s2 = O.Sequence(A.n)
    s2.solve(A, b, 1e-10, O.make_policy("srks", "block_jacobi3", ritz_eps=1e-8, max_aug=2))
    assert s2.nc == min(2, st["n_selected"] if st["n_selected"] else 2) or s2.nc <= 2


def test_srks_restart_mode_resets_to_C0():
    A, b = small_problem(2, seed=24)
    s = O.Sequence(A.n)
    C0 = np.random.default_rng(10).standard_normal((A.n, 2))
    s.set_C(C0, as_c0=True)
    pol = O.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, max_aug=3, cap_mode="restart")
    x, st = s.solve(A, b, 1e-10, pol)
    assert st["n_selected"] >= 1
    assert s.nc == 2 and np.array_equal(s.C, C0)


# ----------------------------------------------------------------------------------------
# failure statuses
# ----------------------------------------------------------------------------------------

def test_status_not_spd_matrix():
    A, b = small_problem(2, seed=25)
    A.vals[A.row_ptr[0]:A.row_ptr[1]][list(A.col_idx[A.row_ptr[0]:A.row_ptr[1]]).index(0)] *= -1
    s, x, st = run(A, b, 1e-8, precond="jacobi")
    assert st["status"] == O.ERR_NOT_SPD


def test_status_rank_deficient_C():
    n = 12
    lam = np.arange(1.0, n + 1)
    lam[0] = 4.0
    A = dense_bsr(np.diag(lam))
    C = np.zeros((n, 2))
    C[0, 0] = C[0, 1] = 1.0  # duplicated column, exact arithmetic: G = [[4, 4], [4, 4]]
    s, x, st = run(A, np.ones(n), 1e-8, C=C, precond="identity")
    assert st["status"] == O.ERR_NOT_SPD
    C2 = np.zeros((n, 2))
    C2[1, 0] = 1.0
    s2, x2, st2 = run(A, np.ones(n), 1e-8, C=C2, precond="identity")
    assert st2["status"] == O.ERR_NOT_SPD


def test_status_nan_rhs_and_no_convergence_keeps_C():
    A, b = small_problem(2, seed=26)
    bn = b.copy()
    bn[3] = np.nan
    s, x, st = run(A, bn, 1e-8)
    assert st["status"] == O.ERR_INVALID_ARG
    s = O.Sequence(A.n)
    pol = O.make_policy("trks", "jacobi")
    s.solve(A, b, 1e-6, pol)
    C_before = s.C.copy()
    x, st = s.solve(A, P.traction_rhs(2, P.random_traction(2, 9)), 1e-14,
                    O.make_policy("trks", "jacobi", max_iter=2))
    assert st["status"] == O.ERR_NO_CONVERGENCE
    assert np.array_equal(s.C, C_before)


def test_zero_rhs():
    A, b = small_problem(2, seed=27)
    s, x, st = run(A, np.zeros(A.n), 1e-8)
    assert st["status"] == 0 and st["m"] == 0 and np.all(x == 0)


# ----------------------------------------------------------------------------------------
# Cluster reselection (Section 4.4, end): three-piece least-squares fit of the gaps
# ----------------------------------------------------------------------------------------

def _brute_cluster(v):
    """Every three-piece split of the gap sequence, fitted by its piece means, in plain
    numpy; returns the keep mask the reading prescribes (drop the central piece's values
    when it is strictly denser than every non-empty outer piece)."""
    v = np.asarray(v, dtype=float)
    s = v.size
    keep = np.ones(s, dtype=bool)
    if s < 3:
        return keep
    d = np.diff(v)
    ng = d.size
    minsize = max(2, -(-s // 5))
    best = None
    for a in range(ng):
        for b in range(a, ng):
            if b - a + 2 < minsize:
                continue
            pieces = [d[:a], d[a:b + 1], d[b + 1:]]
            err = sum(float(((p - p.mean()) ** 2).sum()) if p.size else 0.0 for p in pieces)
            if best is None or err < best[0]:
                best = (err, a, b, [p.mean() if p.size else None for p in pieces])
    _, a, b, (m0, m1, m2) = best
    outer = [m for m in (m0, m2) if m is not None]
    if outer and all(m1 < m for m in outer):
        keep[a:b + 2] = False
    return keep


def test_cluster_hand_example():
    """Values with a dense run in the middle (gaps 0.1) between sparse ends (gaps 1): the
    three-piece fit is exact and the run 2.0 .. 2.5 is the central cluster."""
    v = [0.0, 1.0, 2.0, 2.1, 2.2, 2.3, 2.4, 2.5, 3.5, 4.5]
    keep = O.cluster_reselect(v)
    assert keep.tolist() == [True, True, False, False, False, False, False, False, True, True]


def test_cluster_uniform_and_small():
    """Evenly spaced values have no denser piece: nothing is dropped; fewer than three
    values are never touched."""
    assert O.cluster_reselect(np.arange(12.0)).all()
    assert O.cluster_reselect([1.0, 2.0]).all()
    assert O.cluster_reselect([]).size == 0


def test_cluster_matches_brute_force_and_invariants():
    rng = np.random.Generator(np.random.PCG64(77))
    for trial in range(60):
        s = int(rng.integers(3, 13))
        gaps = rng.uniform(0.5, 2.0, s - 1)
        if trial % 2 == 0 and s >= 5:  # plant a dense run
            a = int(rng.integers(0, s - 3))
            L = int(rng.integers(2, s - a))
            gaps[a:a + L - 1] *= 0.01
        v = np.concatenate([[0.0], np.cumsum(gaps)])
        keep = O.cluster_reselect(v)
        assert keep.tolist() == _brute_cluster(v).tolist(), (trial, v)
        dropped = np.flatnonzero(~keep)
        if dropped.size:
            assert np.all(np.diff(dropped) == 1)              # one contiguous run
            assert dropped.size >= max(2, -(-s // 5))         # minimum cluster size
            assert keep.any()                                 # an outer piece survives


def test_srks_select_with_cluster_reselection():
    """theta_{m-1} = the first m-1 values of theta_m: Eq. 16's first test preselects
    indices 0..m-2 (ascending: 2.0, 3.0 .. 3.5, 4.5, 5.5); reselection drops the dense run
    3.0 .. 3.5 (gaps 0.1 between gaps of 1.0); the result is in ascending theta order and
    the cap applies after reselection."""
    vals_desc = np.array([4.5, 3.5, 2.5, 2.4, 2.3, 2.2, 2.1, 2.0, 1.0, 0.0]) + 1.0
    tm1 = vals_desc[:-1].copy()
    sel_all = O.srks_select(vals_desc, tm1, 1e-12)
    assert sel_all.tolist() == list(range(8, -1, -1))
    sel = O.srks_select(vals_desc, tm1, 1e-12, reselect=1)
    assert sel.tolist() == [8, 1, 0]
    assert O.srks_select(vals_desc, tm1, 1e-12, reselect=1, room=2).tolist() == [8, 1]
