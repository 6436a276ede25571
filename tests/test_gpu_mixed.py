"""Mixed-precision refinement (KRS_MIXED_IR): FP32 inner APCG with FP64 outer residuals,
FP64 coarse Cholesky and eigensolve.  Parity is stated per result as the error against the
FP64 oracle's solution (no iteration-count requirement): the FP64 outer residual bounds
the error by kappa(A) * tol."""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1301_7530_gb300 import binding as B
from paper_1301_7530_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _exact(A, b):
    """Reference solution by a dense Cholesky solve (library routine, tiny systems)."""
    return sla.cho_solve(sla.cho_factor(A.to_dense()), b)


def _kappa(A):
    ev = np.linalg.eigvalsh(A.to_dense())
    return ev[-1] / ev[0]


@pytest.mark.parametrize("recycle", ["none", "trks", "srks"])
def test_mixed_sequence_error_against_oracle(gpu_lib, recycle):
    """6^3 cube with stiff inclusions (contrast 1e3), 4 systems, tol 1e-8."""
    N = 6
    A = P.elasticity_inclusions(N, 3, fraction=0.05)
    kap = _kappa(A)
    seq = B.Sequence(A.n)
    pol = B.make_policy(recycle, "block_jacobi3", precision="mixed_ir", ritz_eps=1e-6, theta_frac=0.5, max_aug=80)
    m_first = []
    for k in range(4):
        b = P.traction_rhs(N, P.random_traction(N, 3000 + k))
        x, st = seq.solve(A, b, 1e-8, pol, version=1)
        assert st["status"] == 0, st
        assert st["true_rel_res"] <= 1e-8
        assert st["outer_iters"] >= 1
        xe = _exact(A, b)
        err = np.linalg.norm(x - xe) / np.linalg.norm(xe)
        assert err <= kap * 1e-8, (err, kap)
        m_first.append(st["inner_m_first"])
        if recycle != "none":
            assert st["n_c_after"] >= st["n_c"]
    if recycle == "trks":
        assert m_first[-1] < m_first[0]


def test_mixed_srks_vectors_are_A_normalised(gpu_lib):
    """Selected Ritz vectors from the first inner solve, scaled by 1/sqrt(theta): their
    A-Gram matrix is close to the identity (exactly I for exact Ritz pairs; the FP32 inner
    solve perturbs it at the FP32 level)."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 3, 4, 2000)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("srks", "block_jacobi3", precision="mixed_ir", ritz_eps=1e-5, theta_frac=0.3, max_aug=60)
    for k, Ak in gen:
        nc0 = seq.nc
        x, st = seq.solve(Ak, b, 1e-8, pol, version=k + 1)
        assert st["status"] == 0 and st["true_rel_res"] <= 1e-8
        if st["n_selected"]:
            Y = seq.export_space()[:, nc0:]
            G = Y.T @ (Ak.to_scipy() @ Y)
            assert np.abs(G - np.eye(G.shape[0])).max() <= 2e-3


def test_mixed_exec_modes_bitwise_equal(gpu_lib):
    N = 5
    A = P.elasticity_inclusions(N, 8, fraction=0.05)
    b = P.traction_rhs(N, P.random_traction(N, 5))
    xs = []
    for mode in ("persistent", "kernels"):
        seq = B.Sequence(A.n)
        pol = B.make_policy("srks", "block_jacobi3", precision="mixed_ir", ritz_eps=1e-5, exec=mode)
        out = []
        for k in range(2):
            x, st = seq.solve(A, b * (1.0 + k), 1e-9, pol, version=1)
            out.append((x.copy(), st["m"], st["outer_iters"]))
        xs.append((out, seq.export_space()))
    for (xa, ma, oa), (xb, mb, ob) in zip(xs[0][0], xs[1][0]):
        assert ma == mb and oa == ob and np.array_equal(xa, xb)
    assert np.array_equal(xs[0][1], xs[1][1])


def test_mixed_fp64_equivalence_of_outer_residual(gpu_lib):
    """The reported true residual is the FP64 ||b - A x|| / ||b||, recomputed here."""
    N = 7
    A = P.elasticity_inclusions(N, 11, fraction=0.05)
    b = P.traction_rhs(N, P.random_traction(N, 21))
    x, st = B.Sequence(A.n).solve(A, b, 1e-9, B.make_policy("none", "block_jacobi3", precision="mixed_ir"), version=1)
    r = b - A.to_scipy() @ x
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - st["true_rel_res"]) <= 1e-12
    assert st["true_rel_res"] <= 1e-9


def test_mixed_no_convergence_keeps_space(gpu_lib):
    N = 5
    A = P.elasticity_inclusions(N, 2, fraction=0.05)
    b = P.traction_rhs(N, P.random_traction(N, 1))
    seq = B.Sequence(A.n)
    seq.solve(A, b, 1e-6, B.make_policy("trks", "block_jacobi3", precision="mixed_ir"), version=1)
    C0 = seq.export_space()
    x, st = seq.solve(A, 2 * b + 1e-3, 1e-14, B.make_policy("trks", "block_jacobi3", precision="mixed_ir", max_outer=1),
                      version=1, raise_on_error=False)
    assert st["status"] == B.ERR_NO_CONVERGENCE
    assert np.array_equal(seq.export_space(), C0)


@pytest.mark.parametrize("N", [16, 32])
def test_mixed_refinement_on_stiff_inclusion_cube(gpu_lib, N):
    """Stiff inclusions (contrast 1e3) make kappa(A) u_32 large enough that plain iterative
    refinement (x += d) stalls; the flexible CG over the FP32 corrections converges to the FP64
    tolerance, and its result is as close to the tight FP64 solution as an FP64 solve at the
    same tolerance is (error of each against an FP64 solve to 1e-11, whose own parity with the
    oracle the FP64 tests establish)."""
    A = P.elasticity_inclusions(N, 3000)
    b = P.traction_rhs(N, P.random_traction(N, 3100))
    ref, st_ref = B.Sequence(A.n).solve(A, b, 1e-11, B.make_policy("none", "block_jacobi3", max_iter=12000),
                                        version=1)
    x64, st64 = B.Sequence(A.n).solve(A, b, 1e-8, B.make_policy("none", "block_jacobi3", max_iter=12000), version=1)
    seq = B.Sequence(A.n)
    x, st = seq.solve(A, b, 1e-8, B.make_policy("none", "block_jacobi3", precision="mixed_ir", max_iter=16000),
                      version=1, raise_on_error=False)
    assert st["status"] == 0, st
    assert st["true_rel_res"] <= 1e-8
    e_mixed = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    e_fp64 = np.linalg.norm(x64 - ref) / np.linalg.norm(ref)
    assert e_mixed <= 10 * e_fp64 + 1e-12, (e_mixed, e_fp64, st["outer_iters"], st["m"])
