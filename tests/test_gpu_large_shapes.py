"""Parity on the shapes of the largest single sequence (the 64^3 stiff-inclusion cube,
811,200 dofs, augmentation size up to 300, thousands of stored directions).

At these sizes every CTA of the iteration owns more than one staging chunk of rows (2,048),
which sends the FP64 tall-skinny product V^T u to its warp-block layout at any width --
the branch the small cases never reach.  Checked here, through the C ABI:
  * krs_gemv_t / krs_gemv_n_sub at 400,000 rows (2,632 rows per row block) with 17, 300 and
    1,100 columns, and at 811,200 rows (5,340 rows per block) with 300 columns, against
    numpy in FP64 (rounding bound of the dot products);
  * a whole APCG solve (Algorithm 1 with full reorthogonalisation, Section 2.1 remark) on
    the 48^3 inclusion cube (345,744 dofs, 2,280 rows per CTA) with an imported full-rank
    augmentation space of 300 columns, 40 iterations on both sides, in FP64 and in the
    double-float precision: the 40th iterates agree to the lock-step bar (1e-9 relative).
"""
import numpy as np
import pytest

import oracle as O
from paper_1301_7530_gb300 import binding as B
from paper_1301_7530_gb300 import problems as P

from .lockstep import SOL_TOL, rel

pytestmark = pytest.mark.gpu


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n,k", [(400000, 17), (400000, 300), (400000, 1100), (811200, 300)])
def test_tall_skinny_large_rows_per_block(gpu_lib, n, k):
    import torch
    rng = np.random.default_rng(7 * n + k)
    ld = (n + 31) // 32 * 32
    V = np.zeros((k, ld))
    V[:, :n] = rng.random((k, n)) - 0.5
    u = np.zeros(ld)
    u[:n] = rng.random(n) - 0.5
    s = rng.random(k) - 0.5
    Vd = torch.as_tensor(V, device="cuda")
    ud = torch.as_tensor(u, device="cuda")
    sd = torch.as_tensor(s, device="cuda")
    td = torch.zeros(k, device="cuda", dtype=torch.float64)
    zd = torch.zeros(ld, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_gemv_t(n, k, Vd.data_ptr(), ld, ud.data_ptr(), td.data_ptr(), _stream()) == 0
    assert gpu_lib.krs_gemv_n_sub(n, k, Vd.data_ptr(), ld, sd.data_ptr(), ud.data_ptr(), zd.data_ptr(),
                                  _stream()) == 0
    torch.cuda.synchronize()
    t, z = td.cpu().numpy(), zd.cpu().numpy()
    Vn = V[:, :n]
    t_ref = Vn @ u[:n]
    z_ref = u[:n] - Vn.T @ s
    bound_t = 1e-15 * np.sqrt(n) * (np.abs(Vn) @ np.abs(u[:n])) * 8
    bound_z = 1e-15 * np.sqrt(k) * (np.abs(Vn.T) @ np.abs(s) + np.abs(u[:n])) * 8
    assert np.all(np.abs(t - t_ref) <= bound_t), np.max(np.abs(t - t_ref) / bound_t)
    assert np.all(np.abs(z[:n] - z_ref) <= bound_z), np.max(np.abs(z[:n] - z_ref) / bound_z)
    assert np.all(z[n:] == 0.0)


N48 = 48
NC48 = 300
ITERS48 = 40


@pytest.fixture(scope="module")
def cube48():
    """48^3 inclusion cube, one traction right-hand side, a seeded full-rank space of 300
    columns, and the oracle's 40th iterate from that space."""
    A = P.elasticity_inclusions(N48, 3000)
    b = P.traction_rhs(N48, P.random_traction(N48, 3100))
    rng = np.random.default_rng(4848)
    C = rng.random((A.n, NC48)) - 0.5
    ora = O.Sequence(A.n)
    ora.set_C(C)
    xo, so = ora.solve(A, b, 1e-8, O.make_policy("none", "block_jacobi3", max_iter=ITERS48))
    return A, b, C, xo, so


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
def test_lockstep_48cube_imported_space(gpu_lib, cube48, precision):
    A, b, C, xo, so = cube48
    assert so["status"] == O.ERR_NO_CONVERGENCE and so["m"] == ITERS48
    seq = B.Sequence(A.n)
    seq.import_space(C)
    pol = B.make_policy("none", "block_jacobi3", max_iter=ITERS48, precision=precision)
    x, st = seq.solve(A, b, 1e-8, pol, version=1, raise_on_error=False)
    assert st["status"] == B.ERR_NO_CONVERGENCE and st["m"] == ITERS48, st
    err = rel(x, xo)
    assert err <= SOL_TOL, err
    # the iterate satisfies the projection's Galerkin condition C^T r = 0 (Eq. 5)
    r = b - A.to_scipy() @ x
    assert np.abs(C.T @ r).max() <= 1e-9 * np.linalg.norm(C, axis=0).max() * np.linalg.norm(b)
    seq.close()
