"""Single kernels through the C ABI against the oracle / numpy on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O
from paper_1301_7530_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("N", [1, 3, 5, 9])
def test_spmv_vs_oracle(gpu_lib, N):
    import torch
    rng = np.random.default_rng(N)
    A = P.assemble(N, rng.uniform(0.5, 2.0, size=(N, N, N)))
    x = rng.standard_normal(A.n)
    rp, ci, v = _dev(A.row_ptr), _dev(A.col_idx), _dev(A.vals)
    xd, yd = _dev(x), torch.zeros(A.n, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_spmv_bsr3(A.n_block_rows, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), xd.data_ptr(),
                                 yd.data_ptr(), _stream()) == 0
    y = _np(yd)
    yo = O.spmv(A, x)
    scale = np.abs(A.vals).max() * np.abs(x).max() * 81
    assert np.abs(y - yo).max() <= 1e-15 * scale


@pytest.mark.parametrize("kind", ["jacobi", "block_jacobi3", "identity"])
def test_precond_vs_oracle(gpu_lib, kind):
    import torch
    rng = np.random.default_rng(3)
    N = 4
    A = P.assemble(N, rng.uniform(0.5, 2.0, size=(N, N, N)))
    k = {"jacobi": 0, "block_jacobi3": 1, "identity": 2}[kind]
    rp, ci, v = _dev(A.row_ptr), _dev(A.col_idx), _dev(A.vals)
    minv = torch.zeros(9 * A.n_block_rows, device="cuda", dtype=torch.float64)
    st = torch.zeros(1, device="cuda", dtype=torch.int32)
    assert gpu_lib.krs_precond_setup(k, A.n_block_rows, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), minv.data_ptr(),
                                     st.data_ptr(), _stream()) == 0
    r = rng.standard_normal(A.n)
    rd, ud = _dev(r), torch.zeros(A.n, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_precond_apply(k, A.n_block_rows, minv.data_ptr(), rd.data_ptr(), ud.data_ptr(), _stream()) == 0
    assert int(_np(st)[0]) == 0
    uo = O.precond_apply(kind, A.n_block_rows, O.precond_setup(A, kind), r)
    assert np.allclose(_np(ud), uo, rtol=1e-13, atol=1e-15)


def test_precond_detects_non_spd_block(gpu_lib):
    import torch
    A = P.assemble(2, P.uniform_modulus(2))
    i = list(A.col_idx[A.row_ptr[1]:A.row_ptr[2]]).index(1)
    A.vals[A.row_ptr[1] + i] *= -1.0
    rp, ci, v = _dev(A.row_ptr), _dev(A.col_idx), _dev(A.vals)
    minv = torch.zeros(9 * A.n_block_rows, device="cuda", dtype=torch.float64)
    st = torch.zeros(1, device="cuda", dtype=torch.int32)
    gpu_lib.krs_precond_setup(1, A.n_block_rows, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), minv.data_ptr(),
                              st.data_ptr(), _stream())
    assert int(_np(st)[0]) == 2


@pytest.mark.parametrize("n,k", [(1, 1), (7, 3), (1003, 37), (20000, 300), (12345, 1100)])
def test_tall_skinny_vs_numpy(gpu_lib, n, k):
    import torch
    rng = np.random.default_rng(n + k)
    ld = (n + 31) // 32 * 32
    V = np.zeros((k, ld))
    V[:, :n] = rng.standard_normal((k, n))
    u = np.zeros(ld)
    u[:n] = rng.standard_normal(n)
    s = rng.standard_normal(k)
    Vd, ud, sd = _dev(V), _dev(u), _dev(s)
    td = torch.zeros(k, device="cuda", dtype=torch.float64)
    zd = torch.zeros(ld, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_gemv_t(n, k, Vd.data_ptr(), ld, ud.data_ptr(), td.data_ptr(), _stream()) == 0
    assert gpu_lib.krs_gemv_n_sub(n, k, Vd.data_ptr(), ld, sd.data_ptr(), ud.data_ptr(), zd.data_ptr(), _stream()) == 0
    Vn = V[:, :n]
    t_ref = Vn @ u[:n]
    z_ref = u[:n] - Vn.T @ s
    bound_t = 1e-15 * np.sqrt(n) * (np.abs(Vn) @ np.abs(u[:n])) * 8 + 1e-300
    assert np.all(np.abs(_np(td) - t_ref) <= bound_t)
    bound_z = 1e-15 * np.sqrt(k) * (np.abs(Vn.T) @ np.abs(s) + np.abs(u[:n])) * 8
    z = _np(zd)
    assert np.all(np.abs(z[:n] - z_ref) <= bound_z)
    assert np.all(z[n:] == 0.0)  # padding untouched


def test_tall_skinny_rejects_bad_layout(gpu_lib):
    import torch
    V = torch.zeros(64, device="cuda", dtype=torch.float64)
    t = torch.zeros(2, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_gemv_t(30, 2, V.data_ptr(), 30, V.data_ptr(), t.data_ptr(), _stream()) == 1
    assert gpu_lib.krs_gemv_t(30, 2, V.data_ptr() + 8, 32, V.data_ptr(), t.data_ptr(), _stream()) == 1


def test_axpy2_dot(gpu_lib):
    import torch
    rng = np.random.default_rng(4)
    n = 5000
    w, q, x, r = (rng.standard_normal(n) for _ in range(4))
    al = np.array([0.37])
    wd, qd, xd, rd, ad = _dev(w), _dev(q), _dev(x), _dev(r), _dev(al)
    rr = torch.zeros(1, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_axpy2_dot(n, ad.data_ptr(), wd.data_ptr(), qd.data_ptr(), xd.data_ptr(), rd.data_ptr(),
                                 rr.data_ptr(), _stream()) == 0
    xr, rr_ref = x + 0.37 * w, r - 0.37 * q
    assert np.allclose(_np(xd), xr, rtol=1e-15, atol=1e-15)
    assert np.allclose(_np(rd), rr_ref, rtol=1e-15, atol=1e-15)
    assert abs(_np(rr)[0] - rr_ref @ rr_ref) <= 1e-13 * (rr_ref @ rr_ref)


@pytest.mark.parametrize("m", [1, 2, 9, 64, 333, 15000])
def test_tridiag_eigvals_closed_form(gpu_lib, m):
    """tridiag(1, 2, 1): eigenvalues 2 + 2 cos(k pi / (m + 1)).  m = 15000 is too long for the
    matrix to be staged in shared memory (the bisection reads it from global memory)."""
    import torch
    d, e = _dev(np.full(m, 2.0)), _dev(np.ones(max(m - 1, 1)))
    th = torch.zeros(m, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_tridiag_eigvals(m, d.data_ptr(), e.data_ptr(), th.data_ptr(), _stream()) == 0
    k = np.arange(1, m + 1)
    exact = 2.0 + 2.0 * np.cos(k * np.pi / (m + 1))
    assert np.allclose(_np(th), exact, atol=4e-15 * 4)


def _lanczos_like(m, seed):
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(0.2, 3.0, m)
    rho = np.cumprod(rng.uniform(0.3, 1.2, m))
    return O.lanczos(alpha, rho)


@pytest.mark.parametrize("m", [5, 80, 400])
def test_tridiag_eig_vs_oracle(gpu_lib, m):
    import torch
    delta, eta = _lanczos_like(m, m)
    th_o, Q_o = O.tridiag_eig(delta, eta)
    d, e = _dev(delta), _dev(eta if m > 1 else np.zeros(1))
    th = torch.zeros(m, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_tridiag_eigvals(m, d.data_ptr(), e.data_ptr(), th.data_ptr(), _stream()) == 0
    thg = _np(th)
    assert np.allclose(thg, th_o, atol=8 * 2.2e-16 * np.abs(th_o).max())
    # eigenvectors of a few values, ascending, against the oracle's (sign-normalised)
    pick = sorted(set([m - 1, m - 2, m // 2, 0]))[: min(4, m)]
    pick = sorted(pick, key=lambda i: th_o[i])
    ts = _dev(np.array([thg[i] for i in pick]))
    Qd = torch.zeros(len(pick) * m, device="cuda", dtype=torch.float64)
    assert gpu_lib.krs_tridiag_eigvecs(m, d.data_ptr(), e.data_ptr(), len(pick), ts.data_ptr(), Qd.data_ptr(),
                                       _stream()) == 0
    Qg = _np(Qd).reshape(len(pick), m)
    gaps = np.diff(np.sort(th_o))
    for c, i in enumerate(pick):
        q = Q_o[:, i].copy()
        q *= np.sign(q[np.argmax(np.abs(q))])
        others = np.abs(th_o - th_o[i])
        others[i] = np.inf
        gap = others.min()
        tol = 1e-13 * np.abs(th_o).max() / gap * 10 + 1e-12
        assert np.linalg.norm(Qg[c] - q) <= tol, (i, gap)
