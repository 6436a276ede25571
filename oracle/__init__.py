"""FP64 CPU oracle for augmented PCG with Krylov-subspace recycling (TRKS / SRKS).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are the only callers.  The product path (``paper_1301_7530_gb300``) never
imports this package.  The arithmetic lives in ``krs_oracle.c`` (plain C, FP64, evaluated
as written); this module only compiles it with gcc and marshals numpy arrays.

Two builds of the same file: ``liborc.so`` (the parity oracle, sequential sums) and
``liborc_omp.so`` (``-fopenmp``: the long loops split across host threads), which only the
benchmark's CPU baseline loads (``omp=True``) to time the oracle on all host cores.

Parity status of each function (what pins it; the pins live under tests/):
  spmv, precond            -- dense products on tiny meshes, block inverse identity
  cholesky / chol_solve    -- numpy.linalg.cholesky / solve (library references)
  lanczos                  -- V^T A V = H_m with V built from the solve's Z (any size)
  sym_eig / tridiag_eig    -- numpy.linalg.eigh (library reference), orthonormality
  srks_select              -- hand-built (theta_m, theta_{m-1}) arrays with known sets
  cluster_reselect         -- hand-worked gap sequences, evenly spaced values, and an
                              exhaustive three-piece least-squares fit written in numpy
                              on random tiny inputs (Section 4.4, end)
  Sequence.solve           -- dense Cholesky solution, textbook CG/PCG written in the test,
                              C^T r = 0, A-conjugacy, finite termination, Proposition 1 /
                              Corollary 1 / Proposition 2 reductions, TRKS m = 0 case,
                              Ritz Y^T A Y = Theta, deflation closed form.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "krs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liborc_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

OK, ERR_INVALID_ARG, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_OOM = 0, 1, 2, 3, 4
RECYCLE = {"none": 0, "trks": 1, "srks": 2}
PRECOND = {"jacobi": 0, "block_jacobi3": 1, "identity": 2}
REORTH = {"full": 0, "none": 1}
CAP = {"truncate": 0, "restart": 1}


class Policy(ct.Structure):
    _fields_ = [("recycle", ct.c_int32), ("precond", ct.c_int32), ("reorth", ct.c_int32),
                ("cap_mode", ct.c_int32), ("max_aug", ct.c_int32), ("max_iter", ct.c_int32),
                ("ritz_eps", ct.c_double), ("theta_frac", ct.c_double),
                ("reselect", ct.c_int32), ("pad", ct.c_int32)]


class Stats(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("m", ct.c_int32), ("n_c", ct.c_int32),
                ("n_selected", ct.c_int32), ("n_c_after", ct.c_int32),
                ("rel_res", ct.c_double), ("true_rel_res", ct.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _compile(path: str, extra, force: bool) -> str:
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            return path
        tmp = path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True)
        os.replace(tmp, path)
        return path


def build(force: bool = False) -> str:
    """Compile krs_oracle.c with gcc into oracle/_build/liborc.so (the parity oracle) and,
    when the compiler supports OpenMP, oracle/_build/liborc_omp.so (the timing build)."""
    path = _compile(_LIB_PATH, [], force)
    try:
        _compile(_LIB_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass  # the timing build is optional; build_omp() raises the reason
    return path


def build_omp(force: bool = False) -> str:
    """The OpenMP timing build (raises when the compiler cannot build it)."""
    return _compile(_LIB_OMP_PATH, ["-fopenmp"], force)


def lib(omp: bool = False):
    """The parity oracle (omp=False) or the OpenMP timing build (omp=True)."""
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = _declare(ct.CDLL(build_omp()))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ct.CDLL(build()))
    return _lib


def _declare(L):
    """Argument types of the library's functions."""
    dp, ip = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int32)
    L.orc_spmv.argtypes = [ct.c_int, ip, ip, dp, dp, dp]
    L.orc_precond_setup.argtypes = [ct.c_int, ct.c_int, ip, ip, dp, dp]
    L.orc_precond_apply.argtypes = [ct.c_int, ct.c_int, dp, dp, dp]
    L.orc_cholesky.argtypes = [ct.c_int, dp]
    L.orc_chol_solve.argtypes = [ct.c_int, dp, dp]
    L.orc_lanczos.argtypes = [ct.c_int, dp, dp, dp, dp]
    L.orc_sym_eig.argtypes = [ct.c_int, dp, dp, dp]
    L.orc_tridiag_eig.argtypes = [ct.c_int, dp, dp, dp, dp]
    L.orc_srks_select.argtypes = [ct.c_int, dp, dp, ct.c_double, ct.c_double, ct.c_int, ip]
    L.orc_srks_select2.argtypes = [ct.c_int, dp, dp, ct.c_double, ct.c_double, ct.c_int, ct.c_int, ip]
    L.orc_cluster_reselect.argtypes = [ct.c_int, dp, ip]
    L.orc_cluster_reselect.restype = None
    L.orc_seq_create.argtypes = [ct.c_int64]
    L.orc_seq_create.restype = ct.c_void_p
    L.orc_seq_destroy.argtypes = [ct.c_void_p]
    for f in ("orc_seq_nc", "orc_seq_m", "orc_seq_nsel"):
        getattr(L, f).argtypes = [ct.c_void_p]
    L.orc_seq_get_C.argtypes = [ct.c_void_p, dp]
    L.orc_seq_set_C.argtypes = [ct.c_void_p, ct.c_int, dp, ct.c_int]
    L.orc_seq_get_W.argtypes = [ct.c_void_p, dp]
    L.orc_seq_get_AW.argtypes = [ct.c_void_p, dp]
    L.orc_seq_get_Z.argtypes = [ct.c_void_p, dp]
    L.orc_seq_get_coeffs.argtypes = [ct.c_void_p, dp, dp, dp]
    L.orc_seq_get_ritz.argtypes = [ct.c_void_p, dp, dp, ip, dp]
    L.orc_seq_solve.argtypes = [ct.c_void_p, ct.c_int, ip, ip, dp, dp, dp, ct.c_double,
                                ct.POINTER(Policy), ct.POINTER(Stats)]
    L.orc_seq_get_times.argtypes = [ct.c_void_p, dp]
    L.orc_num_threads.argtypes = []
    return L


def num_threads(omp: bool = False) -> int:
    """Host threads the build's loops use (1 for the parity build)."""
    return int(lib(omp).orc_num_threads())


def _d(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _i(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _bsr_args(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.vals, dtype=np.float64)
    return rp, ci, v


def spmv(A, x, omp: bool = False):
    rp, ci, v = _bsr_args(A)
    x = _f64(x)
    y = np.empty(A.n)
    lib(omp).orc_spmv(A.n_block_rows, _i(rp), _i(ci), _d(v), _d(x), _d(y))
    return y


def precond_setup(A, kind: str):
    rp, ci, v = _bsr_args(A)
    out = np.zeros(9 * A.n_block_rows)
    st = lib().orc_precond_setup(PRECOND[kind], A.n_block_rows, _i(rp), _i(ci), _d(v), _d(out))
    if st:
        raise RuntimeError(f"precond setup status {st}")
    return out


def precond_apply(kind: str, nbr: int, minv, r):
    r = _f64(r)
    u = np.empty_like(r)
    lib().orc_precond_apply(PRECOND[kind], nbr, _d(_f64(minv)), _d(r), _d(u))
    return u


def cholesky(G):
    """Lower Cholesky factor (raises on failure)."""
    m = G.shape[0]
    a = np.asfortranarray(G, dtype=np.float64).copy(order="F")
    st = lib().orc_cholesky(m, a.ctypes.data_as(ct.POINTER(ct.c_double)))
    if st:
        raise np.linalg.LinAlgError("not SPD")
    return np.tril(a)


def chol_solve(L, y):
    m = L.shape[0]
    a = np.asfortranarray(L, dtype=np.float64).copy(order="F")
    y = _f64(y).copy()
    lib().orc_chol_solve(m, a.ctypes.data_as(ct.POINTER(ct.c_double)), _d(y))
    return y


def lanczos(alpha, rho):
    alpha, rho = _f64(alpha), _f64(rho)
    m = alpha.shape[0]
    delta = np.empty(m)
    eta = np.empty(max(m, 1))
    lib().orc_lanczos(m, _d(alpha), _d(rho), _d(delta), _d(eta))
    return delta, eta[:max(m - 1, 0)]


def sym_eig(S):
    """Eigenvalues (descending) and eigenvectors of a dense symmetric matrix."""
    m = S.shape[0]
    a = np.asfortranarray(S, dtype=np.float64).copy(order="F")
    th = np.empty(m)
    Q = np.empty((m, m), order="F")
    st = lib().orc_sym_eig(m, a.ctypes.data_as(ct.POINTER(ct.c_double)), _d(th),
                           Q.ctypes.data_as(ct.POINTER(ct.c_double)))
    if st:
        raise MemoryError
    return th, np.asarray(Q)


def tridiag_eig(delta, eta, vectors=True, omp: bool = False):
    delta, eta = _f64(delta), _f64(eta)
    m = delta.shape[0]
    th = np.empty(m)
    Q = np.empty((m, m), order="F") if vectors else None
    e = eta if eta.size else np.zeros(1)
    lib(omp).orc_tridiag_eig(m, _d(delta), _d(e), _d(th),
                          Q.ctypes.data_as(ct.POINTER(ct.c_double)) if vectors else None)
    return (th, np.asarray(Q)) if vectors else th


def srks_select(theta_m, theta_m1, eps, theta_frac=0.0, room=1 << 30, reselect=0):
    theta_m, theta_m1 = _f64(theta_m), _f64(theta_m1)
    m = theta_m.shape[0]
    out = np.zeros(max(m, 1), dtype=np.int32)
    t1 = theta_m1 if theta_m1.size else np.zeros(1)
    cnt = lib().orc_srks_select2(m, _d(theta_m), _d(t1), float(eps), float(theta_frac), int(reselect),
                                 int(min(room, 1 << 30)), _i(out))
    return out[:cnt].copy()


def cluster_reselect(values):
    """keep mask of cluster reselection on ascending values (Section 4.4, end)."""
    v = _f64(values)
    keep = np.ones(max(v.shape[0], 1), dtype=np.int32)
    lib().orc_cluster_reselect(int(v.shape[0]), _d(v), _i(keep))
    return keep[:v.shape[0]].astype(bool)


def make_policy(recycle="none", precond="jacobi", reorth="full", cap_mode="truncate",
                max_aug=0, max_iter=5000, ritz_eps=1e-14, theta_frac=0.0, reselect="none") -> Policy:
    return Policy(RECYCLE[recycle], PRECOND[precond], REORTH[reorth], CAP[cap_mode],
                  int(max_aug), int(max_iter), float(ritz_eps), float(theta_frac),
                  {"none": 0, "cluster": 1}[reselect], 0)


class Sequence:
    """Oracle sequence state: the augmentation basis C and the last solve's internals."""

    def __init__(self, n: int, omp: bool = False):
        self.n = int(n)
        self._L = lib(omp)
        self._h = self._L.orc_seq_create(self.n)
        if not self._h:
            raise MemoryError

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_seq_destroy(h)
            self._h = None

    @property
    def nc(self) -> int:
        return self._L.orc_seq_nc(self._h)

    @property
    def m(self) -> int:
        return self._L.orc_seq_m(self._h)

    @property
    def C(self) -> np.ndarray:
        nc = self.nc
        out = np.empty((nc, self.n))
        if nc:
            self._L.orc_seq_get_C(self._h, _d(out))
        return out.T  # n x nc view (column-major storage)

    def set_C(self, C, as_c0: bool = False):
        C = np.asarray(C, dtype=np.float64)
        nc = 0 if C.size == 0 else C.shape[1]
        buf = np.ascontiguousarray(C.T) if nc else np.zeros(1)
        st = self._L.orc_seq_set_C(self._h, nc, _d(buf), int(as_c0))
        if st:
            raise MemoryError

    def _cols(self, fn, k):
        out = np.empty((k, self.n))
        if k:
            fn(self._h, _d(out))
        return out.T

    @property
    def W(self):
        return self._cols(self._L.orc_seq_get_W, self.m)

    @property
    def AW(self):
        return self._cols(self._L.orc_seq_get_AW, self.m)

    @property
    def Z(self):
        return self._cols(self._L.orc_seq_get_Z, self.m)

    def coeffs(self):
        m = self.m
        a, r, g = np.empty(max(m, 1)), np.empty(max(m, 1)), np.empty(max(m, 1))
        self._L.orc_seq_get_coeffs(self._h, _d(a), _d(r), _d(g))
        return a[:m], r[:m], g[:m]

    def ritz(self):
        m, ns = self.m, self._L.orc_seq_nsel(self._h)
        tm, tm1 = np.empty(max(m, 1)), np.empty(max(m, 1))
        sel = np.empty(max(ns, 1), dtype=np.int32)
        Y = np.empty((max(ns, 1), self.n))
        self._L.orc_seq_get_ritz(self._h, _d(tm), _d(tm1), _i(sel), _d(Y))
        return tm[:m], tm1[:max(m - 1, 0)], sel[:ns], Y[:ns].T

    def times(self):
        """Wall-clock seconds of the last solve's set-up, iterations and recycling."""
        out = np.zeros(3)
        self._L.orc_seq_get_times(self._h, _d(out))
        return out

    def solve(self, A, b, tol: float, policy: Policy):
        rp, ci, v = _bsr_args(A)
        b = _f64(b)
        x = np.zeros(self.n)
        st = Stats()
        self._L.orc_seq_solve(self._h, A.n_block_rows, _i(rp), _i(ci), _d(v), _d(b), _d(x),
                            float(tol), ct.byref(policy), ct.byref(st))
        return x, st.as_dict()
