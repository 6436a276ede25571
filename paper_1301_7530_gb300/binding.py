"""Thin ctypes binding of the C ABI in include/krs.h (argument marshalling only).

Every step of a solve runs in the CUDA library (``_build/libkrs.so``); this module only
loads it, declares the structs and signatures, and converts numpy arrays / torch tensors
to pointers.  There is no CPU fallback: ``lib()`` raises if the library cannot be built or
loaded.  PyTorch is used for device memory (the caching allocator is handed to the
library as its allocator) and for the CUDA stream.
"""
from __future__ import annotations

import ctypes as ct
import itertools
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_NOT_SPD, ERR_NO_CONVERGENCE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "NO_CONVERGENCE", 4: "OOM", 5: "CUDA", 6: "TIMEOUT"}
RECYCLE = {"none": 0, "trks": 1, "srks": 2}
PRECOND = {"jacobi": 0, "block_jacobi3": 1, "identity": 2}
REORTH = {"full": 0, "none": 1}
PRECISION = {"fp64": 0, "mixed_ir": 1, "mixed_proj": 2, "double_float": 3}
CAP = {"truncate": 0, "restart": 1}
EXEC = {"persistent": 0, "kernels": 1}
RESELECT = {"none": 0, "cluster": 1}


class krs_bsr(ct.Structure):
    _fields_ = [("n_block_rows", ct.c_int32), ("block_dim", ct.c_int32), ("nnzb", ct.c_int64),
                ("row_ptr", ct.c_void_p), ("col_idx", ct.c_void_p), ("values", ct.c_void_p),
                ("on_device", ct.c_int32), ("version", ct.c_uint64)]


class krs_policy(ct.Structure):
    _fields_ = [("recycle", ct.c_int32), ("precond", ct.c_int32), ("reorth", ct.c_int32),
                ("precision", ct.c_int32), ("ritz_eps", ct.c_double), ("theta_frac", ct.c_double),
                ("max_aug", ct.c_int32), ("cap_mode", ct.c_int32), ("max_iter", ct.c_int32),
                ("exec", ct.c_int32), ("inner_tol", ct.c_double), ("max_outer", ct.c_int32),
                ("reselect", ct.c_int32)]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p)


class krs_device(ct.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ct.c_void_p),
                ("cuda_stream", ct.c_void_p), ("device", ct.c_int32)]


class krs_solve_stats(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("m", ct.c_int32), ("n_c", ct.c_int32),
                ("n_selected", ct.c_int32), ("n_c_after", ct.c_int32), ("rel_res", ct.c_double),
                ("true_rel_res", ct.c_double), ("t_setup_ms", ct.c_double), ("t_iter_ms", ct.c_double),
                ("t_recycle_ms", ct.c_double), ("t_total_ms", ct.c_double),
                ("kernel_launches", ct.c_int64), ("outer_iters", ct.c_int32), ("inner_m_first", ct.c_int32),
                ("inner_m2", ct.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class krs_batch_config(ct.Structure):
    _fields_ = [("group_ctas", ct.c_int32), ("group_scale", ct.c_int32), ("quantum", ct.c_int32),
                ("reserved", ct.c_int32 * 5)]


class krs_batch_stats(ct.Structure):
    _fields_ = [("group_ctas", ct.c_int32), ("groups", ct.c_int32), ("classes", ct.c_int32),
                ("in_flight", ct.c_int32), ("last_launch_solves", ct.c_int32), ("tuned_group_scale", ct.c_int32),
                ("launches", ct.c_int64), ("kernel_launches", ct.c_int64),
                ("last_kernel_ms", ct.c_double), ("total_kernel_ms", ct.c_double),
                ("tune_candidates", ct.c_int32), ("tune_scale", ct.c_int32 * 8), ("tune_ms", ct.c_double * 8),
                ("tune_rate", ct.c_double * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("tune_scale", "tune_ms", "tune_rate")}
        k = min(self.tune_candidates, 8)
        d["tune"] = [(self.tune_scale[i], self.tune_ms[i], self.tune_rate[i]) for i in range(k)]
        return d


RELEASE_SCRATCH, RELEASE_SPACE, RELEASE_MATRIX = 1, 2, 4

_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_V, _P, _I32, _I64, _D = ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
SIGNATURES = {
    "krs_create_sequence": (ct.c_int, [_I64, ct.POINTER(krs_device), ct.POINTER(ct.c_void_p)]),
    "krs_solve": (ct.c_int, [_V, ct.POINTER(krs_bsr), _P, _P, _D, ct.POINTER(krs_policy)]),
    "krs_stats": (ct.c_int, [_V, ct.POINTER(krs_solve_stats)]),
    "krs_destroy_sequence": (ct.c_int, [_V]),
    "krs_last_error": (ct.c_char_p, []),
    "krs_policy_default": (ct.c_int, [ct.POINTER(krs_policy)]),
    "krs_space_size": (ct.c_int, [_V, ct.POINTER(ct.c_int32)]),
    "krs_export_space": (ct.c_int, [_V, _P]),
    "krs_import_space": (ct.c_int, [_V, _I32, _P, _I32]),
    "krs_last_coeffs": (ct.c_int, [_V, _P, _P, _P]),
    "krs_last_ritz": (ct.c_int, [_V, _P, _P, _P]),
    "krs_last_vectors": (ct.c_int, [_V, _I32, _P]),
    "krs_set_spin_limit": (ct.c_int, [_V, _I64]),
    "krs_spmv_bsr3": (ct.c_int, [_I32, _P, _P, _P, _P, _P, _P]),
    "krs_precond_setup": (ct.c_int, [_I32, _I32, _P, _P, _P, _P, _P, _P]),
    "krs_precond_apply": (ct.c_int, [_I32, _I32, _P, _P, _P, _P]),
    "krs_gemv_t": (ct.c_int, [_I64, _I32, _P, _I64, _P, _P, _P]),
    "krs_gemv_n_sub": (ct.c_int, [_I64, _I32, _P, _I64, _P, _P, _P, _P]),
    "krs_gemv_t_noalloc": (ct.c_int, [_I64, _I32, _P, _I64, _P, _P, _P]),
    "krs_axpy2_dot": (ct.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P]),
    "krs_tridiag_eigvals": (ct.c_int, [_I32, _P, _P, _P, _P]),
    "krs_tridiag_eigvecs": (ct.c_int, [_I32, _P, _P, _I32, _P, _P, _P]),
    "krs_validate_bsr": (ct.c_int, [_I32, _I64, _P, _P]),
    "krs_device_bytes": (ct.c_int, [_V, ct.POINTER(ct.c_int64)]),
    "krs_release": (ct.c_int, [_V, _I32]),
    "krs_batch_create": (ct.c_int, [ct.POINTER(krs_device), ct.POINTER(krs_batch_config), ct.POINTER(ct.c_void_p)]),
    "krs_batch_destroy": (ct.c_int, [_V]),
    "krs_batch_submit": (ct.c_int, [_V, _V, ct.POINTER(krs_bsr), _P, _P, _D, ct.POINTER(krs_policy), _I64]),
    "krs_batch_step": (ct.c_int, [_V, _I32, _P, _P, ct.POINTER(ct.c_int32)]),
    "krs_solve_batch": (ct.c_int, [_V, _I32, _P, ct.POINTER(krs_bsr), _P, _P, _D, ct.POINTER(krs_policy), _P]),
    "krs_batch_get_stats": (ct.c_int, [_V, ct.POINTER(krs_batch_stats)]),
    "krs_version": (ct.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def lib(build: bool = True):
    """Load (building first if needed) the CUDA library; raises if it is not available."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run paper_1301_7530_gb300.build.build()")
            L = ct.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class KrsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().krs_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def check(status: int, where: str):
    if status != OK:
        raise KrsError(status, where)


# ----------------------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------------------

def ptr(a) -> int:
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def make_policy(recycle="none", precond="block_jacobi3", reorth="full", precision="fp64",
                ritz_eps=1e-14, theta_frac=0.0, max_aug=0, cap_mode="truncate", max_iter=2000,
                exec="persistent", inner_tol=0.0, max_outer=0, reselect="none") -> krs_policy:
    return krs_policy(RECYCLE[recycle], PRECOND[precond], REORTH[reorth], PRECISION[precision],
                      float(ritz_eps), float(theta_frac), int(max_aug), CAP[cap_mode], int(max_iter),
                      EXEC[exec], float(inner_tol), int(max_outer), RESELECT[reselect])


_versions = itertools.count(1)


def new_version() -> int:
    return next(_versions)


def bsr_struct(A, version: int, on_device: bool | None = None, keep=None) -> krs_bsr:
    """krs_bsr for a problems.BSR3 (host numpy) or a dict of device tensors
    {'row_ptr', 'col_idx', 'values'} (torch, int32/int32/float64)."""
    if isinstance(A, dict):
        rp, ci, v = A["row_ptr"], A["col_idx"], A["values"]
        nbr = int(rp.shape[0]) - 1
        nnzb = int(ci.shape[0])
        dev = True if on_device is None else on_device
    else:
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
        v = np.ascontiguousarray(A.vals, dtype=np.float64)
        nbr, nnzb, dev = A.n_block_rows, A.nnzb, False
    if keep is not None:
        keep.extend([rp, ci, v])
    return krs_bsr(nbr, 3, nnzb, ptr(rp), ptr(ci), ptr(v), int(dev), int(version))


class TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device: int, stream):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream
        self.failures = 0

        def _alloc(size, ctx):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(size), device=self.device, stream=self.stream)
            except Exception:  # noqa: BLE001 -- reported to the library as NULL (KRS_ERR_OOM)
                self.failures += 1
                return None

        def _free(p, ctx):
            if p:
                self._torch.cuda.caching_allocator_delete(p)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class Sequence:
    """A sequence of systems sharing one recycled augmentation space (device resident)."""

    def __init__(self, n: int, device: int = 0, stream=None, torch_allocator: bool = True,
                 alloc_fn=None, free_fn=None):
        import torch
        L = lib()
        self.n = int(n)
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._alloc = None
        dev = krs_device()
        if alloc_fn is not None:
            dev.alloc, dev.free = alloc_fn, free_fn
            self._alloc = (alloc_fn, free_fn)
        elif torch_allocator:
            self._alloc = TorchAllocator(self.device, self.stream)
            dev.alloc, dev.free = self._alloc.alloc_fn, self._alloc.free_fn
        dev.ctx = None
        dev.cuda_stream = self.stream.cuda_stream
        dev.device = self.device
        h = ct.c_void_p()
        check(L.krs_create_sequence(self.n, ct.byref(dev), ct.byref(h)), "krs_create_sequence")
        self._h = h
        self._dev = dev

    def close(self):
        if getattr(self, "_h", None):
            lib().krs_destroy_sequence(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def solve(self, A, b, tol: float, policy: krs_policy, x=None, version: int | None = None,
              raise_on_error: bool = True):
        """Solve A x = b; returns (x, stats dict).  b/x: numpy (host) or torch (device)."""
        keep = []
        bs = bsr_struct(A, new_version() if version is None else version, keep=keep)
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(self.n)
        st = lib().krs_solve(self._h, ct.byref(bs), ptr(b), ptr(x), float(tol), ct.byref(policy))
        stats = self.stats()
        if st != OK and raise_on_error and st not in (ERR_NO_CONVERGENCE,):
            raise KrsError(st, "krs_solve")
        stats["status"] = st
        return x, stats

    def stats(self) -> dict:
        out = krs_solve_stats()
        check(lib().krs_stats(self._h, ct.byref(out)), "krs_stats")
        return out.as_dict()

    @property
    def nc(self) -> int:
        v = ct.c_int32()
        check(lib().krs_space_size(self._h, ct.byref(v)), "krs_space_size")
        return v.value

    def export_space(self) -> np.ndarray:
        nc = self.nc
        out = np.zeros((nc, self.n))
        if nc:
            check(lib().krs_export_space(self._h, out.ctypes.data), "krs_export_space")
        return out.T

    def import_space(self, C, as_c0: bool = False):
        C = np.asarray(C, dtype=np.float64)
        nc = 0 if C.size == 0 else C.shape[1]
        buf = np.ascontiguousarray(C.T) if nc else None
        check(lib().krs_import_space(self._h, nc, ptr(buf), int(as_c0)), "krs_import_space")

    def set_spin_limit(self, spins: int):
        check(lib().krs_set_spin_limit(self._h, int(spins)), "krs_set_spin_limit")

    def device_bytes(self) -> int:
        v = ct.c_int64()
        check(lib().krs_device_bytes(self._h, ct.byref(v)), "krs_device_bytes")
        return v.value

    def release(self, what: int):
        check(lib().krs_release(self._h, int(what)), "krs_release")

    def last_coeffs(self):
        m = self.stats()["m"]
        a, r, g = np.zeros(max(m, 1)), np.zeros(max(m, 1)), np.zeros(max(m, 1))
        check(lib().krs_last_coeffs(self._h, a.ctypes.data, r.ctypes.data, g.ctypes.data), "krs_last_coeffs")
        return a[:m], r[:m], g[:m]

    def last_ritz(self):
        s = self.stats()
        m, ns = s["m"], s["n_selected"]
        tm, tm1 = np.zeros(max(m, 1)), np.zeros(max(m, 1))
        sel = np.zeros(max(ns, 1), dtype=np.int32)
        check(lib().krs_last_ritz(self._h, tm.ctypes.data, tm1.ctypes.data, sel.ctypes.data), "krs_last_ritz")
        return tm[:m], tm1[:max(m - 1, 0)], sel[:ns]

    def last_vectors(self, which: str) -> np.ndarray:
        m = self.stats()["m"]
        out = np.zeros((max(m, 1), self.n))
        idx = {"W": 0, "AW": 1, "Z": 2}[which]
        check(lib().krs_last_vectors(self._h, idx, out.ctypes.data), "krs_last_vectors")
        return out[:m].T


def _device_struct(device: int, stream, allocator):
    dev = krs_device()
    if allocator is not None:
        dev.alloc, dev.free = allocator.alloc_fn, allocator.free_fn
    dev.ctx = None
    dev.cuda_stream = stream.cuda_stream
    dev.device = device
    return dev


class Batch:
    """Batched engine (krs_batch_t): solves of many sequences in one persistent launch."""

    def __init__(self, device: int = 0, stream=None, group_ctas: int = 0, quantum: int = 0,
                 group_scale: int = 0, torch_allocator: bool = True):
        import torch
        L = lib()
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._alloc = TorchAllocator(self.device, self.stream) if torch_allocator else None
        self._dev = _device_struct(self.device, self.stream, self._alloc)
        cfg = krs_batch_config(int(group_ctas), int(group_scale), int(quantum))
        h = ct.c_void_p()
        check(L.krs_batch_create(ct.byref(self._dev), ct.byref(cfg), ct.byref(h)), "krs_batch_create")
        self._h = h
        self._pending = {}  # tag -> (x, keep-alive objects)

    def close(self):
        if getattr(self, "_h", None):
            lib().krs_batch_destroy(self._h)
            self._h = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def submit(self, seq: Sequence, A, b, tol: float, policy: krs_policy, tag: int, x=None,
               version: int | None = None):
        """Queue one solve of `seq`; x (returned by step() under `tag`) receives the result."""
        keep = []
        bs = bsr_struct(A, new_version() if version is None else version, keep=keep)
        if x is None:
            x = np.zeros(seq.n) if isinstance(b, np.ndarray) else b.new_zeros(seq.n)
        check(lib().krs_batch_submit(self._h, seq._h, ct.byref(bs), ptr(b), ptr(x), float(tol),
                                     ct.byref(policy), int(tag)), "krs_batch_submit")
        self._pending[int(tag)] = x
        return x

    def step(self):
        """One launch; returns [(tag, status, x)] of the solves that were returned."""
        cap = max(len(self._pending), 1)
        tags = np.zeros(cap, dtype=np.int64)
        sts = np.zeros(cap, dtype=np.int32)
        nd = ct.c_int32()
        check(lib().krs_batch_step(self._h, cap, tags.ctypes.data, sts.ctypes.data, ct.byref(nd)), "krs_batch_step")
        out = []
        for i in range(nd.value):
            t = int(tags[i])
            out.append((t, int(sts[i]), self._pending.pop(t, None)))
        return out

    def solve(self, seqs, As, bs, tol: float, policy: krs_policy, xs=None, versions=None):
        """One solve per sequence (krs_solve_batch); returns (xs, statuses)."""
        n = len(seqs)
        keep = []
        mats = (krs_bsr * max(n, 1))()
        for i, A in enumerate(As):
            mats[i] = bsr_struct(A, new_version() if versions is None else versions[i], keep=keep)
        if xs is None:
            xs = [np.zeros(s.n) if isinstance(b, np.ndarray) else b.new_zeros(s.n) for s, b in zip(seqs, bs)]
        hs = (ct.c_void_p * max(n, 1))(*[s._h.value for s in seqs])
        rp = (ct.c_void_p * max(n, 1))(*[ptr(b) for b in bs])
        xp = (ct.c_void_p * max(n, 1))(*[ptr(x) for x in xs])
        sts = np.zeros(max(n, 1), dtype=np.int32)
        st = lib().krs_solve_batch(self._h, n, hs, mats, rp, xp, float(tol), ct.byref(policy), sts.ctypes.data)
        if st not in (OK, ERR_NO_CONVERGENCE) and not np.any(sts[:n] != OK):
            raise KrsError(st, "krs_solve_batch")
        return xs, [int(v) for v in sts[:n]]

    def stats(self) -> dict:
        out = krs_batch_stats()
        check(lib().krs_batch_get_stats(self._h, ct.byref(out)), "krs_batch_get_stats")
        return out.as_dict()


# re-export the C function names as thin callables (same names as the C ABI)
def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
