"""The C-ABI library builds, loads and exports every function declared in include/krs.h;
host-only entry points (pattern validation, policy defaults) work without a GPU."""
import ctypes as ct
import os
import re

import numpy as np

from paper_1301_7530_gb300 import binding as B
from paper_1301_7530_gb300 import problems as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "krs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(krs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("krs_create_sequence", "krs_solve", "krs_stats", "krs_destroy_sequence", "krs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(B.SIGNATURES), set(declared_functions()) - set(B.SIGNATURES)


def test_version_and_policy_default():
    L = B.lib()
    assert L.krs_version().decode().startswith("krs")
    p = B.krs_policy()
    assert L.krs_policy_default(ct.byref(p)) == 0
    assert p.precond == 1 and p.reorth == 0 and p.max_iter == 2000 and p.ritz_eps == 1e-14 and p.exec == 0
    assert L.krs_policy_default(None) == B.ERR_INVALID_ARG


def _validate(rp, ci, nbr=None):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    nbr = len(rp) - 1 if nbr is None else nbr
    return B.lib().krs_validate_bsr(nbr, len(ci), rp.ctypes.data, ci.ctypes.data)


def test_validate_bsr_host():
    A = P.assemble(3, P.uniform_modulus(3))
    assert _validate(A.row_ptr, A.col_idx) == 0
    bad = A.col_idx.copy()
    bad[5] = A.n_block_rows + 2  # out of range
    assert _validate(A.row_ptr, bad) == B.ERR_INVALID_ARG
    assert "out of range" in B.lib().krs_last_error().decode()
    unsorted = A.col_idx.copy()
    unsorted[[0, 1]] = unsorted[[1, 0]]
    assert _validate(A.row_ptr, unsorted) == B.ERR_INVALID_ARG
    nodiag = np.array([0, 1, 2], dtype=np.int32), np.array([1, 0], dtype=np.int32)
    assert _validate(*nodiag) == B.ERR_INVALID_ARG
    rp = A.row_ptr.copy()
    rp[0] = 1
    assert _validate(rp, A.col_idx) == B.ERR_INVALID_ARG
    assert _validate(np.array([0], np.int32), np.array([], np.int32)) == 0
