"""Lock-step GPU <-> oracle comparison of one solve of a sequence.

Before each solve the GPU sequence's augmentation space is copied into the oracle, so a
rounding-level difference in a Ritz selection cannot compound across the sequence.
Bar: iteration counts within +-2; relative solution difference <= 1e-9 at the same
iteration count (when the counts differ the oracle is rerun for exactly the GPU's count).
"""
import numpy as np

import oracle as O

SOL_TOL = 1e-9
ITER_TOL = 2


def oracle_policy(gpol):
    rec = {0: "none", 1: "trks", 2: "srks"}[gpol.recycle]
    pre = {0: "jacobi", 1: "block_jacobi3", 2: "identity"}[gpol.precond]
    reo = {0: "full", 1: "none"}[gpol.reorth]
    cap = {0: "truncate", 1: "restart"}[gpol.cap_mode]
    res = {0: "none", 1: "cluster"}[gpol.reselect]
    return O.make_policy(rec, pre, reo, cap, gpol.max_aug, gpol.max_iter, gpol.ritz_eps, gpol.theta_frac, res)


def rel(a, b):
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def solve_pair(gseq, A, b, tol, gpol, version):
    """One lock-step solve; returns (x_gpu, stats_gpu, x_oracle, stats_oracle, oracle_seq)."""
    C = gseq.export_space()
    ora = O.Sequence(A.n)
    ora.set_C(C)
    opol = oracle_policy(gpol)
    x, st = gseq.solve(A, b, tol, gpol, version=version, raise_on_error=False)
    xo, so = ora.solve(A, b, tol, opol)
    return x, st, xo, so, ora, C


def check_pair(A, b, tol, gpol, x, st, xo, so, C):
    assert st["status"] == so["status"], (st, so)
    if st["status"] != 0:
        return None
    assert abs(st["m"] - so["m"]) <= ITER_TOL, (st["m"], so["m"])
    if st["m"] == so["m"]:
        err = rel(x, xo)
    else:
        ora2 = O.Sequence(A.n)
        ora2.set_C(C)
        p2 = oracle_policy(gpol)
        p2.max_iter = st["m"]
        xo2, so2 = ora2.solve(A, b, 0.0, p2)
        assert so2["m"] == st["m"]
        err = rel(x, xo2)
    assert err <= SOL_TOL, err
    return err
