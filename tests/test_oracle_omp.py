"""The oracle's OpenMP timing build (used only to time the oracle on all host cores) computes
the same solve as the parity build: the same iteration count and the same solution, Ritz
values and selection to rounding (its parallel sums add in another order)."""
import numpy as np
import pytest

import oracle as O
from paper_1301_7530_gb300 import problems as P


def _omp_or_skip():
    try:
        O.build_omp()
    except Exception as exc:  # noqa: BLE001 -- no OpenMP toolchain on this host
        pytest.skip(f"no OpenMP build: {exc}")


def test_omp_build_solves_like_the_parity_build():
    _omp_or_skip()
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 3, 11, 2000)
    pol = O.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60)
    a = O.Sequence(3 * N * (N + 1) ** 2)
    c = O.Sequence(3 * N * (N + 1) ** 2, omp=True)
    for k, Ak in gen:
        c.set_C(a.C)  # lock-step: the same space before each solve
        xa, sa = a.solve(Ak, b, 1e-8, pol)
        xc, sc = c.solve(Ak, b, 1e-8, pol)
        assert sa["status"] == sc["status"] == 0
        assert abs(sa["m"] - sc["m"]) <= 1
        assert np.linalg.norm(xa - xc) <= 1e-9 * np.linalg.norm(xa)
        if sa["m"] == sc["m"]:
            # Ritz values to their own stagnation gap (as in the GPU parity tests): those
            # converged to 1e-12 agree to 1e-9 theta_max, all of them to 1e-3 theta_max
            ta, ta1, sela, _ = a.ritz()
            tc, _, selc, _ = c.ritz()
            conv = np.zeros(len(ta), bool)
            conv[O.srks_select(ta, ta1, 1e-12, 0.0)] = True
            d = np.abs(ta - tc)
            assert d[conv].max(initial=0.0) <= 1e-9 * ta[0]
            assert d.max() <= 1e-3 * ta[0]
    assert O.num_threads(omp=True) >= 1 and O.num_threads() == 1


def test_stage_times_are_recorded():
    A, bs = P.elasticity_sequence_fixed(4, 1, 5)
    s = O.Sequence(A.n)
    x, st = s.solve(A, bs[0], 1e-8, O.make_policy("none", "jacobi"))
    t = s.times()
    assert st["status"] == 0 and t.shape == (3,)
    assert t[0] >= 0.0 and t[1] > 0.0 and t[2] >= 0.0
