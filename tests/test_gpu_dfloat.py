"""Double-float precision (KRS_DOUBLE_FLOAT) against the FP64 oracle.

The solve is the FP64 one (preconditioner, recurrences, projection with the FP64 C and AC,
coarse set-up, H_m) except that W, AW, Z and the matrix values are stored as double-float
pairs (48-bit significand) and the operator product and the reorthogonalisation's products
are taken on the FP32 pipes with error-free products and compensated sums (about 2^-46
relative).  That is far below the solve tolerance, so the FP64 parity bar applies to the
solves unchanged: lock-step with the oracle, iterations within +-2, relative solution
difference <= 1e-9 at equal counts.  Ritz values that have not converged are the one
quantity held to a looser, derived bound (test_dfloat_srks_damage_sequence).
"""
import numpy as np
import pytest

import oracle as O
from paper_1301_7530_gb300 import binding as B
from paper_1301_7530_gb300 import problems as P

from .lockstep import check_pair, oracle_policy, rel, solve_pair

pytestmark = pytest.mark.gpu

DF = "double_float"


def test_dfloat_trks_fixed_matrix_sequence(gpu_lib):
    """8^3 cube, Jacobi, TRKS over 10 systems; the appended columns are the solve's
    directions converted to FP64 exactly as krs_last_vectors returns them."""
    A, bs = P.elasticity_sequence_fixed(8, 10, 1000)
    seq = B.Sequence(A.n)
    pol = B.make_policy("trks", "jacobi", max_iter=2000, precision=DF)
    ms = []
    for k, b in enumerate(bs):
        x, st, xo, so, ora, C = solve_pair(seq, A, b, 1e-8, pol, version=1)
        check_pair(A, b, 1e-8, pol, x, st, xo, so, C)
        assert st["n_c_after"] == st["n_c"] + st["m"]
        assert st["true_rel_res"] <= 2e-8
        ms.append(st["m"])
    assert ms[-1] < ms[0] / 2
    W = seq.last_vectors("W")
    C = seq.export_space()
    assert np.array_equal(C[:, -W.shape[1]:], W)
    # the stored directions are the FP64 ones to the double-float significand: A W against
    # the returned A W
    AW = seq.last_vectors("AW")
    assert rel(A.to_scipy() @ W, AW) <= 1e-12


@pytest.mark.parametrize("eps,frac", [(1e-6, 0.1), (1e-10, 0.0)])
def test_dfloat_srks_damage_sequence(gpu_lib, eps, frac):
    """6^3 damage sequence, block Jacobi, SRKS in lock-step.  The selection is Eq. 16 applied
    to the GPU's own Ritz values; selected (converged) values match the oracle's to 1e-9
    theta_max.  Ritz values that have not converged depend on the last iterations' alpha and
    rho, which sit at the residual's rounding floor: the recursive residual carries the
    operator products' rounding, ~m 2^-46 ||r_0|| in double-float, so relative to a residual
    of tol ||b|| the last coefficients move by ~m 2^-46 / tol (1e-4 at m = 80, tol = 1e-8);
    all values are held to 1e-3 theta_max."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 6, 11, 2000)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=eps, theta_frac=frac, max_aug=60, precision=DF)
    total_sel = 0
    for k, Ak in gen:
        x, st, xo, so, ora, C = solve_pair(seq, Ak, b, 1e-8, pol, version=k + 1)
        check_pair(Ak, b, 1e-8, pol, x, st, xo, so, C)
        tm, tm1, sel = seq.last_ritz()
        otm, otm1, osel, oY = ora.ritz()
        if st["m"] == so["m"] and st["m"] >= 2:
            assert np.max(np.abs(tm - otm)) <= 1e-3 * otm[0]
            assert list(O.srks_select(tm, tm1, eps, frac, 60 - st["n_c"])) == list(sel)
            if list(sel) == list(osel):
                for i in sel:
                    assert abs(tm[i] - otm[i]) <= 1e-9 * otm[0]
            if list(sel) == list(osel) and len(sel):
                Yg = seq.export_space()[:, st["n_c"]:]
                for c in range(len(sel)):
                    th = tm[sel[c]]
                    gap = np.min(np.abs(np.delete(tm, sel[c]) - th))
                    if gap > 1e-3 * tm[0]:
                        a, bb = Yg[:, c], oY[:, c]
                        assert min(rel(a, bb), rel(a, -bb)) <= 1e-6
        total_sel += st["n_selected"]
    assert total_sel > 0


def test_dfloat_exec_modes_bitwise_equal(gpu_lib):
    N = 5
    mask, b, gen = P.elasticity_sequence_damage(N, 3, 5, 2001)
    mats = [Ak for _, Ak in gen]
    res = {}
    for mode in ("persistent", "kernels"):
        seq = B.Sequence(3 * N * (N + 1) ** 2)
        pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, exec=mode, precision=DF)
        xs = []
        for k, Ak in enumerate(mats):
            x, st = seq.solve(Ak, b, 1e-9, pol, version=k + 1)
            xs.append((x.copy(), st["m"], st["n_c_after"]))
        res[mode] = (xs, seq.export_space())
    for (xa, ma, na), (xb, mb, nb) in zip(res["persistent"][0], res["kernels"][0]):
        assert ma == mb and na == nb and np.array_equal(xa, xb)
    assert np.array_equal(res["persistent"][1], res["kernels"][1])


@pytest.mark.parametrize("N", [1, 2, 7])
def test_dfloat_small_and_ragged_sizes(gpu_lib, N):
    A, bs = P.elasticity_sequence_fixed(N, 2, 50 + N)
    seq = B.Sequence(A.n)
    pol = B.make_policy("trks", "block_jacobi3", precision=DF)
    for b in bs:
        x, st, xo, so, ora, C = solve_pair(seq, A, b, 1e-10, pol, version=1)
        check_pair(A, b, 1e-10, pol, x, st, xo, so, C)


def test_dfloat_mixed_with_fp64_in_one_sequence(gpu_lib):
    """Precisions may alternate within a sequence (C and AC are FP64 in both)."""
    N = 5
    mask, b, gen = P.elasticity_sequence_damage(N, 4, 9, 2002)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    for k, Ak in gen:
        prec = DF if k % 2 == 0 else "fp64"
        pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=40, precision=prec)
        x, st, xo, so, ora, C = solve_pair(seq, Ak, b, 1e-8, pol, version=k + 1)
        check_pair(Ak, b, 1e-8, pol, x, st, xo, so, C)


def test_dfloat_full_size_first_system(gpu_lib):
    """First system of the 32^3 damage sequence (104,544 dofs): the double-float solve
    against the FP64 GPU solve (itself in lock-step with the oracle in test_gpu_solve):
    iterations within +-2 and the same solution to 1e-9 when the counts agree."""
    mask, b, gen = P.elasticity_sequence_damage(32, 1, 2000, 2000)
    A = next(gen)[1]
    x64, st64 = B.Sequence(A.n).solve(A, b, 1e-8, B.make_policy("none", "block_jacobi3"), version=1)
    xdf, stdf = B.Sequence(A.n).solve(A, b, 1e-8, B.make_policy("none", "block_jacobi3", precision=DF), version=1)
    assert stdf["status"] == 0 and stdf["true_rel_res"] <= 1.05e-8
    assert abs(stdf["m"] - st64["m"]) <= 2
    if stdf["m"] == st64["m"]:
        assert rel(xdf, x64) <= 1e-9


def test_dfloat_batched_lockstep(gpu_lib):
    """Four damage sequences of uneven sizes in the batched engine in double-float, three
    systems each, each solve against the oracle from the same space."""
    Ns = [4, 7, 5, 6]
    probs = []
    for i, N in enumerate(Ns):
        mask, b, gen = P.elasticity_sequence_damage(N, 3, 40 + i, 3000 + i)
        probs.append((N, b, [Ak for _, Ak in gen]))
    seqs = [B.Sequence(3 * N * (N + 1) ** 2) for N, _, _ in probs]
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60, precision=DF)
    eng = B.Batch(group_ctas=0)
    for k in range(3):
        Cs = [s.export_space() for s in seqs]
        xs, sts = eng.solve(seqs, [p[2][k] for p in probs], [p[1] for p in probs], 1e-8, pol,
                            versions=[k + 1] * len(seqs))
        assert sts == [0] * len(seqs)
        for (N, b, mats), s, x, C in zip(probs, seqs, xs, Cs):
            st = s.stats()
            st["status"] = 0
            ora = O.Sequence(3 * N * (N + 1) ** 2)
            ora.set_C(C)
            xo, so = ora.solve(mats[k], b, 1e-8, oracle_policy(pol))
            check_pair(mats[k], b, 1e-8, pol, x, st, xo, so, C)


def test_dfloat_and_fp64_in_one_engine(gpu_lib):
    """FP64 and double-float solves submitted to one engine (each step launches once per
    precision present): every result against the oracle from the same space, two systems."""
    Ns = [5, 6, 4, 7]
    precs = ["fp64", DF, DF, "fp64"]
    probs = []
    for i, N in enumerate(Ns):
        mask, b, gen = P.elasticity_sequence_damage(N, 2, 60 + i, 3100 + i)
        probs.append((N, b, [Ak for _, Ak in gen]))
    seqs = [B.Sequence(3 * N * (N + 1) ** 2) for N, _, _ in probs]
    pols = [B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60, precision=p)
            for p in precs]
    eng = B.Batch(group_ctas=0)
    for k in range(2):
        Cs = [s.export_space() for s in seqs]
        for i, (s, (N, b, mats)) in enumerate(zip(seqs, probs)):
            eng.submit(s, mats[k], b, 1e-8, pols[i], tag=i, version=k + 1)
        done = {}
        for _ in range(1000):
            for tag, status, x in eng.step():
                done[tag] = (status, x)
            if len(done) == len(seqs):
                break
        assert sorted(done) == list(range(len(seqs)))
        for i, ((N, b, mats), s, C) in enumerate(zip(probs, seqs, Cs)):
            status, x = done[i]
            assert status == 0
            st = s.stats()
            ora = O.Sequence(3 * N * (N + 1) ** 2)
            ora.set_C(C)
            xo, so = ora.solve(mats[k], b, 1e-8, oracle_policy(pols[i]))
            check_pair(mats[k], b, 1e-8, pols[i], np.asarray(x), st, xo, so, C)
    eng.close()


def test_dfloat_trks_changing_matrix(gpu_lib):
    """TRKS over a damage sequence (A changes every system): the appended double-float
    directions are converted to FP64 and A C is recomputed by the FP64 product; lock-step."""
    N = 5
    mask, b, gen = P.elasticity_sequence_damage(N, 4, 17, 2003)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("trks", "block_jacobi3", max_aug=150, precision=DF)
    for k, Ak in gen:
        x, st, xo, so, ora, C = solve_pair(seq, Ak, b, 1e-8, pol, version=k + 1)
        check_pair(Ak, b, 1e-8, pol, x, st, xo, so, C)
        assert st["n_c_after"] == min(150, st["n_c"] + st["m"])


def test_dfloat_after_release(gpu_lib):
    """Releasing the scratch (directions, FP64 copies of w and q, the double-float matrix) and
    the matrix between solves: the next double-float solve re-creates them and gives the same
    bits."""
    A, bs = P.elasticity_sequence_fixed(5, 1, 77)
    seq = B.Sequence(A.n)
    pol = B.make_policy("none", "block_jacobi3", precision=DF)
    x1, st1 = seq.solve(A, bs[0], 1e-9, pol, version=1)
    held = seq.device_bytes()
    seq.release(B.RELEASE_SCRATCH | B.RELEASE_MATRIX)
    assert seq.device_bytes() < held
    x2, st2 = seq.solve(A, bs[0], 1e-9, pol, version=1)
    assert st2["m"] == st1["m"] and np.array_equal(x1, x2)
