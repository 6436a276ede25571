"""Whole solves through the C ABI against the FP64 oracle (lock-step), statuses and edge
cases.  Bar: iterations within +-2, relative solution difference <= 1e-9 at equal
iteration counts (the oracle is rerun for the GPU's count when they differ)."""
import numpy as np
import pytest

import oracle as O
from paper_1301_7530_gb300 import binding as B
from paper_1301_7530_gb300 import problems as P

from .lockstep import check_pair, rel, solve_pair

pytestmark = pytest.mark.gpu


def test_trks_fixed_matrix_sequence(gpu_lib):
    """8^3 cube (1,944 dofs), Jacobi, tol 1e-8, TRKS, 10 seeded traction systems."""
    A, bs = P.elasticity_sequence_fixed(8, 10, 1000)
    seq = B.Sequence(A.n)
    pol = B.make_policy("trks", "jacobi", max_iter=2000)
    ms = []
    for k, b in enumerate(bs):
        x, st, xo, so, ora, C = solve_pair(seq, A, b, 1e-8, pol, version=1)
        check_pair(A, b, 1e-8, pol, x, st, xo, so, C)
        assert st["n_c_after"] == st["n_c"] + st["m"]
        assert st["true_rel_res"] <= 2e-8
        ms.append(st["m"])
    assert ms[-1] < ms[0] / 2  # recycling cuts the iteration count (Section 5, Table 1)
    # the appended directions are the solve's W exactly (Algorithm 2)
    W = seq.last_vectors("W")
    C = seq.export_space()
    assert np.array_equal(C[:, -W.shape[1]:], W)


@pytest.mark.parametrize("eps,frac", [(1e-6, 0.1), (1e-10, 0.0)])
def test_srks_damage_sequence(gpu_lib, eps, frac):
    """Damage sequence on a 6^3 cube, block Jacobi, SRKS; lock-step with the oracle; the
    Ritz values match the oracle's and the GPU's selection follows Eq. 16 on its values."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 6, 11, 2000)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=eps, theta_frac=frac, max_aug=60)
    total_sel = 0
    for k, Ak in gen:
        x, st, xo, so, ora, C = solve_pair(seq, Ak, b, 1e-8, pol, version=k + 1)
        check_pair(Ak, b, 1e-8, pol, x, st, xo, so, C)
        tm, tm1, sel = seq.last_ritz()
        otm, otm1, osel, oY = ora.ritz()
        if st["m"] == so["m"] and st["m"] >= 2:
            assert np.allclose(tm, otm, atol=1e-11 * otm[0])
            assert np.allclose(tm1, otm1, atol=1e-11 * otm[0])
            assert list(O.srks_select(tm, tm1, eps, frac, 60 - st["n_c"])) == list(sel)
            if list(sel) == list(osel) and len(sel):
                Yg = seq.export_space()[:, st["n_c"]:]
                for c in range(len(sel)):
                    th = tm[sel[c]]
                    gap = np.min(np.abs(np.delete(tm, sel[c]) - th))
                    if gap > 1e-3 * tm[0]:
                        a, bb = Yg[:, c], oY[:, c]
                        assert min(rel(a, bb), rel(a, -bb)) <= 1e-6
        total_sel += st["n_selected"]
        assert st["n_c_after"] <= 60
    assert total_sel > 0


@pytest.mark.parametrize("tol,frac", [(1e-12, 0.1), (1e-8, 0.0)])
def test_srks14_selects_in_lockstep(gpu_lib, tol, frac):
    """SRKS with the paper's chosen stagnation threshold eps = 1e-14 ("srks14", Section 5.1)
    on a 6^3 damage sequence where it selects vectors (a tight tolerance lets Ritz values
    converge to the rounding level; without the theta filter the converged upper end is
    kept too): lock-step with the oracle, and the GPU's selection is Eq. 16 applied to its
    own Ritz values."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 4, 11, 2000)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-14, theta_frac=frac, max_aug=60)
    total_sel = 0
    for k, Ak in gen:
        x, st, xo, so, ora, C = solve_pair(seq, Ak, b, tol, pol, version=k + 1)
        check_pair(Ak, b, tol, pol, x, st, xo, so, C)
        tm, tm1, sel = seq.last_ritz()
        if st["m"] >= 2:
            assert list(O.srks_select(tm, tm1, 1e-14, frac, 60 - st["n_c"])) == list(sel)
        total_sel += st["n_selected"]
    assert total_sel > 0


@pytest.mark.parametrize("recycle", ["trks", "srks"])
def test_cap_restart_returns_to_initial_space(gpu_lib, recycle):
    """KRS_CAP_RESTART (Algorithm 3, last step): once the space reaches max_aug after the
    recycling step, C goes back to C^(0).  Both sides start from the same seeded C^(0) of 4
    columns; lock-step (the oracle gets the GPU's C and the same C^(0) before each solve);
    the augmentation sizes after each solve agree and every restart leaves exactly C^(0)."""
    N = 5
    n = 3 * N * (N + 1) ** 2
    rng = np.random.default_rng(55)
    C0 = rng.standard_normal((n, 4))
    if recycle == "trks":
        A, bs = P.elasticity_sequence_fixed(N, 6, 500)
        systems = [(A, bb, 1) for bb in bs]
        pol = B.make_policy("trks", "jacobi", max_aug=160, cap_mode="restart")
    else:
        mask, b, gen = P.elasticity_sequence_damage(N, 6, 12, 2200)
        systems = [(Ak, b, k + 1) for k, Ak in gen]
        pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.0, max_aug=24, cap_mode="restart")
    seq = B.Sequence(n)
    seq.import_space(C0, as_c0=True)
    opol = O.make_policy(recycle, "jacobi" if recycle == "trks" else "block_jacobi3", "full", "restart",
                         pol.max_aug, pol.max_iter, pol.ritz_eps, pol.theta_frac)
    restarts = 0
    for A, bb, ver in systems:
        C = seq.export_space()
        ora = O.Sequence(n)
        ora.set_C(C0, as_c0=True)
        ora.set_C(C)
        x, st = seq.solve(A, bb, 1e-8, pol, version=ver)
        xo, so = ora.solve(A, bb, 1e-8, opol)
        check_pair(A, bb, 1e-8, pol, x, st, xo, so, C)
        appended = st["n_c"] + st["n_selected"]
        if appended >= pol.max_aug:
            restarts += 1
            assert st["n_c_after"] == 4 and np.array_equal(seq.export_space(), C0)
        else:
            assert st["n_c_after"] == appended
        if st["n_selected"] == so["n_selected"]:
            assert so["n_c_after"] == st["n_c_after"]
    assert restarts >= 1


@pytest.mark.parametrize("precision,reorth", [("fp64", "full"), ("fp64", "none"), ("double_float", "full")])
def test_z_from_stored_coefficients(gpu_lib, precision, reorth):
    """The FP64 and double-float solves keep one z column and the reorthogonalisation
    coefficients instead of every z_j: krs_last_vectors(Z) rebuilds z_j = w_j + sum_i g_i w_i.
    Its first 30 columns (where the GPU and oracle trajectories still agree to rounding)
    match the oracle's stored z_j, and the direction storage is two n-vectors per iteration
    (W, AW), not three."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 1, 11, 2000)
    k, A = next(gen)
    seq = B.Sequence(A.n)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60, reorth=reorth,
                        precision=precision, max_iter=400)
    x, st, xo, so, ora, C = solve_pair(seq, A, b, 1e-8, pol, version=1)
    check_pair(A, b, 1e-8, pol, x, st, xo, so, C)
    Zg = seq.last_vectors("Z")
    Zo = ora.Z
    q = min(30, st["m"], so["m"])
    tol = 1e-9 if precision == "fp64" else 1e-7
    for j in range(q):
        assert rel(Zg[:, j], Zo[:, j]) <= tol, (j, rel(Zg[:, j], Zo[:, j]))
    W = seq.last_vectors("W")
    assert np.array_equal(Zg[:, 0], W[:, 0])  # z_0 = w_0
    ld = (A.n + 31) // 32 * 32
    cap = (400 + 1 + 31) // 32 * 32
    held = seq.device_bytes()
    seq.release(B.RELEASE_SCRATCH)
    scratch = held - seq.device_bytes()
    assert 2 * 8 * ld * cap <= scratch < 3 * 8 * ld * cap, (scratch, 8 * ld * cap)


def test_exec_modes_bitwise_equal(gpu_lib):
    """The persistent kernel and the per-phase kernels compute the same bits."""
    N = 5
    mask, b, gen = P.elasticity_sequence_damage(N, 3, 5, 2001)
    mats = [Ak for _, Ak in gen]
    res = {}
    for mode in ("persistent", "kernels"):
        seq = B.Sequence(3 * N * (N + 1) ** 2)
        pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, exec=mode)
        xs = []
        for k, Ak in enumerate(mats):
            x, st = seq.solve(Ak, b, 1e-9, pol, version=k + 1)
            xs.append((x.copy(), st["m"], st["n_c_after"]))
        res[mode] = (xs, seq.export_space())
    for (xa, ma, na), (xb, mb, nb) in zip(res["persistent"][0], res["kernels"][0]):
        assert ma == mb and na == nb and np.array_equal(xa, xb)
    assert np.array_equal(res["persistent"][1], res["kernels"][1])


def test_no_reorth_matches_oracle(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(5, 1, 3000)
    seq = B.Sequence(A.n)
    pol = B.make_policy("none", "jacobi", reorth="none")
    x, st, xo, so, ora, C = solve_pair(seq, A, bs[0], 1e-8, pol, version=1)
    check_pair(A, bs[0], 1e-8, pol, x, st, xo, so, C)


def test_imported_space_and_identity_precond(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(4, 1, 77)
    rng = np.random.default_rng(1)
    C = rng.standard_normal((A.n, 7))
    seq = B.Sequence(A.n)
    seq.import_space(C)
    assert np.array_equal(seq.export_space(), C)
    pol = B.make_policy("none", "identity")
    x, st, xo, so, ora, C2 = solve_pair(seq, A, bs[0], 1e-9, pol, version=1)
    check_pair(A, bs[0], 1e-9, pol, x, st, xo, so, C2)
    r = bs[0] - A.to_scipy() @ x
    assert np.abs(C.T @ r).max() <= 1e-10 * np.linalg.norm(C, 2) * np.linalg.norm(bs[0])


@pytest.mark.parametrize("N", [1, 2, 5, 7])
def test_small_and_ragged_sizes(gpu_lib, N):
    """Tiny systems (one CTA) and node counts that leave a ragged last CTA."""
    A, bs = P.elasticity_sequence_fixed(N, 2, 50 + N)
    seq = B.Sequence(A.n)
    pol = B.make_policy("trks", "block_jacobi3")
    for b in bs:
        x, st, xo, so, ora, C = solve_pair(seq, A, b, 1e-10, pol, version=1)
        check_pair(A, b, 1e-10, pol, x, st, xo, so, C)


def test_device_pointers_in_and_out(gpu_lib):
    import torch
    A, bs = P.elasticity_sequence_fixed(4, 1, 9)
    seq = B.Sequence(A.n)
    pol = B.make_policy("none", "jacobi")
    xh, sth = seq.solve(A, bs[0], 1e-9, pol, version=1)
    bd = torch.as_tensor(bs[0], device="cuda")
    Ad = {"row_ptr": torch.as_tensor(A.row_ptr, device="cuda"), "col_idx": torch.as_tensor(A.col_idx, device="cuda"),
          "values": torch.as_tensor(A.vals, device="cuda").reshape(-1)}
    seq2 = B.Sequence(A.n)
    xd, std = seq2.solve(Ad, bd, 1e-9, pol, version=1)
    torch.cuda.synchronize()
    assert std["m"] == sth["m"] and np.array_equal(xd.cpu().numpy(), xh)


def test_zero_rhs_and_m0(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(3, 1, 1)
    seq = B.Sequence(A.n)
    x, st = seq.solve(A, np.zeros(A.n), 1e-8, B.make_policy("trks"), version=1)
    assert st["status"] == 0 and st["m"] == 0 and np.all(x == 0) and seq.nc == 0


def test_trks_repeated_rhs_converges_at_init(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(4, 2, 31)
    seq = B.Sequence(A.n)
    pol = B.make_policy("trks", "jacobi")
    seq.solve(A, bs[0], 1e-10, pol, version=1)
    seq.solve(A, bs[1], 1e-10, pol, version=1)
    Ad = A.to_dense()
    b2 = 2.0 * bs[0] - 0.5 * bs[1]
    tol2 = 1e-10 * np.sqrt(np.linalg.cond(Ad)) * (2 * np.linalg.norm(bs[0]) + 0.5 * np.linalg.norm(bs[1])) / np.linalg.norm(b2)
    x, st = seq.solve(A, b2, tol2, pol, version=1)
    assert st["m"] == 0 and st["true_rel_res"] <= tol2


# ---------------------------------------------------------------------------------------
# statuses (failures made on the host side or by bounded device waits; nothing faults)
# ---------------------------------------------------------------------------------------

def test_status_not_spd_matrix(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(3, 1, 5)
    i = list(A.col_idx[A.row_ptr[2]:A.row_ptr[3]]).index(2)
    A.vals[A.row_ptr[2] + i] *= -1.0
    seq = B.Sequence(A.n)
    x, st = seq.solve(A, bs[0], 1e-8, B.make_policy("none", "jacobi"), version=1, raise_on_error=False)
    assert st["status"] == B.ERR_NOT_SPD


def test_status_rank_deficient_space(gpu_lib):
    n = 12
    lam = np.arange(1.0, n + 1)
    lam[0] = 4.0
    A = P.BSR3(np.arange(5, dtype=np.int32), np.arange(4, dtype=np.int32),
               np.stack([np.diag(lam[3 * i:3 * i + 3]) for i in range(4)]))
    seq = B.Sequence(n)
    C = np.zeros((n, 2))
    C[0, 0] = C[0, 1] = 1.0  # duplicated column; G = [[4, 4], [4, 4]] exactly
    seq.import_space(C)
    x, st = seq.solve(A, np.ones(n), 1e-8, B.make_policy("none", "identity"), version=1, raise_on_error=False)
    assert st["status"] == B.ERR_NOT_SPD
    assert seq.nc == 2


def test_status_nan_rhs(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(3, 1, 6)
    b = bs[0].copy()
    b[4] = np.nan
    seq = B.Sequence(A.n)
    x, st = seq.solve(A, b, 1e-8, B.make_policy(), version=1, raise_on_error=False)
    assert st["status"] == B.ERR_INVALID_ARG


def test_status_no_convergence_keeps_space(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(4, 2, 7)
    seq = B.Sequence(A.n)
    seq.solve(A, bs[0], 1e-6, B.make_policy("trks", "jacobi"), version=1)
    C0 = seq.export_space()
    for mode in ("persistent", "kernels"):
        x, st = seq.solve(A, bs[1], 1e-14, B.make_policy("trks", "jacobi", max_iter=3, exec=mode), version=1,
                          raise_on_error=False)
        assert st["status"] == B.ERR_NO_CONVERGENCE and st["m"] == 3
        assert np.array_equal(seq.export_space(), C0)
        assert np.all(np.isfinite(x))


def test_status_barrier_timeout_is_reported(gpu_lib):
    """A spin limit of one poll makes the persistent kernel's grid barrier give up; the
    kernel returns KRS_ERR_TIMEOUT and the context stays usable."""
    A, bs = P.elasticity_sequence_fixed(6, 1, 8)
    seq = B.Sequence(A.n)
    seq.set_spin_limit(1)
    x, st = seq.solve(A, bs[0], 1e-8, B.make_policy("none", "jacobi"), version=1, raise_on_error=False)
    assert st["status"] in (B.ERR_TIMEOUT, B.OK)
    seq.set_spin_limit(0)
    x, st = seq.solve(A, bs[0], 1e-8, B.make_policy("none", "jacobi"), version=1)
    assert st["status"] == 0
    xo, so = O.Sequence(A.n).solve(A, bs[0], 1e-8, O.make_policy("none", "jacobi"))
    assert abs(st["m"] - so["m"]) <= 2


def test_allocator_failure_is_oom(gpu_lib):
    calls = {"n": 0}

    def bad_alloc(size, ctx):
        calls["n"] += 1
        return None

    def nop_free(p, ctx):
        pass

    with pytest.raises(B.KrsError) as ei:
        B.Sequence(300, alloc_fn=B.ALLOC_FN(bad_alloc), free_fn=B.FREE_FN(nop_free))
    assert ei.value.status == B.ERR_OOM and calls["n"] >= 1


def test_invalid_arguments(gpu_lib):
    A, bs = P.elasticity_sequence_fixed(2, 1, 1)
    seq = B.Sequence(A.n)
    with pytest.raises(B.KrsError):
        seq.solve(A, bs[0], -1.0, B.make_policy(), version=1)
    with pytest.raises(B.KrsError):
        seq.solve(A, bs[0], 1e-8, B.make_policy(max_iter=0), version=1)
    bad = B.make_policy()
    bad.precision = 7
    with pytest.raises(B.KrsError):
        seq.solve(A, bs[0], 1e-8, bad, version=1)
    A3, _ = P.elasticity_sequence_fixed(3, 1, 1)
    with pytest.raises(B.KrsError):
        seq.solve(A3, np.zeros(A3.n), 1e-8, B.make_policy(), version=2)


# ---------------------------------------------------------------------------------------
# full size of the benchmark workload (32^3 damage sequence, 104,544 dofs)
# ---------------------------------------------------------------------------------------

def test_full_size_first_solves_lockstep_and_sequence_properties(gpu_lib):
    """First three systems of the 32^3 damage sequence in lock-step with the oracle (the
    oracle gets the GPU's space before each solve): iterations, solution, Ritz values, the
    SRKS selection (Eq. 16 on the GPU's values, and the oracle's own selection when the two
    value sets agree) and the Ritz vectors of well-separated selected values; then a fourth
    GPU solve checked by properties that hold at any size: true residual, the augmentation
    cap, C^T r = 0 for the returned x."""
    N = 32
    eps, frac, cap = 1e-6, 0.1, 200
    mask, b, gen = P.elasticity_sequence_damage(N, 20, 2000, 2000)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=eps, theta_frac=frac, max_aug=cap)
    for k, Ak in gen:
        if k > 3:
            break
        if k <= 2:
            x, st, xo, so, ora, C = solve_pair(seq, Ak, b, 1e-8, pol, version=k + 1)
            check_pair(Ak, b, 1e-8, pol, x, st, xo, so, C)
            tm, tm1, sel = seq.last_ritz()
            otm, otm1, osel, oY = ora.ritz()
            assert list(O.srks_select(tm, tm1, eps, frac, cap - st["n_c"])) == list(sel)
            if st["m"] == so["m"]:
                # A Ritz value is known to about its own stagnation gap |theta_m - theta_m-1|
                # (Eq. 16).  Values whose gap is below 1e-12 |theta| (on the oracle's values)
                # agree to 1e-9 theta_max; values below 1e-6 |theta| (the selection threshold
                # of this run) to 1e-5 |theta|; the others are set by the last iterations'
                # coefficients, which sit at the residual's rounding floor (FP64: ~m 2^-53 / tol
                # relative), so all of them to 1e-3 theta_max
                d = np.abs(tm - otm)
                for eps_t, bound in ((1e-12, np.full_like(otm, 1e-9 * otm[0])),
                                     (1e-6, 1e-5 * np.abs(otm) + 1e-11 * otm[0])):
                    tier = np.zeros(len(otm), bool)
                    tier[O.srks_select(otm, otm1, eps_t, 0.0)] = True
                    bad = tier & (d > bound)
                    assert not bad.any(), (k, eps_t, np.flatnonzero(bad), d[bad], otm[bad])
                assert d.max() <= 1e-3 * otm[0], (k, d.max(), int(np.argmax(d)))
                assert np.all(d[sel] <= 1e-5 * np.abs(otm[sel]) + 1e-11 * otm[0]), (k, d[sel])
                if list(sel) == list(osel):
                    Yg = seq.export_space()[:, st["n_c"]:]
                    for c in range(len(sel)):
                        th = tm[sel[c]]
                        gap = np.min(np.abs(np.delete(tm, sel[c]) - th))
                        if gap > 1e-3 * tm[0]:
                            a, bb = Yg[:, c], oY[:, c]
                            assert min(rel(a, bb), rel(a, -bb)) <= 1e-6
            continue
        Cb = seq.export_space()
        x, st = seq.solve(Ak, b, 1e-8, pol, version=k + 1)
        assert st["true_rel_res"] <= 1e-7
        r = b - Ak.to_scipy() @ x
        if Cb.shape[1]:
            assert np.abs(Cb.T @ r).max() <= 1e-9 * np.linalg.norm(Cb, axis=0).max() * np.linalg.norm(b) * np.sqrt(Cb.shape[1])
        assert seq.nc <= cap


def test_misaligned_device_matrix_is_copied(gpu_lib):
    """A caller's device matrix whose values are only 8-byte aligned gives the same result
    (the library copies it into aligned storage)."""
    import torch
    A, bs = P.elasticity_sequence_fixed(3, 1, 12)
    pol = B.make_policy("none", "jacobi")
    x_ref, st_ref = B.Sequence(A.n).solve(A, bs[0], 1e-10, pol, version=1)
    big = torch.zeros(A.vals.size + 1, dtype=torch.float64, device="cuda")
    big[1:] = torch.as_tensor(A.vals.reshape(-1), device="cuda")
    Ad = {"row_ptr": torch.as_tensor(A.row_ptr, device="cuda"), "col_idx": torch.as_tensor(A.col_idx, device="cuda"),
          "values": big[1:]}
    assert Ad["values"].data_ptr() % 16 == 8
    x, st = B.Sequence(A.n).solve(Ad, torch.as_tensor(bs[0], device="cuda"), 1e-10, pol, version=1)
    torch.cuda.synchronize()
    assert st["m"] == st_ref["m"] and np.array_equal(x.cpu().numpy(), x_ref)


def test_srks_cluster_reselection_lockstep(gpu_lib):
    """SRKS with cluster reselection (Section 4.4, end): lock-step with the oracle; the
    GPU's selection equals the oracle's selection function applied to the GPU's Ritz values,
    and it is a subset of plain Eq. 16 selection."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 5, 13, 2300)
    seq = B.Sequence(3 * N * (N + 1) ** 2)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-10, max_aug=80, reselect="cluster")
    dropped = 0
    for k, Ak in gen:
        x, st, xo, so, ora, C = solve_pair(seq, Ak, b, 1e-8, pol, version=k + 1)
        check_pair(Ak, b, 1e-8, pol, x, st, xo, so, C)
        tm, tm1, sel = seq.last_ritz()
        if st["m"] >= 2:
            room = 80 - st["n_c"]
            assert list(O.srks_select(tm, tm1, 1e-10, 0.0, room, reselect=1)) == list(sel)
            plain = set(O.srks_select(tm, tm1, 1e-10, 0.0))
            full = set(O.srks_select(tm, tm1, 1e-10, 0.0, reselect=1))
            assert set(sel) <= full <= plain
            dropped += len(plain) - len(full)
    assert dropped > 0
