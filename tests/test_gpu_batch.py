"""Batched engine (krs_batch_t): many sequences of different sizes in one persistent launch.

Parity: every batched solve against the FP64 oracle in lock-step (iterations within +-2,
relative solution difference <= 1e-9 at equal counts).  Determinism: with the group size
fixed, a solve's bits do not depend on the mix or on how its iterations are split across
launches, so those comparisons are exact; the adaptive group size (chosen per launch,
with draining) changes partitions with the load and the timing, so engines in that mode
agree to the lock-step bar instead.
"""
import numpy as np
import pytest

import oracle as O
from paper_1301_7530_gb300 import binding as B
from paper_1301_7530_gb300 import problems as P

from .lockstep import check_pair, oracle_policy, rel

pytestmark = pytest.mark.gpu


def _damage_set(Ns, systems, seed0=40):
    out = []
    for i, N in enumerate(Ns):
        mask, b, gen = P.elasticity_sequence_damage(N, systems, seed0 + i, 3000 + i)
        out.append((N, b, [Ak for _, Ak in gen]))
    return out


def _n(N):
    return 3 * N * (N + 1) ** 2


def test_batch_lockstep_vs_oracle(gpu_lib):
    """Five damage sequences (4^3 .. 8^3, uneven sizes) advance together, three systems
    each, SRKS; each batched solve matches the oracle's solve from the same space."""
    probs = _damage_set([4, 7, 5, 8, 6], 3)
    seqs = [B.Sequence(_n(N)) for N, _, _ in probs]
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60)
    eng = B.Batch(group_ctas=0)
    for k in range(3):
        Cs = [s.export_space() for s in seqs]
        xs, sts = eng.solve(seqs, [p[2][k] for p in probs], [p[1] for p in probs], 1e-8, pol,
                            versions=[k + 1] * len(seqs))
        assert sts == [0] * len(seqs)
        for (N, b, mats), s, x, C in zip(probs, seqs, xs, Cs):
            st = s.stats()
            st["status"] = 0
            ora = O.Sequence(_n(N))
            ora.set_C(C)
            xo, so = ora.solve(mats[k], b, 1e-8, oracle_policy(pol))
            check_pair(mats[k], b, 1e-8, pol, x, st, xo, so, C)
            assert st["true_rel_res"] <= 2e-8
    bst = eng.stats()
    assert bst["tuned_group_scale"] in [r for r, _, _ in bst["tune"]]
    assert bst["in_flight"] == 0 and bst["launches"] >= 3


def _run_engine(probs, idx, g, quantum, pol, systems, warm_tol=None, group_scale=0):
    """Solve `systems` systems of the sequences probs[idx] in one engine; returns the
    per-sequence list of (x, m, n_c_after, C)."""
    seqs = {i: B.Sequence(_n(probs[i][0])) for i in idx}
    if warm_tol is not None:  # a short first solve makes the storage estimate small
        for i in idx:
            seqs[i].solve(probs[i][2][0], probs[i][1], warm_tol, B.make_policy("none", "block_jacobi3"), version=99)
    eng = B.Batch(group_ctas=g, quantum=quantum, group_scale=group_scale)
    res = {i: [] for i in idx}
    for k in range(systems):
        xs, sts = eng.solve([seqs[i] for i in idx], [probs[i][2][k] for i in idx], [probs[i][1] for i in idx],
                            1e-9, pol, versions=[k + 1] * len(idx))
        assert sts == [0] * len(idx)
        for i, x in zip(idx, xs):
            st = seqs[i].stats()
            res[i].append((x.copy(), st["m"], st["n_c_after"], seqs[i].export_space()))
    return res, eng


def test_same_alone_and_in_mix(gpu_lib):
    """A sequence gives the same bits solved alone and in a mix of five others."""
    probs = _damage_set([6, 4, 8, 5, 7, 6], 3, seed0=70)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60)
    alone, _ = _run_engine(probs, [0], 4, 0, pol, 3)
    mixed, _ = _run_engine(probs, list(range(6)), 4, 0, pol, 3)
    for (xa, ma, na, Ca), (xb, mb, nb, Cb) in zip(alone[0], mixed[0]):
        assert ma == mb and na == nb
        assert np.array_equal(xa, xb)
        assert np.array_equal(Ca, Cb)


def test_quantum_and_storage_growth_bitwise(gpu_lib):
    """Splitting solves over many launches (quantum 7) and growing direction storage
    between launches (small first estimate) leave the bits unchanged."""
    probs = _damage_set([7, 5, 6], 2, seed0=90)
    pol = B.make_policy("trks", "block_jacobi3", max_aug=400)
    ref, _ = _run_engine(probs, [0, 1, 2], 2, 0, pol, 2)
    split, eng = _run_engine(probs, [0, 1, 2], 2, 7, pol, 2, warm_tol=0.5)
    assert eng.stats()["launches"] > 10
    for i in range(3):
        for (xa, ma, na, Ca), (xb, mb, nb, Cb) in zip(ref[i], split[i]):
            assert ma == mb and na == nb
            assert np.array_equal(xa, xb)
            assert np.array_equal(Ca, Cb)


def test_autotuned_engine_matches_fixed_choice(gpu_lib):
    """The autotuner's probe iterations leave no trace: an engine that tuned its group
    scale agrees with an engine created with that scale (same submissions) to the
    lock-step bar (iterations within +-2; relative difference <= 1e-9 at equal counts)."""
    probs = _damage_set([5, 7, 4, 6], 2, seed0=110)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60)
    tuned, eng = _run_engine(probs, [0, 1, 2, 3], 0, 0, pol, 2)
    r = eng.stats()["tuned_group_scale"]
    assert r > 0
    fixed, _ = _run_engine(probs, [0, 1, 2, 3], 0, 0, pol, 2, group_scale=r)
    for i in range(4):
        for (xa, ma, na, _), (xb, mb, nb, _) in zip(tuned[i], fixed[i]):
            assert abs(ma - mb) <= 2
            if ma == mb and na == nb:
                assert rel(xa, xb) <= 1e-9


def test_submit_step_tags_and_statuses(gpu_lib):
    """Request-level interface: submissions return by tag; a zero right-hand side ends at
    m = 0; a sequence with a solve in flight is refused; the FP32-projection precision is
    not batched."""
    probs = _damage_set([5, 6, 4], 1, seed0=130)
    seqs = [B.Sequence(_n(N)) for N, _, _ in probs]
    pol = B.make_policy("none", "block_jacobi3")
    eng = B.Batch(group_ctas=8, quantum=5)
    for t, ((N, b, mats), s) in enumerate(zip(probs, seqs)):
        eng.submit(s, mats[0], b, 1e-8, pol, tag=100 + t, version=1)
    with pytest.raises(B.KrsError):
        eng.submit(seqs[0], probs[0][2][0], probs[0][1], 1e-8, pol, tag=7, version=1)
    z = B.Sequence(_n(4))
    eng.submit(z, probs[2][2][0], np.zeros(_n(4)), 1e-8, pol, tag=200, version=1)
    with pytest.raises(B.KrsError):
        eng.submit(B.Sequence(_n(4)), probs[2][2][0], probs[2][1], 1e-8,
                   B.make_policy("none", "block_jacobi3", precision="mixed_proj"), tag=8, version=1)
    done = {}
    for _ in range(500):
        for tag, st, x in eng.step():
            done[tag] = (st, x)
        if eng.stats()["in_flight"] == 0:
            break
    assert sorted(done) == [100, 101, 102, 200]
    assert all(st == 0 for st, _ in done.values())
    assert z.stats()["m"] == 0 and np.all(done[200][1] == 0)
    for t, ((N, b, mats), s) in enumerate(zip(probs, seqs)):
        x = done[100 + t][1]
        r = b - mats[0].to_dense() @ x if _n(N) <= 600 else None
        if r is not None:
            assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b)
        assert s.stats()["true_rel_res"] <= 2e-8


def test_release_and_device_bytes(gpu_lib):
    """Releasing scratch and space lowers the bytes held; a re-imported space gives the
    same solve to rounding."""
    N = 6
    mask, b, gen = P.elasticity_sequence_damage(N, 3, 5, 2100)
    mats = [Ak for _, Ak in gen]
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=60)
    s = B.Sequence(_n(N))
    for k in range(2):
        s.solve(mats[k], b, 1e-9, pol, version=k + 1)
    ref = B.Sequence(_n(N))
    ref.import_space(s.export_space())
    x_ref, st_ref = ref.solve(mats[2], b, 1e-9, pol, version=3)
    full = s.device_bytes()
    C = s.export_space()
    s.release(B.RELEASE_SCRATCH)
    after_scratch = s.device_bytes()
    s.release(B.RELEASE_SPACE | B.RELEASE_MATRIX)
    after_all = s.device_bytes()
    assert full > after_scratch > after_all > 0
    assert s.nc == 0
    s.import_space(C)
    x, st = s.solve(mats[2], b, 1e-9, pol, version=3)
    assert st["n_c"] == st_ref["n_c"] and abs(st["m"] - st_ref["m"]) <= 2
    assert rel(x, x_ref) <= 1e-8


def test_batch_mixed_refinement(gpu_lib):
    """Mixed-precision refinement (FP32 passes, FP64 residual) in the batched engine: every
    result meets the FP64 residual tolerance and is within kappa(A) * tol of the dense
    solution; with a fixed group size a solve gives the same bits alone and in a mix."""
    import scipy.linalg as sla
    probs = _damage_set([5, 4, 6], 2, seed0=150)
    pol = B.make_policy("srks", "block_jacobi3", precision="mixed_ir", ritz_eps=1e-6, theta_frac=0.3,
                        max_aug=60, max_iter=800, inner_tol=1e-5)

    def run(idx):
        seqs = [B.Sequence(_n(probs[i][0])) for i in idx]
        eng = B.Batch(group_ctas=2, quantum=9)
        out = []
        for k in range(2):
            xs, sts = eng.solve(seqs, [probs[i][2][k] for i in idx], [probs[i][1] for i in idx], 1e-8, pol,
                                versions=[k + 1] * len(idx))
            assert sts == [0] * len(idx), sts
            out.append([(x.copy(), s.stats()) for x, s in zip(xs, seqs)])
        return out

    mix = run([0, 1, 2])
    for k in range(2):
        for i, (x, st) in enumerate(mix[k]):
            A = probs[i][2][k]
            assert st["true_rel_res"] <= 1.0001e-8 and st["outer_iters"] >= 1
            D = A.to_dense()
            ev = np.linalg.eigvalsh(D)
            xe = sla.cho_solve(sla.cho_factor(D), probs[i][1])
            assert rel(x, xe) <= ev[-1] / ev[0] * 1e-8
    alone = run([1])
    for k in range(2):
        xa, sa = alone[k][0]
        xm, sm = mix[k][1]
        assert sa["m"] == sm["m"] and np.array_equal(xa, xm)
