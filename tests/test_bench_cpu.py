"""bench.py's host logic: the reading of the committed ncu summaries (the `traffic` of a
roofline object), the algorithmic counts, the shared config of both arms and the CPU cost
model's arithmetic.

Every persistent-kernel summary names the captured launch (kernel, precision, problem, cube
size, iterations, augmentation size) and carries a source digest, the launch's DRAM traffic
and its algorithmic bytes; the traffic is within a few percent of the algorithmic bytes (no
re-reads), and a summary is used only for the kernel, precision and workload it was taken
on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1301_7530_gb300 import problems as P  # noqa: E402


def _summaries():
    out = []
    for f in sorted(os.listdir(bench.PROFILES)):
        if f.endswith(".md"):
            v = bench.profile_fields(os.path.join(bench.PROFILES, f))
            if v.get("kernel") == "k_apcg_persistent":
                out.append((f, v))
    return out


def test_persistent_summaries_name_their_launch():
    s = _summaries()
    assert s, "no persistent-kernel summary"
    for f, v in s:
        for key in ("precision", "problem", "N", "iterations", "n_c", "csrc_sha256", "traffic_bytes_per_launch",
                    "algorithmic_bytes_per_launch"):
            assert key in v, (f, key)
        ratio = float(v["traffic_bytes_per_launch"]) / float(v["algorithmic_bytes_per_launch"])
        assert 0.95 <= ratio <= 1.05, (f, ratio)
        # the algorithmic bytes are bench's own count for the captured launch
        alg = bench.alg_counts(int(v["N"]), 24, int(v["iterations"]), int(v["n_c"]))[1]
        assert abs(alg - float(v["algorithmic_bytes_per_launch"])) <= 1e-4 * alg, f


def test_traffic_only_for_the_captured_workload(monkeypatch):
    f, v = _summaries()[0]
    monkeypatch.setattr(bench, "csrc_digest", lambda: v["csrc_sha256"])  # read it whatever the sources
    ratio, desc, path = bench.profiled_traffic(v["precision"], v["problem"], int(v["N"]))
    assert ratio is not None and path.endswith(".md") and v["problem"] in desc
    other_n = 7 if v["N"] != "7" else 9
    assert bench.profiled_traffic(v["precision"], v["problem"], other_n) == (None, None, None)
    assert bench.profiled_traffic("mixed_ir", v["problem"], int(v["N"])) == (None, None, None)


def test_stale_digest_gives_no_traffic(monkeypatch):
    monkeypatch.setattr(bench, "csrc_digest", lambda: "0000000000000000")
    for f, v in _summaries():
        assert bench.profiled_traffic(v["precision"], v["problem"], int(v["N"])) == (None, None, None)


@pytest.mark.parametrize("N,m,nc", [(8, 1, 0), (32, 426, 0), (64, 7, 300), (16, 50, 17)])
def test_alg_counts_sum_of_phases(N, m, nc):
    """Closed form against the per-iteration sum of the phase counts."""
    s = P.sizes(N)
    n, nb, nodes = s["n"], s["nb"], s["free_nodes"]
    f = b = 0.0
    for j in range(m):
        f += 18 * nb + 16 * n + 2 * n * nc
        b += 76 * nb + 4 * (nodes + 1) + 24 * n + 8 * n * nc + 48 * n
        if j < m - 1:
            f += 2 * nc * nc + 2 * n * nc + 2 * n + 4 * n * (j + 1)
            b += 8 * n * nc + 16 * n * (j + 1) + 16 * n
    assert bench.alg_counts(N, 24, m, nc) == (f, b)


def test_both_arms_print_the_same_config():
    args = bench.parse_args([])
    ref = bench.parse_args(["--impl", "reference"])

    class _A:
        n, nnzb, n_block_rows = 811200, 7077310, 270400
    assert bench.make_config(args, _A, 1) == bench.make_config(ref, _A, 1)
    assert args.problem == "inclusions" and args.N == 64 and args.step_unit == "system"
    assert bench.step_systems(args, 14) == [14] and bench.step_systems(args, 15) == [0]
    d = bench.parse_args(["--problem", "damage"])
    assert d.N == 32 and bench.step_systems(d, 3) == list(range(20))


def test_cost_model_terms():
    cal = {"t_pre": 1.0, "c_fix": 0.5, "c_col": 0.01, "t_spmv": 0.2, "t_dot": 0.001, "t_eig_cal": 2.0,
           "m_eig_cal": 100, "eig_exponent": 3.0}
    t_set, t_it, t_rec = bench.oracle_model_seconds(cal, 10, 200, 4)
    assert t_set == pytest.approx(1.0 + 10 * 0.21 + 100 * 0.001)
    assert t_it == pytest.approx(200 * 0.5 + 0.01 * (200 * 10 + 200 * 201 / 2))
    assert t_rec == pytest.approx(2.0 * 8 + 4 * 200 * 0.01 / 2)
    assert bench.oracle_model_seconds(cal, 0, 1, 0)[2] == 0.0


def test_sequence_profile_shape():
    prof = bench.SEQ64_PROFILE
    assert prof is not None and len(prof) == 15
    assert prof[0][1] == 0  # the sequence starts from an empty space
    for k in range(1, 15):  # n_c grows by the selected vectors, up to the cap
        assert prof[k][1] == min(300, prof[k - 1][1] + prof[k - 1][2])


def test_cost_model_calibration_runs_on_a_small_cube():
    """The CPU baseline's calibration (bounded oracle samples) on a 6^3 cube: every constant
    is a positive time and the model grows with the iteration count and the space size."""
    A = P.elasticity_inclusions(6, 3000)
    b = P.traction_rhs(6, P.random_traction(6, 3100))
    cal = bench.oracle_calibrate(A, b, eig=False)
    for key in ("t_pre", "c_fix", "t_spmv"):
        assert cal[key] > 0.0, (key, cal)
    assert cal["c_col"] >= 0.0 and cal["t_dot"] >= 0.0 and cal["threads"] >= 1
    cal.update({"t_eig_cal": 1.0, "m_eig_cal": 100, "eig_exponent": 3.0})
    t1 = sum(bench.oracle_model_seconds(cal, 0, 100, 1))
    t2 = sum(bench.oracle_model_seconds(cal, 50, 200, 1))
    assert t2 > t1 > 0.0
