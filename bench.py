#!/usr/bin/env python3
"""Benchmark: solves/s and p50/p99 latency at relative residual 1e-8, and the achieved
throughput of the dominant kernel (the persistent APCG iteration kernel) against its roofs.

Default workload: the largest single sequence -- Q1 elasticity on 64^3 hexahedra (811,200
FP64 dofs in 3x3 BSR) with seeded stiff spherical inclusions (5 % of the elements, modulus
contrast 1e3), 15 systems with the fixed matrix and one seeded traction draw each;
block-Jacobi preconditioner; SRKS (Algorithm 3) with stagnation threshold 1e-6, Ritz values
below 0.1 theta_max, at most 300 augmentation vectors; FP64 throughout.  One "step" is one
system of the sequence, taken in order; after the 15th system the sequence starts again
from an empty augmentation space.  The matrix and every right-hand side are resident on the
device when the timed region starts; the direction storage streamed every iteration (tens
of GB) is far larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl krs|reference]

Beside the headline the line carries: the same systems in the double-float precision (a
bounded sample), the sequence's first systems in the mixed precision (FP32 passes under an
FP64 flexible-CG outer step) against FP64's time and results on them, the 32^3 damage
sequence in FP64 (one step = its 20 systems), an end-to-end figure through the C ABI with
host buffers, and the oracle's CPU baseline.
Multi-GPU (torchrun): every rank solves its own sequence (independent problems, no data
collective); value = all ranks' solves / the slowest rank's time ("weak" scaling).
--impl reference times the FP64 CPU oracle (rank 0 only): each step a bounded sample of the
same system, extrapolated to the whole system by a cost model calibrated on the spot.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1301_7530_gb300 import problems as P  # noqa: E402

METRIC = "solves/s and p50/p99 latency at rel. residual 1e-8; SpMV+proj HBM GB/s vs 8 TB/s"
UNIT = "solves/s"
TOL = 1e-8
PROFILES = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_1301_7530_gb300", "csrc")

# the two sequences: (cube, systems, cap, stored-direction budget, step unit)
SEQUENCES = {
    "inclusions": {"N": 64, "systems": 15, "max_aug": 300, "max_iter": 7000, "step": "system"},
    "damage": {"N": 32, "systems": 20, "max_aug": 200, "max_iter": 2000, "step": "sequence"},
}

# Work of each system of the 64^3 inclusion sequence under the default policy: iteration
# count m, augmentation size n_c at the start of the solve and vectors selected after it.
# The iteration counts are the method's (the FP64 oracle and the GPU agree to +-2 by the
# parity bar); they are the input of the CPU cost model of --impl reference, which cannot
# run a 4,000-iteration solve on 811,200 dofs itself.  Recorded from a full FP64 run of
# the sequence; the GPU arm reports the counts it actually took beside them.
SEQ64_PROFILE = [(6162, 0, 140), (2458, 140, 20), (1975, 160, 14), (1829, 174, 7), (1777, 181, 6),
                 (1761, 187, 6), (1700, 193, 9), (1642, 202, 8), (1678, 210, 11), (1617, 221, 7),
                 (1621, 228, 8), (1582, 236, 8), (1486, 244, 5), (1533, 249, 9), (1478, 258, 7)]


def dtype_of(precision):
    """Arithmetic type of the path: FP64; FP64 with double-float (two-FP32) directions; or
    FP32 inner passes with FP64 refinement."""
    return {"fp64": "f64", "double_float": "f64+df32x2"}.get(precision, "f32+f64")


# FP64 ALU roof of GB300: 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x 2.07 GHz
# (NVIDIA's 1.25 TFLOP/s FP64 figure; the unit count measured 1.9 FMA/clk/SM).
SMS, FP64_FMA_PER_CLK_SM, SM_MAX_MHZ = 152, 2, 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["krs", "reference"], default="krs")
    ap.add_argument("--problem", choices=["inclusions", "damage"], default="inclusions",
                    help="sequence workload: the 64^3 stiff-inclusion cube (default) or the 32^3 damage sequence")
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--systems", type=int, default=None)
    ap.add_argument("--step-unit", choices=["system", "sequence"], default=None,
                    help="one timed step: one system (inclusions default) or a whole sequence (damage default)")
    ap.add_argument("--systems-many", type=int, default=None, help="batched/served: systems per sequence (10 / 30)")
    ap.add_argument("--exec", choices=["persistent", "kernels"], default="persistent")
    ap.add_argument("--ritz-eps", type=float, default=1e-6)
    ap.add_argument("--theta-frac", type=float, default=0.1)
    ap.add_argument("--max-aug", type=int, default=None)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--max-iter", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the extra objects (double-float sample, 32^3 damage sequence)")
    ap.add_argument("--mixed-systems", type=int, default=3,
                    help="systems of the mixed-precision sample (the sequence's first ones, from an empty space)")
    ap.add_argument("--mixed-inner-tol", type=float, default=0.0,
                    help="mixed-precision sample: relative residual of the first FP32 pass (0: the library default)")
    ap.add_argument("--variant-systems", type=int, default=3,
                    help="systems of the double-float sample of the headline sequence")
    ap.add_argument("--precision", choices=["fp64", "double_float", "mixed_ir", "mixed_proj"], default="fp64",
                    help="sequence workload: FP64, FP32 refinement passes, or FP32 projection passes")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed_ir: relative residual of each FP32 pass (0: the library default 0.1)")
    ap.add_argument("--reselect", choices=["none", "cluster"], default="none",
                    help="SRKS cluster reselection (Section 4.4, end)")
    ap.add_argument("--capture-one", type=int, default=0,
                    help="profiling: solve system 0 only, for at most this many iterations, and exit "
                         "(a bounded launch for ncu; no timing line)")
    ap.add_argument("--capture-nc", type=int, default=0,
                    help="profiling: the captured solve starts from a seeded space of this many columns")
    ap.add_argument("--workload", choices=["sequence", "batched", "served", "conditioning", "fp64peak"],
                    default="sequence",
                    help="sequence: one sequence (default); batched: many sequences of uneven size "
                         "through the batched engine; served: Poisson requests of many clients")
    ap.add_argument("--nseq", type=int, default=None, help="batched/served: sequences (256 / 64)")
    ap.add_argument("--nmin", type=int, default=None, help="batched/served: smallest cube (16 / 12)")
    ap.add_argument("--nmax", type=int, default=None, help="batched/served: largest cube (40 / 48)")
    ap.add_argument("--rate", type=float, default=200.0, help="served: offered requests per second")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served: device memory budget")
    ap.add_argument("--group-ctas", type=int, default=0, help="batched/served: CTAs per solve (0: autotune)")
    ap.add_argument("--quantum", type=int, default=None, help="batched/served: iterations per launch")
    ap.add_argument("--group-scale", type=int, default=0, help="batched/served: group size scale in percent (0: autotune)")
    ap.add_argument("--lanczos-steps", type=int, default=12, help="conditioning: Lanczos steps on A^-1")
    ap.add_argument("--check-sample", type=int, default=8,
                    help="batched/served: error of the results of this many (smallest) sequences, first and "
                         "last system, against the FP64 oracle's solution")
    ap.add_argument("--baseline-seqs", type=int, default=None,
                    help="batched/served: sequences in the per-solve reference sample (default all)")
    args = ap.parse_args(argv)
    d = SEQUENCES[args.problem]
    for key, attr in (("N", "N"), ("systems", "systems"), ("max_aug", "max_aug"), ("max_iter", "max_iter"),
                      ("step", "step_unit")):
        if getattr(args, attr) is None:
            setattr(args, attr, d[key])
    return args


# ----------------------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------------------

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(v, world, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def all_max(v, world):
    """Largest v over the ranks (the job's time is the slowest rank's)."""
    import torch.distributed as dist
    return _reduce(v, world, dist.ReduceOp.MAX if world > 1 else None)


def all_sum(v, world):
    """Sum of v over the ranks (the job's solves)."""
    import torch.distributed as dist
    return _reduce(v, world, dist.ReduceOp.SUM if world > 1 else None)


# ----------------------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------------------

def workload(N, systems, rank, problem="inclusions"):
    """(matrices, right-hand sides) of the sequence: the inclusion cube (fixed A with seeded
    stiff spheres, one traction draw per system) or the damage sequence (one A^(k) per
    system, fixed b)."""
    if problem == "inclusions":
        A = P.elasticity_inclusions(N, 3000 + rank)
        bs = [P.traction_rhs(N, P.random_traction(N, 3100 + 100 * rank + k)) for k in range(systems)]
        return [A] * systems, bs
    mask, b, gen = P.elasticity_sequence_damage(N, systems, 2000, 2000 + rank)
    mats = [A for _, A in gen]
    return mats, [b] * systems


def step_systems(args, step_index):
    """System indices one step solves (a step counts from the first warm-up step)."""
    if args.step_unit == "sequence":
        return list(range(args.systems))
    return [step_index % args.systems]


def workload_name(args):
    if args.problem == "inclusions":
        return (f"{args.N}^3 Q1 elasticity with stiff spherical inclusions (5 %, contrast 1e3), "
                f"{args.systems}-system traction sequence, SRKS, one system per step")
    return f"{args.N}^3 Q1 elasticity damage sequence, {args.systems} systems per step, SRKS"


def make_config(args, A, world):
    """The `config` object of the line; both arms print the same one."""
    solves_per_step = args.systems if args.step_unit == "sequence" else 1
    if args.problem == "inclusions":
        l2 = ("inputs larger than L2: the matrix (0.54 GB) and the stored directions (tens of GB) "
              "are streamed every iteration")
    else:
        l2 = (f"inputs larger than L2: {args.systems} resident matrices "
              f"({args.systems * (76 * A.nnzb + 4 * (A.n_block_rows + 1)) / 1e9:.2f} GB), plus the direction "
              "storage streamed every iteration")
    return {
        "workload": workload_name(args), "problem": args.problem, "N": args.N, "n": A.n, "nnzb": A.nnzb,
        "systems_in_sequence": args.systems, "solves_per_step": solves_per_step,
        "order": "systems in sequence order; after the last one the sequence restarts from an empty space",
        "precision": args.precision, "precond": "block_jacobi3", "recycle": "srks", "ritz_eps": args.ritz_eps,
        "theta_frac": args.theta_frac, "max_aug": args.max_aug, "reselect": args.reselect, "tol": TOL,
        "reorth": "full", "exec": args.exec, "parallelism": f"{world} independent sequence(s), one per GPU",
        "l2": l2}


def alg_counts(N, precond_bytes_per_dof, m, nc, passes=1, m2=None):
    """Algorithmic FP64 flops and bytes of the iteration kernel over m iterations with
    augmentation size nc: every array counted once per phase that needs it -- the operator
    product 76 bytes and 18 flops per block, the updates and the preconditioner O(n), the two
    projection products 8 n nc bytes each, the reorthogonalisation 16 n (j + 1) bytes at
    iteration j of its pass; the last iteration of a pass stops after the convergence test.
    One pass by default; for the refinement precisions, `passes` passes whose iteration
    counts sum to m and whose squares sum to m2."""
    s = P.sizes(N)
    n, nb, nodes = s["n"], s["nb"], s["free_nodes"]
    if m <= 0:
        return 0.0, 0.0
    if m2 is None:
        m2 = float(m) * m
    # P1-P2 (every iteration): SpMV, (w,q), (r,w), x/r update, (r,r), M^-1 r, (AC)^T u
    f12 = 18 * nb + 4 * n + 6 * n + 6 * n + 2 * n * nc
    b12 = 76 * nb + 4 * (nodes + 1) + precond_bytes_per_dof * n + 8 * n * nc + 48 * n
    # P4-P7 (all but the last of each pass): s = G^-1 t, z = u - C s, (r,z), g = (AW)^T z,
    # w = z - W g; sum over the passes of sum_{j < m_p - 1} (j + 1) = (m2 - m) / 2
    k = m - passes
    sj = (m2 - m) / 2.0
    f47 = k * (2 * nc * nc + 2 * n * nc + 2 * n) + 4 * n * sj
    b47 = k * (8 * n * nc + 16 * n) + 16 * n * sj
    return m * f12 + f47, m * b12 + b47


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("krs_device.cuh", "krs_apcg.cu")  # everything k_apcg_persistent is built from


def csrc_digest():
    """Digest of the persistent kernel's sources: a profile taken on other sources is stale."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_fields(path):
    """`key: value` list items of a profile summary (markdown)."""
    vals = {}
    with open(path) as fh:
        for line in fh:
            item = line.strip().lstrip("-* ").strip()
            if ":" in item and not item.startswith("|"):
                k, v = item.split(":", 1)
                k = k.strip().strip("`")
                if k.replace("_", "").isalnum():
                    vals[k] = v.strip().strip("`")
    return vals


def profiled_traffic(precision, problem, N):
    """DRAM traffic of the persistent kernel from the committed ncu summaries: the summary
    whose captured launch is of this precision, problem and cube size, taken on the current
    kernel sources.  Returns (DRAM bytes / algorithmic bytes of the captured launch, the
    capture's description, file) or (None, None, None) when no summary matches."""
    if not os.path.isdir(PROFILES):
        return None, None, None
    for f in sorted(os.listdir(PROFILES)):
        if not f.endswith(".md"):
            continue
        v = profile_fields(os.path.join(PROFILES, f))
        if v.get("kernel") != "k_apcg_persistent":
            continue
        if (v.get("precision"), v.get("problem"), v.get("N")) != (precision, problem, str(N)):
            continue
        if v.get("csrc_sha256") != csrc_digest():
            continue
        try:
            ratio = float(v["traffic_bytes_per_launch"]) / float(v["algorithmic_bytes_per_launch"])
        except (KeyError, ValueError, ZeroDivisionError):
            continue
        desc = (f"{v.get('problem')} N={v.get('N')} {v.get('precision')}, captured launch: "
                f"m = {v.get('iterations')}, n_c = {v.get('n_c')}")
        return ratio, desc, f"profiles/{f}"
    return None, None, None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.proc = None
        self.path = None
        if not enabled:
            return
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="krs_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [nm for i, nm in enumerate(names) if any(r[5 + i].lower().startswith("active") for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_index_of(local):
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            return int(cvd.split(",")[local])
        except (ValueError, IndexError):
            pass
    return local


# ----------------------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------------------

def roofline_of(args, stats, t_step_ms, precision, hbm_peak, hbm_kind):
    """Roofline object of the persistent iteration kernel over the solves `stats`: its
    algorithmic FP64 flops and bytes (alg_counts) / its event-timed duration."""
    flops = byts = t_iter = 0.0
    refine = precision in ("mixed_ir", "mixed_proj")
    for st in stats:
        if refine:  # the passes of the refinement, FP32 directions: half the value bytes
            f, bb = alg_counts(args.N, 24, st["m"], st["n_c"], max(1, st["outer_iters"]), st["inner_m2"])
            bb *= 0.5
        else:
            f, bb = alg_counts(args.N, 24, st["m"], st["n_c"])
        flops += f
        byts += bb
        t_iter += st["t_iter_ms"]
    launches = sum(1 for st in stats if st["m"] > 0)
    tflops = flops / (t_iter / 1e3) / 1e12 if t_iter > 0 else 0.0
    gbs = byts / (t_iter / 1e3) / 1e9 if t_iter > 0 else 0.0
    ratio, desc, pfile = profiled_traffic(precision, args.problem, args.N)
    per_launch = byts / launches if launches else 0.0
    traffic = {"traffic": ratio * per_launch if ratio else None,
               "traffic_rule": (f"DRAM/algorithmic bytes {ratio:.3f} of the ncu capture in {pfile} ({desc}) x the "
                                "timed launches' mean algorithmic bytes per launch" if ratio else
                                "null: no ncu summary of this kernel, precision and workload on the current sources"),
               "alg_bytes_per_launch": per_launch}
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "peak_kind": hbm_kind,
           "what": "algorithmic bytes of the iteration kernel / its time"}
    fp64 = {"achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tflops / FP64_PEAK_TFLOPS,
            "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz"}
    if precision == "double_float":
        # the streams run on the FP32 pipes: memory is the bound
        r = {"kernel": "k_apcg_persistent<PrecE>", "bound": "hbm", **hbm, **traffic,
             "fp64_view": dict(fp64, what="FP64-equivalent algorithmic flops / time (part of them on FP32 pipes)")}
    elif refine:
        # FP32 passes: memory is the bound; bytes counted per pass (stats: m, passes, sum m_p^2)
        r = {"kernel": "k_apcg_persistent<PrecF>", "bound": "hbm", **hbm, **traffic,
             "what": "half the FP64 algorithmic bytes of the inner passes (FP32 values) / iteration kernel time"}
    else:
        r = {"kernel": "k_apcg_persistent", "bound": "alu", **fp64,
             "flops": "FP64 algorithmic flops of the iterations" if precision == "fp64" else
                      "FP64-equivalent flops of the iterations (mixed-precision passes)",
             **traffic, "hbm_view": hbm}
    r.update({"launches": launches, "share_of_step_time": t_iter / t_step_ms if t_step_ms > 0 else None,
              "timing": "CUDA events recorded by the library around each launch, on its stream"})
    return r, hbm


def run_krs(args, rank, world, local):
    import torch
    from paper_1301_7530_gb300 import binding as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    mats, bs = workload(args.N, args.systems, rank, args.problem)
    n = mats[0].n
    fixed_A = args.problem == "inclusions"
    uniq = mats[:1] if fixed_A else mats
    dmats = [{"row_ptr": torch.as_tensor(A.row_ptr, device=dev), "col_idx": torch.as_tensor(A.col_idx, device=dev),
              "values": torch.as_tensor(A.vals, device=dev).reshape(-1)} for A in uniq]
    b_ds = [torch.as_tensor(bk, device=dev) for bk in bs]
    x_d = torch.zeros(n, dtype=torch.float64, device=dev)

    def policy(precision):
        return B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                             max_aug=args.max_aug, max_iter=args.max_iter, exec=args.exec, precision=precision,
                             reselect=args.reselect, inner_tol=args.inner_tol)

    pol = policy(args.precision)
    seq = B.Sequence(n, device=local, stream=stream)
    # matrix versions: the fixed matrix keeps one version for the whole run; the damage
    # sequence's k-th matrix has its own
    ver_of = (lambda k: 1) if fixed_A else (lambda k: k + 1)
    mat_of = (lambda k: dmats[0]) if fixed_A else (lambda k: dmats[k])

    if args.capture_one:
        cap = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                            max_aug=args.max_aug, max_iter=args.capture_one, exec=args.exec,
                            precision=args.precision, reselect=args.reselect)
        if args.capture_nc > 0:
            rng = np.random.default_rng(777)
            seq.import_space(rng.random((n, args.capture_nc)) - 0.5)
        _, st = seq.solve(mat_of(0), b_ds[0], TOL, cap, x=x_d, version=ver_of(0), raise_on_error=False)
        torch.cuda.synchronize()
        f, bb = alg_counts(args.N, 24, st["m"], st["n_c"])
        print(json.dumps({"capture_one": True, "problem": args.problem, "N": args.N, "precision": args.precision,
                          "status": st["status"], "m": st["m"], "n_c": st["n_c"], "alg_bytes": bb, "alg_flops": f,
                          "t_iter_ms": st["t_iter_ms"], "csrc_sha256": csrc_digest()}))
        seq.close()
        return

    counter = {"step": 0}

    keep_x = {}  # FP64 results of the sequence's first systems (the mixed-precision sample's reference)
    mixed_ks = list(range(min(args.mixed_systems, args.systems))) if args.problem == "inclusions" else []

    def one_step(record=None, lat=None, sq=None, pl=None):
        sq = sq or seq
        pl = pl or pol
        for k in step_systems(args, counter["step"]):
            if k == 0:
                sq.import_space(np.zeros((n, 0)))
            t0 = time.perf_counter()
            _, st = sq.solve(mat_of(k), b_ds[k], TOL, pl, x=x_d, version=ver_of(k))
            if lat is not None:
                lat.append((time.perf_counter() - t0) * 1e3)
            if st["status"] != 0:
                raise RuntimeError(f"solve {k} failed: {st}")
            if record is not None:
                record.append(dict(st, system=k))
                if k in mixed_ks and k not in keep_x:
                    keep_x[k] = x_d.clone()  # 6.5 MB device copy, microseconds
        counter["step"] += 1

    gpu_index = gpu_index_of(local)
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    C_warm = seq.export_space()  # the recycled space the first timed step starts from
    first_timed = counter["step"]
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index, enabled=not args.no_clocks)
    stats, lat = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        one_step(stats, lat)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = all_max(ms, world)
    solves = len(stats)
    total_solves = all_sum(solves, world)
    value = total_solves / (ms_max / 1e3)
    hbm_peak, hbm_kind = measured_peaks()
    roof, hbm = roofline_of(args, stats, ms, args.precision, hbm_peak, hbm_kind)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region:
    # the systems of the first timed steps again, from the same recycled space; the matrix
    # is uploaded by the first of them (a new matrix version), every b and x crosses each step
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        pin = []
        for A in uniq:
            rp = torch.as_tensor(A.row_ptr).pin_memory()
            ci = torch.as_tensor(A.col_idx).pin_memory()
            vv = torch.as_tensor(A.vals).pin_memory()
            pin.append(P.BSR3(rp.numpy(), ci.numpy(), vv.numpy()))
        b_hs = [torch.as_tensor(bk).pin_memory().numpy() for bk in bs]
        x_h = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
        ks = []
        for i in range(args.e2e_steps):
            ks += step_systems(args, first_timed + i)
        seq.import_space(C_warm)
        vbase = 1000
        barrier(world)
        torch.cuda.synchronize()
        h2d = 0
        t0 = time.perf_counter()
        for idx, k in enumerate(ks):
            if k == 0:
                seq.import_space(np.zeros((n, 0)))
            A_h = pin[0] if fixed_A else pin[k]
            ver = vbase if fixed_A else vbase + k
            if idx == 0 or not fixed_A:
                h2d += 4 * (A_h.n_block_rows + 1) + 4 * A_h.nnzb + 72 * A_h.nnzb
            h2d += 8 * n
            _, st = seq.solve(A_h, b_hs[k], TOL, pol, x=x_h, version=ver)
            if st["status"] != 0:
                raise RuntimeError(f"e2e solve {k} failed: {st}")
        torch.cuda.synchronize()
        e_ms = all_max((time.perf_counter() - t0) * 1e3, world)
        e_solves = all_sum(len(ks), world)
        dev_same = float(np.sum(lat[:len(ks)])) / 1e3  # the same systems in the timed region
        e2e = {"value": e_solves / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / args.e2e_steps), "d2h_bytes_per_step": int(8 * n * len(ks) / args.e2e_steps),
               "steps": args.e2e_steps, "systems": ks,
               "device_resident_same_systems": {"value": len(ks) / dev_same, "unit": UNIT,
                                                "what": "the same systems in the timed region (inputs on the device)"},
               "what": "krs_solve with pinned host A, b and x (A uploaded by the first solve, b and x every "
                       "solve), from the recycled space the timed region started from; wall clock.  These are the "
                       "first timed steps' systems, not the timed region's mix (which includes a first system of "
                       "the sequence): compare with device_resident_same_systems"}

    def df_sample():
        """The first timed systems again in the double-float precision, from the same space."""
        seq.import_space(C_warm)
        pdf = policy("double_float")
        vstats, vlat = [], []
        torch.cuda.synchronize()
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        ks = []
        for i in range(args.variant_systems):
            ks += step_systems(args, first_timed + i)
        for k in ks:
            if k == 0:
                seq.import_space(np.zeros((n, 0)))
            t0 = time.perf_counter()
            _, st = seq.solve(mat_of(k), b_ds[k], TOL, pdf, x=x_d, version=ver_of(k) + 2000)
            vlat.append((time.perf_counter() - t0) * 1e3)
            if st["status"] != 0:
                raise RuntimeError(f"double-float solve {k} failed: {st}")
            vstats.append(dict(st, system=k))
        v1.record(stream)
        torch.cuda.synchronize()
        vms = v0.elapsed_time(v1)
        vroof, _ = roofline_of(args, vstats, vms, "double_float", hbm_peak, hbm_kind)
        fp64_same = lat[:len(ks)]
        return {
            "precision": "double_float", "dtype": dtype_of("double_float"), "systems": ks,
            "value": len(ks) / (vms / 1e3), "unit": UNIT, "ms_per_system": vms / len(ks),
            "fp64_ms_per_system_same_systems": float(np.sum(fp64_same) / len(fp64_same)),
            "m": [st["m"] for st in vstats], "fp64_m": [st["m"] for st in stats[:len(ks)]],
            "true_rel_res_max": float(max(st["true_rel_res"] for st in vstats)),
            "roofline": vroof, "gpu_launches": int(sum(st["kernel_launches"] for st in vstats)),
            "what": "a bounded sample: the first timed systems again from the same recycled space, precision "
                    "KRS_DOUBLE_FLOAT (FP64 recurrences, projection and coarse solve; double-float directions "
                    "and matrix values)"}

    def mixed_sample():
        """The sequence's first systems in KRS_MIXED_IR (FP32 passes, FP64 flexible-CG outer
        step) from an empty space, against FP64's time and result on the same systems."""
        seq.release(B.RELEASE_SCRATCH)  # the FP64 direction storage makes room for the FP32 passes'
        seq.import_space(np.zeros((n, 0)))
        pmx = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                            max_aug=args.max_aug, max_iter=16000, exec=args.exec, precision="mixed_ir",
                            inner_tol=args.mixed_inner_tol)
        mstats, mdiff = [], []
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        for k in mixed_ks:
            _, st = seq.solve(mat_of(k), b_ds[k], TOL, pmx, x=x_d, version=ver_of(k) + 3000)
            if st["status"] != 0:
                raise RuntimeError(f"mixed-precision solve {k} failed: {st}")
            mstats.append(dict(st, system=k))
            mdiff.append(float(torch.linalg.norm(x_d - keep_x[k]) / torch.linalg.norm(keep_x[k])))
        m1.record(stream)
        torch.cuda.synchronize()
        mms = m0.elapsed_time(m1)
        fp64_ms = [lt for st, lt in zip(stats, lat) if st["system"] in mixed_ks][:len(mixed_ks)]
        mroof, _ = roofline_of(args, mstats, mms, "mixed_ir", hbm_peak, hbm_kind)
        return {
            "precision": "mixed_ir", "dtype": dtype_of("mixed_ir"), "systems": mixed_ks,
            "inner_tol": args.mixed_inner_tol or 0.1,
            "value": len(mixed_ks) / (mms / 1e3), "unit": UNIT, "ms_per_system": mms / len(mixed_ks),
            "fp64_ms_per_system_same_systems": float(np.mean(fp64_ms)) if fp64_ms else None,
            "inner_iterations": [st["m"] for st in mstats], "passes": [st["outer_iters"] for st in mstats],
            "inner_m_first": [st["inner_m_first"] for st in mstats], "n_c": [st["n_c"] for st in mstats],
            "n_selected": [st["n_selected"] for st in mstats],
            "fp64_m": [st["m"] for st in stats if st["system"] in mixed_ks][:len(mixed_ks)],
            "true_rel_res_max": float(max(st["true_rel_res"] for st in mstats)),
            "rel_diff_from_fp64_result": mdiff,
            "roofline": mroof, "gpu_launches": int(sum(st["kernel_launches"] for st in mstats)),
            "what": "the sequence's first systems from an empty space in KRS_MIXED_IR: FP32 operator, "
                    "preconditioner, projection and reorthogonalisation in the passes, FP64 flexible-CG outer "
                    "step, residual, coarse Cholesky and Ritz eigensolve; rel_diff_from_fp64_result is each "
                    "result's relative difference from the FP64 solve of the same system in the timed region "
                    "(both at relative residual 1e-8)"}

    # extra objects: never allowed to take the headline line down
    extra = {}
    variants = not args.no_variant and args.precision == "fp64" and args.problem == "inclusions"
    for name, fn, on in (("double_float", df_sample, variants and args.variant_systems > 0),
                         ("mixed_ir", mixed_sample, variants and bool(mixed_ks) and all(k in keep_x for k in mixed_ks))):
        if on:
            try:
                extra[name] = fn()
            except Exception as exc:  # noqa: BLE001
                extra[name] = {"error": f"{type(exc).__name__}: {exc}"}
    seq.close()
    keep_x.clear()
    if variants:
        try:
            extra["cube32_damage_sequence"] = damage_line(args, rank, world, local, hbm_peak, hbm_kind)
        except Exception as exc:  # noqa: BLE001
            extra["cube32_damage_sequence"] = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, mats[0], bs, stats)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(args.precision), "data": "synthetic",
            "config": make_config(args, mats[0], world),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat)), "what": "per solve, host clock around krs_solve"},
            "solves": {"count": solves, "systems": [st["system"] for st in stats],
                       "m": [st["m"] for st in stats], "n_c": [st["n_c"] for st in stats],
                       "n_selected": [st["n_selected"] for st in stats],
                       "m_mean": float(np.mean([s["m"] for s in stats])),
                       "n_c_max": int(max(s["n_c_after"] for s in stats)),
                       "true_rel_res_max": float(max(s["true_rel_res"] for s in stats)),
                       "t_setup_ms_mean": float(np.mean([s["t_setup_ms"] for s in stats])),
                       "t_iter_ms_mean": float(np.mean([s["t_iter_ms"] for s in stats])),
                       "t_recycle_ms_mean": float(np.mean([s["t_recycle_ms"] for s in stats])),
                       "profile_check": profile_check(args, stats)},
            "roofline": roof,
            "hbm": hbm,
            "e2e": e2e,
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        out.update(extra)
        print(json.dumps(out))


def profile_check(args, stats):
    """Largest difference between the timed systems' iteration counts and the recorded
    profile the CPU cost model of --impl reference uses."""
    if args.problem != "inclusions" or SEQ64_PROFILE is None or args.N != 64:
        return None
    d = [abs(st["m"] - SEQ64_PROFILE[st["system"]][0]) for st in stats]
    return {"max_abs_m_diff": int(max(d)), "max_rel_m_diff": float(max(
        abs(st["m"] - SEQ64_PROFILE[st["system"]][0]) / max(1, SEQ64_PROFILE[st["system"]][0]) for st in stats))}


def damage_line(args, rank, world, local, hbm_peak, hbm_kind, steps=2, warmup=1):
    """The 32^3 damage sequence in FP64 (20 systems per step, device-resident matrices): a
    smaller workload with many short solves, where the fixed per-iteration work and the work
    between solves weigh more."""
    import torch
    from paper_1301_7530_gb300 import binding as B
    d = argparse.Namespace(**vars(args))
    d.problem, d.N, d.systems, d.max_aug, d.max_iter, d.step_unit = "damage", 32, 20, 200, 2000, "sequence"
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    mats, bs = workload(d.N, d.systems, rank, "damage")
    n = mats[0].n
    dmats = [{"row_ptr": torch.as_tensor(A.row_ptr, device=dev), "col_idx": torch.as_tensor(A.col_idx, device=dev),
              "values": torch.as_tensor(A.vals, device=dev).reshape(-1)} for A in mats]
    b_d = torch.as_tensor(bs[0], device=dev)
    x_d = torch.zeros(n, dtype=torch.float64, device=dev)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac, max_aug=200,
                        max_iter=2000, exec=args.exec, precision="fp64")
    seq = B.Sequence(n, device=local, stream=stream)
    stats, lat = [], []

    def seq_step(record):
        seq.import_space(np.zeros((n, 0)))
        for k, Ad in enumerate(dmats):
            t0 = time.perf_counter()
            _, st = seq.solve(Ad, b_d, TOL, pol, x=x_d, version=k + 1)
            if st["status"] != 0:
                raise RuntimeError(f"32^3 solve {k} failed: {st}")
            if record:
                lat.append((time.perf_counter() - t0) * 1e3)
                stats.append(st)

    for _ in range(warmup):
        seq_step(False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        seq_step(True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    seq.close()
    roof, hbm = roofline_of(d, stats, ms, "fp64", hbm_peak, hbm_kind)
    return {"workload": workload_name(d), "precision": "fp64", "value": len(stats) / (ms / 1e3), "unit": UNIT,
            "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "m_mean": float(np.mean([st["m"] for st in stats])),
            "true_rel_res_max": float(max(st["true_rel_res"] for st in stats)),
            "roofline": roof, "gpu_launches": int(sum(st["kernel_launches"] for st in stats))}


# ----------------------------------------------------------------------------------------
# the oracle: cpu_baseline of the GPU arm, and the reference arm
# ----------------------------------------------------------------------------------------
#
# The FP64 oracle (OpenMP timing build, all host cores) cannot run a system of the 64^3
# sequence in a bounded time (4,000 iterations over up to 4,000 stored directions, then a
# dense cyclic-Jacobi eigensolve of order m).  It is timed on bounded samples of the same
# system and the whole solve is extrapolated by this cost model of its own loops:
#   T(n_c, m, s) = T_set(n_c) + m c_fix + c_col (m n_c + m (m + 1) / 2)
#                  + T_eig(m) + T_eig'(m - 1) + s m c_col / 2
#   T_set(n_c)   = t_pre + n_c (t_spmv + c_col) + n_c^2 t_dot   (AC, C^T A C, x0 / r0)
#   c_fix        per-iteration work that does not depend on the stored columns (operator
#                product, preconditioner, updates, dot products);
#   c_col        one stored column in one iteration: a dot product and an update over n;
#   T_eig(m)     the Lanczos matrix's eigenpairs (and T_eig' its leading block's values),
#                t_eig(m_cal) (m / m_cal)^p with p fitted between two calibration orders.
# Samples: (1) empty space, I iterations; (2) a seeded space of N_COL columns, I iterations
# (both NO_CONVERGENCE by construction); (3) one operator product; (4) the eigensolver at
# two orders.  c_col = (loop_2 - loop_1) / (I N_COL), c_fix from loop_1, t_dot from the
# set-up difference of (2) and (1).

CAL_ITERS = 8
CAL_COLS = 48
CAL_EIG = (300, 600)


def _omp_oracle():
    import oracle as O
    try:
        O.build_omp()
        return O, True
    except Exception:  # noqa: BLE001 -- no OpenMP toolchain: time the parity build
        return O, False


def oracle_calibrate(A, b, eig=True):
    """Constants of the cost model from bounded samples of the oracle on A, b."""
    O, omp = _omp_oracle()
    pol = O.make_policy("none", "block_jacobi3", max_iter=CAL_ITERS)
    t = {}
    s1 = O.Sequence(A.n, omp=omp)
    x, st = s1.solve(A, b, TOL, pol)
    t_set1, loop1, _ = s1.times()
    m1 = st["m"]
    rng = np.random.default_rng(12345)
    C = rng.random((A.n, CAL_COLS)) - 0.5
    s2 = O.Sequence(A.n, omp=omp)
    s2.set_C(C)
    x, st2 = s2.solve(A, b, TOL, pol)
    t_set2, loop2, _ = s2.times()
    m2 = st2["m"]
    del s1, s2
    xs = rng.random(A.n)
    sp = []
    for _ in range(3):
        t0 = time.perf_counter()
        O.spmv(A, xs, omp=omp)
        sp.append(time.perf_counter() - t0)
    t_spmv = float(np.median(sp))
    c_col = max(0.0, (loop2 / max(m2, 1) - loop1 / max(m1, 1)) / CAL_COLS)
    c_fix = max(0.0, (loop1 - c_col * m1 * (m1 + 1) / 2.0) / max(m1, 1))
    t_dot = max(0.0, (t_set2 - t_set1 - CAL_COLS * (t_spmv + c_col)) / CAL_COLS ** 2)
    t.update({"t_pre": t_set1, "c_fix": c_fix, "c_col": c_col, "t_spmv": t_spmv, "t_dot": t_dot,
              "threads": O.num_threads(omp), "omp": omp})
    if eig:
        te = []
        for m in CAL_EIG:
            r2 = np.random.default_rng(m)
            d, e = O.lanczos(r2.uniform(0.2, 3.0, m), np.cumprod(r2.uniform(0.3, 1.2, m)))
            t0 = time.perf_counter()
            O.tridiag_eig(d, e, True, omp=omp)
            O.tridiag_eig(d[:-1], e[:-1], False, omp=omp)
            te.append(time.perf_counter() - t0)
        p = math.log(te[1] / te[0]) / math.log(CAL_EIG[1] / CAL_EIG[0]) if te[0] > 0 and te[1] > 0 else 3.0
        t.update({"t_eig_cal": te[1], "m_eig_cal": CAL_EIG[1], "eig_exponent": min(4.0, max(3.0, p))})
    return t


def oracle_sample_fixed(A, b, cal):
    """Re-measure the column-independent terms (t_pre, c_fix) on one bounded sample of the
    system A x = b (empty space, CAL_ITERS iterations), keeping the other constants."""
    O, omp = _omp_oracle()
    s1 = O.Sequence(A.n, omp=omp)
    x, st = s1.solve(A, b, TOL, O.make_policy("none", "block_jacobi3", max_iter=CAL_ITERS))
    t_set1, loop1, _ = s1.times()
    m1 = max(st["m"], 1)
    out = dict(cal)
    out["t_pre"] = t_set1
    out["c_fix"] = max(0.0, (loop1 - cal["c_col"] * m1 * (m1 + 1) / 2.0) / m1)
    return out


def oracle_model_seconds(cal, n_c, m, s):
    """Modelled oracle seconds of one solve (n_c columns at the start, m iterations, s
    vectors selected), split into (set-up, iterations, recycling)."""
    t_set = cal["t_pre"] + n_c * (cal["t_spmv"] + cal["c_col"]) + n_c * n_c * cal["t_dot"]
    t_it = m * cal["c_fix"] + cal["c_col"] * (m * n_c + m * (m + 1) / 2.0)
    t_rec = 0.0
    if m >= 2:
        t_rec = cal["t_eig_cal"] * (m / cal["m_eig_cal"]) ** cal["eig_exponent"] + s * m * cal["c_col"] / 2.0
    return t_set, t_it, t_rec


def cpu_baseline(args, A, bs, stats):
    """The oracle (OpenMP timing build, all host cores) on the same systems as the timed
    region: bounded samples of the sequence's matrix, extrapolated with the cost model to
    the timed solves' own (n_c, m, selected)."""
    t0 = time.perf_counter()
    cal = oracle_calibrate(A, bs[0])
    wall = time.perf_counter() - t0
    parts = np.zeros(3)
    for st in stats:
        parts += oracle_model_seconds(cal, st["n_c"], st["m"], st["n_selected"])
    total = float(parts.sum())
    return {"value": len(stats) / total, "unit": UNIT, "cores": cal["threads"], "kind": "oracle",
            "sample": (f"cost model of the FP64 oracle ({'OpenMP' if cal['omp'] else 'sequential'} build, "
                       f"{cal['threads']} threads) calibrated in {wall:.1f} s on bounded samples of this "
                       f"matrix ({CAL_ITERS} iterations from an empty and a {CAL_COLS}-column space, one "
                       f"operator product, the eigensolver at orders {CAL_EIG}), applied to the {len(stats)} "
                       "timed solves' own (n_c, m, selected)"),
            "model_seconds": {"setup": float(parts[0]), "iterations": float(parts[1]),
                              "recycling": float(parts[2])},
            "calibration": cal}


def oracle_one_solve(mats, b):
    """Seconds of one oracle solve (OpenMP timing build) of mats[0] from an empty space."""
    O, omp = _omp_oracle()
    s = O.Sequence(mats[0].n, omp=omp)
    pol = O.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=200, max_iter=2000)
    t0 = time.perf_counter()
    x, st = s.solve(mats[0], b, TOL, pol)
    return time.perf_counter() - t0, dict(st, threads=O.num_threads(omp))


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle (OpenMP timing build) on the host cores, rank 0
    only.  Each step is a bounded sample of that step's system (the cost-model samples,
    re-measured every step) extrapolated to the whole solve with the sequence's profile;
    warm-up steps also time the eigensolver calibration."""
    if rank != 0:
        return
    if args.problem != "inclusions" or SEQ64_PROFILE is None or args.N != 64 or args.systems != 15:
        print(json.dumps({"impl": "reference", "unavailable": "the cost model has an iteration profile for the "
                                                                "64^3 15-system inclusion sequence only"}))
        return
    mats, bs = workload(args.N, args.systems, 0, args.problem)
    A = mats[0]
    prof = SEQ64_PROFILE
    base = None
    step_ms, wall_ms = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ks = step_systems(args, i)
        if base is None:  # the whole calibration once (first warm-up step)
            base = oracle_calibrate(A, bs[ks[0]])
            cal = base
        else:  # every other step: a bounded sample of its own system
            cal = oracle_sample_fixed(A, bs[ks[0]], base)
        sec = 0.0
        for k in ks:
            m_k, nc_k, s_k = prof[k]
            sec += sum(oracle_model_seconds(cal, nc_k, m_k, s_k))
        if i >= args.warmup:
            step_ms.append(sec * 1e3)
            wall_ms.append((time.perf_counter() - t0) * 1e3)
    total_s = sum(step_ms) / 1e3
    solves = args.steps * len(step_systems(args, 0))
    value = solves / total_s
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": make_config(args, A, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cal["threads"], "kind": "oracle",
                         "sample": (f"each step: the FP64 oracle ({'OpenMP' if cal['omp'] else 'sequential'} "
                                    f"build, {cal['threads']} threads) timed on a bounded sample of that step's "
                                    f"system ({CAL_ITERS} iterations from an empty space: the per-iteration "
                                    "fixed cost), with the per-column, set-up and eigensolver constants "
                                    f"calibrated once ({CAL_ITERS} iterations from a {CAL_COLS}-column space, one "
                                    f"operator product, the eigensolver at orders {CAL_EIG}), extrapolated to "
                                    "the whole solve by the cost model with the sequence's recorded "
                                    "(m, n_c, selected); value and ms_per_step are modelled oracle time, the "
                                    f"samples took {np.mean(wall_ms):.0f} ms of wall clock per timed step"),
                         "calibration": base},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "what": "modelled oracle time per step"},
    }
    print(json.dumps(out))


# ----------------------------------------------------------------------------------------
# many sequences: batched engine and served requests
# ----------------------------------------------------------------------------------------

def _many(args, kind):
    """Clients of the batched / served workload (generated by a spawn pool before any GPU
    call) and the policy."""
    import multiprocessing as mp
    if kind == "batched":
        nseq, nmin, nmax, systems = args.nseq or 256, args.nmin or 16, args.nmax or 40, args.systems_many or 10
    else:
        nseq, nmin, nmax, systems = args.nseq or 64, args.nmin or 12, args.nmax or 48, args.systems_many or 30
    Ns = P.batch_sizes(nseq, nmin, nmax, 4000 if kind == "batched" else 5000)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        from paper_1301_7530_gb300 import serve as S
        clients = S.make_clients(Ns, systems, 7000 if kind == "batched" else 9000, pool=pool)
    return Ns, systems, clients


def _counts_of(r, Ns):
    """Algorithmic (flops, bytes) of one served request: one pass, or the refinement's passes."""
    return alg_counts(int(Ns[r.cid]), 24, r.m, r.n_c, r.passes, r.m2 if r.m2 > 0 else None)


def _flops_of(reqs, Ns):
    return sum(_counts_of(r, Ns)[0] for r in reqs if r.m > 0)


def _reset(clients):
    for c in clients:
        c.seq.import_space(np.zeros((c.n, 0)))
        c.m_prev = 0


def result_errors(args, kind, Ns, systems, clients, reqs, sample):
    """Error of a seeded sample of results against the FP64 oracle: for the `sample`
    smallest sequences, their first and last system, ||x - x_o|| / ||x_o|| where x_o is the
    oracle's solution of the same A^(k) x = b to relative residual 1e-12 (block-Jacobi, no
    augmentation), beside the result's own FP64 residual.  A result at residual tol is within
    about kappa(A) tol of the exact solution."""
    import oracle as O
    seed = 7000 if kind == "batched" else 9000
    dks = P.damage_factors(systems)
    pick = sorted(range(len(clients)), key=lambda i: (clients[i].n, i))[:sample]
    by = {(r.cid, r.k): r for r in reqs}
    rows = []
    for cid in pick:
        A_out, vin, b = P.damage_parts(int(Ns[cid]), seed + cid, seed + 10000 + cid)
        for k in sorted({0, systems - 1}):
            r = by.get((cid, k))
            if r is None or r.x is None or r.status != 0:
                continue
            A = P.damage_matrix(A_out, vin, dks[k])
            xo, so = O.Sequence(A.n).solve(A, b, 1e-12, O.make_policy("none", "block_jacobi3", max_iter=20000))
            x = r.x.cpu().numpy()
            rows.append({"seq": cid, "N": int(Ns[cid]), "system": k, "m": r.m,
                         "rel_err": float(np.linalg.norm(x - xo) / np.linalg.norm(xo)),
                         "true_rel_res": float(r.true_rel_res), "oracle_m": so["m"]})
    errs = [row["rel_err"] for row in rows]
    return {"what": "||x - x_oracle|| / ||x_oracle||, x_oracle the FP64 oracle's solution of the same system "
                    "to relative residual 1e-12; results of the smallest sequences, first and last system",
            "count": len(rows), "max": max(errs) if errs else None,
            "median": float(np.median(errs)) if errs else None, "results": rows}


def run_many(args, kind):
    import torch
    from paper_1301_7530_gb300 import binding as B
    from paper_1301_7530_gb300 import serve as S
    Ns, systems, clients = _many(args, kind)
    B.lib()
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                        max_aug=100, max_iter=1000 if args.precision in ("fp64", "double_float") else 1500,
                        precision=args.precision, inner_tol=args.inner_tol)
    quantum = args.quantum if args.quantum is not None else (0 if kind == "batched" else 32)
    budget = int(args.budget_gb * (1 << 30)) if kind == "served" else int(200 * (1 << 30))
    srv = S.Server(clients, pol, TOL, budget_bytes=budget, group_ctas=args.group_ctas, quantum=quantum,
                   group_scale=args.group_scale)
    # warm-up: system 0 of every sequence (autotuner, allocations), then empty spaces again
    srv.run([(0.0, c.cid, 0) for c in clients], closed_loop=True, n_systems=1)
    _reset(clients)
    bst0 = srv.engine.stats()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device(), enabled=not args.no_clocks)
    t0 = time.perf_counter()
    if kind == "batched":
        reqs = srv.run([(0.0, c.cid, 0) for c in clients], closed_loop=True, n_systems=systems)
    else:
        reqs = srv.run(S.poisson_arrivals(len(clients), systems, args.rate, 11))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    bst = srv.engine.stats()
    summ = S.latency_summary(reqs)
    kern_ms = bst["total_kernel_ms"] - bst0["total_kernel_ms"]
    flops = _flops_of(reqs, Ns)
    ach = flops / (kern_ms / 1e3) / 1e12 if kern_ms > 0 else 0.0
    byts = sum(_counts_of(r, Ns)[1] for r in reqs if r.m > 0)
    hbm_peak, hbm_kind = measured_peaks()
    gbs = 0.5 * byts / (kern_ms / 1e3) / 1e9 if kern_ms > 0 else 0.0
    value = len(reqs) / wall
    srv.close()
    errors = result_errors(args, kind, Ns, systems, clients, reqs, args.check_sample) if args.check_sample > 0 else None
    # per-solve launches (krs_solve, one full-device persistent launch per solve) on the
    # same sequences: the reference point the batched / served form must beat
    nb = args.baseline_seqs or len(clients)
    _reset(clients)
    base_clients = clients[:nb]
    el, breqs = S.solve_alone(base_clients, pol, TOL)
    base_value = len(breqs) / el
    cpu = None
    if not args.no_cpu_baseline:
        c0 = min(clients, key=lambda c: c.n)
        from paper_1301_7530_gb300 import problems as PP
        A_out, vin, b = PP.damage_parts(int(Ns[c0.cid]), (7000 if kind == "batched" else 9000) + c0.cid,
                                        (7000 if kind == "batched" else 9000) + 10000 + c0.cid)
        sec, st = oracle_one_solve([PP.damage_matrix(A_out, vin, 1.0)], b)
        cpu = {"value": 1.0 / sec, "unit": UNIT, "cores": st["threads"], "kind": "oracle",
               "sample": f"one oracle solve of the smallest sequence's first system (n = {c0.n}, m = {st['m']}), "
                         f"{st['threads']} threads: {sec:.2f} s"}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": systems, "warmup": 1,
        "ms_per_step": wall * 1e3 / systems, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_of(args.precision), "data": "synthetic", "impl": "krs",
        "workload_kind": kind,
        "config": {
            "workload": (f"{len(clients)} damage sequences x {systems} systems, cubes N ~ U{{{min(Ns)}..{max(Ns)}}}"
                         if kind == "batched" else
                         f"{len(clients)} clients x {systems} damage systems, Poisson {args.rate}/s total, "
                         f"cubes N ~ U{{{min(Ns)}..{max(Ns)}}}, budget {args.budget_gb} GB"),
            "total_dofs": int(sum(c.n for c in clients)), "recycle": "srks", "ritz_eps": args.ritz_eps,
            "theta_frac": args.theta_frac, "max_aug": 100, "tol": TOL, "precond": "block_jacobi3",
            "precision": args.precision, "inner_tol": args.inner_tol or None,
            "group_ctas": args.group_ctas or "per solve", "group_scale": bst["tuned_group_scale"] or args.group_scale,
            "quantum": quantum, "autotune": bst["tune"], "l2": "inputs larger than L2 (every sequence's matrices resident)"},
        "latency_ms": {"p50": summ["p50_ms"], "p99": summ["p99_ms"], "mean": summ["mean_ms"],
                       "what": "result returned - request arrival (host clock)"},
        "per_solve_launches": {"value": base_value, "unit": UNIT, "sequences": nb,
                               "what": "the same solves with krs_solve, one full-device launch each"},
        "speedup_vs_per_solve": value / base_value,
        "solves": {"count": len(reqs), "failed": summ["failed"], "true_rel_res_max": summ["max_true_rel_res"],
                   "iterations": int(sum(r.m for r in reqs)),
                   "iterations_per_solve_path": int(sum(r.m for r in breqs))},
        "roofline": ({"kernel": "k_apcg_batched", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                      "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                      "kernel_ms": kern_ms, "share_of_wall": kern_ms / (wall * 1e3)}
                     if args.precision == "fp64" else
                     {"kernel": "k_apcg_batched<PrecE>", "bound": "hbm", "achieved": 2.0 * gbs, "peak": hbm_peak,
                      "unit": "GB/s", "frac": 2.0 * gbs / hbm_peak, "traffic": None,
                      "what": "FP64 algorithmic bytes of all iterations (double-float directions: 8 bytes each) / "
                              "batched kernel time", "kernel_ms": kern_ms, "share_of_wall": kern_ms / (wall * 1e3)}
                     if args.precision == "double_float" else
                     {"kernel": "k_apcg_batched (FP32 passes)", "bound": "hbm", "achieved": gbs,
                      "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "traffic": None,
                      "what": "half the FP64 algorithmic bytes of all inner iterations (FP32 storage) / "
                              "batched kernel time", "kernel_ms": kern_ms, "share_of_wall": kern_ms / (wall * 1e3)}),
        "hbm_peak": {"value": hbm_peak, "kind": hbm_kind},
        "result_errors": errors,
        "server": {"steps": srv.steps, "evictions": srv.evictions, "reimports": srv.reimports,
                   "peak_held_gb": srv.peak_held / 2 ** 30},
        "e2e": None,
        "gpu_launches": int(bst["kernel_launches"] - bst0["kernel_launches"] + sum(r.launches for r in reqs)),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out))
    for c in clients:
        c.close()


def run_conditioning(args):
    """Condition numbers of the inclusion cube's matrix (the quantity that decides whether
    FP32 inner solves can drive an FP64 refinement): kappa(M^-1 A) for the block-Jacobi
    preconditioner from the extreme Ritz values of one tight preconditioned solve (random
    right-hand side), lambda_max(A) by scipy's Lanczos on the host, lambda_min(A) as
    1 / lambda_max(A^-1) by a Lanczos process on A^-1 whose products are library solves
    (block-Jacobi, relative residual 1e-9, TRKS reuse of the earlier solves' directions)."""
    import scipy.sparse.linalg as sla
    import torch
    from paper_1301_7530_gb300 import binding as B
    torch.cuda.set_device(0)
    N = args.N
    A = P.elasticity_inclusions(N, 3000)
    n = A.n
    rng = np.random.default_rng(99)
    t0 = time.perf_counter()
    seq = B.Sequence(n)
    v = rng.standard_normal(n)
    # tolerance 1e-9: CG's recursive residual cannot go much below u kappa(A) (~1e-10 at 48^3)
    _, st = seq.solve(A, v, 1e-9, B.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, max_aug=1, max_iter=12000),
                      version=1)
    th, _, _ = seq.last_ritz()
    kappa_m = float(th[0] / th[-1])
    seq.close()
    lmax = float(sla.eigsh(A.to_scipy(), k=1, which="LA", tol=1e-8, return_eigenvectors=False)[0])
    seq = B.Sequence(n)
    # A^-1 products: solves to 1e-9 recycling (TRKS) at most 1,500 earlier directions, so
    # that each later solve starts deflated and the work stays bounded
    pol = B.make_policy("trks", "block_jacobi3", max_aug=1500, max_iter=12000)
    L = args.lanczos_steps
    Q = np.zeros((n, L + 1))
    q = rng.standard_normal(n)
    Q[:, 0] = q / np.linalg.norm(q)
    al, be = [], []
    for i in range(L):
        w, st2 = seq.solve(A, Q[:, i], 1e-9, pol, version=1)
        a_i = float(Q[:, i] @ w)
        w = w - Q[:, :i + 1] @ (Q[:, :i + 1].T @ w)  # full reorthogonalisation (host, small)
        w = w - Q[:, :i + 1] @ (Q[:, :i + 1].T @ w)
        b_i = float(np.linalg.norm(w))
        al.append(a_i)
        be.append(b_i)
        Q[:, i + 1] = w / b_i
    T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    mu = np.linalg.eigvalsh(T)
    lmin = float(1.0 / mu[-1])
    seq.close()
    out = {"workload": "conditioning", "problem": f"{N}^3 Q1 elasticity with stiff spherical inclusions (5 %, contrast 1e3)",
           "n": n, "kappa_A": lmax / lmin, "lambda_max_A": lmax, "lambda_min_A": lmin,
           "lambda_min_A_change_last_step": float(abs(1.0 / mu[-1] - 1.0 / np.linalg.eigvalsh(T[:-1, :-1])[-1]) / lmin),
           "kappa_MinvA_block_jacobi": kappa_m, "preconditioned_solve_iterations": st["m"],
           "u32": 2.0 ** -24, "kappa_A_u32": lmax / lmin * 2.0 ** -24, "kappa_MinvA_u32": kappa_m * 2.0 ** -24,
           "lanczos_steps": L, "seconds": time.perf_counter() - t0}
    print(json.dumps(out))


def run_fp64peak(args):
    """Measured FP64 rate of this GPU, the co-roof of the FP64 path: torch's FP64 matrix
    product (cuBLAS, 8192^3, 2 N^3 flops), best of 5 after a warm-up, CUDA events, clocks
    sampled meanwhile; beside the derived 152 SMs x 2 FMA/clk x 2 x 2.07 GHz."""
    import torch
    torch.cuda.set_device(0)
    N = 8192
    a = torch.randn(N, N, dtype=torch.float64, device="cuda")
    b = torch.randn(N, N, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index_of(0), enabled=not args.no_clocks)
    times = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    del c
    tf = 2.0 * N ** 3 / (min(times) / 1e3) / 1e12
    print(json.dumps({"workload": "fp64peak", "what": "torch.matmul float64 8192^3 (cuBLAS), best of 5",
                      "tflops": tf, "ms": times, "derived_peak_tflops": FP64_PEAK_TFLOPS,
                      "frac_of_derived": tf / FP64_PEAK_TFLOPS, "clocks": clk}))


def main():
    args = parse_args()
    if args.workload == "conditioning":
        run_conditioning(args)
        return
    if args.workload == "fp64peak":
        run_fp64peak(args)
        return
    if args.impl == "krs" and args.workload != "sequence":
        run_many(args, args.workload)
        return
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        run_reference(args, rank, world)
        return
    rank, world, local = dist_setup()
    run_krs(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
