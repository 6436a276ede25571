#!/usr/bin/env python3
"""Benchmark: solves/s and p50/p99 latency at relative residual 1e-8, and the achieved
throughput of the dominant kernel (the persistent APCG iteration kernel) against its roof.

Workload (one "step"): the 32^3 Q1 elasticity damage sequence -- 20 secant systems on
104,544 FP64 dofs in 3x3 BSR; elements inside a seeded ellipsoid get E * d_k,
d_k = 0.05^(k/19); fixed seeded traction right-hand side; block-Jacobi preconditioner;
SRKS (Algorithm 3) with theta < 0.1 theta_max, at most 200 augmentation vectors, starting
from an empty augmentation space.  All 20 matrices are resident on the device when the
timed region starts (1.35 GB per step, larger than L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl krs|reference]

Multi-GPU (torchrun): every rank solves its own sequence (independent problems, no data
collective); value = all ranks' solves / the slowest rank's time ("weak" scaling).
--impl reference times the FP64 CPU oracle (rank 0 only) on a bounded sample.
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
PROFILE_SUMMARY = {"fp64": os.path.join(ROOT, "profiles", "apcg_persistent_32cube_damage_fp64.md"),
                   "double_float": os.path.join(ROOT, "profiles", "apcg_persistent_32cube_damage_dfloat.md")}


def dtype_of(precision):
    """Arithmetic type of the path: FP64; FP64 with double-float (two-FP32) directions; or
    FP32 inner passes with FP64 refinement."""
    return {"fp64": "f64", "double_float": "f64+df32x2"}.get(precision, "f32+f64")
CSRC = os.path.join(ROOT, "paper_1301_7530_gb300", "csrc")

# FP64 ALU roof of GB300: 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x 2.07 GHz
# (NVIDIA's 1.25 TFLOP/s FP64 figure; the unit count measured 1.9 FMA/clk/SM).
SMS, FP64_FMA_PER_CLK_SM, SM_MAX_MHZ = 152, 2, 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["krs", "reference"], default="krs")
    ap.add_argument("--N", type=int, default=32)
    ap.add_argument("--systems", type=int, default=20)
    ap.add_argument("--systems-many", type=int, default=None, help="batched/served: systems per sequence (10 / 30)")
    ap.add_argument("--exec", choices=["persistent", "kernels"], default="persistent")
    ap.add_argument("--ritz-eps", type=float, default=1e-6)
    ap.add_argument("--theta-frac", type=float, default=0.1)
    ap.add_argument("--max-aug", type=int, default=200)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--max-iter", type=int, default=2000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-variant", action="store_true",
                    help="sequence workload in FP64: skip the double-float line of the same workload")
    ap.add_argument("--precision", choices=["fp64", "double_float", "mixed_ir", "mixed_proj"], default="fp64",
                    help="sequence workload: FP64, FP32 refinement passes, or FP32 projection passes")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed_ir: relative residual of each FP32 pass (0: the library default 0.1)")
    ap.add_argument("--reselect", choices=["none", "cluster"], default="none",
                    help="SRKS cluster reselection (Section 4.4, end)")
    ap.add_argument("--problem", choices=["damage", "inclusions"], default="damage",
                    help="sequence workload: damage sequence (default) or the stiff-inclusion cube")
    ap.add_argument("--workload", choices=["sequence", "batched", "served"], default="sequence",
                    help="sequence: one 32^3 damage sequence (default); batched: many sequences of "
                         "uneven size through the batched engine; served: Poisson requests of many clients")
    ap.add_argument("--nseq", type=int, default=None, help="batched/served: sequences (256 / 64)")
    ap.add_argument("--nmin", type=int, default=None, help="batched/served: smallest cube (16 / 12)")
    ap.add_argument("--nmax", type=int, default=None, help="batched/served: largest cube (40 / 48)")
    ap.add_argument("--rate", type=float, default=200.0, help="served: offered requests per second")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served: device memory budget")
    ap.add_argument("--group-ctas", type=int, default=0, help="batched/served: CTAs per solve (0: autotune)")
    ap.add_argument("--quantum", type=int, default=None, help="batched/served: iterations per launch")
    ap.add_argument("--group-scale", type=int, default=0, help="batched/served: group size scale in percent (0: autotune)")
    ap.add_argument("--baseline-seqs", type=int, default=None,
                    help="batched/served: sequences in the per-solve reference sample (default all)")
    return ap.parse_args()


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

def workload(N, systems, rank, problem="damage"):
    """(matrices, right-hand sides) of the sequence: the damage sequence (one A^(k) per
    system, fixed b), or the inclusion cube (fixed A with seeded stiff spheres, one traction
    draw per system)."""
    if problem == "inclusions":
        A = P.elasticity_inclusions(N, 3000 + rank)
        bs = [P.traction_rhs(N, P.random_traction(N, 3100 + 100 * rank + k)) for k in range(systems)]
        return [A] * systems, bs
    mask, b, gen = P.elasticity_sequence_damage(N, systems, 2000, 2000 + rank)
    mats = [A for _, A in gen]
    return mats, [b] * systems


def alg_counts(N, precond_bytes_per_dof, m, nc):
    """Algorithmic FP64 flops and bytes of one launch of the iteration kernel (m iterations,
    augmentation size nc): every array counted once per phase that needs it -- the operator
    product 76 bytes and 18 flops per block, the updates and the preconditioner O(n), the two
    projection products 8 n nc bytes each, the reorthogonalisation 16 n (j + 1) bytes; the last
    iteration stops after the convergence test."""
    s = P.sizes(N)
    n, nb, nodes = s["n"], s["nb"], s["free_nodes"]
    flops = 0.0
    byts = 0.0
    for j in range(m):
        # P1-P2 (every iteration): SpMV, (w,q), (r,w), x/r update, (r,r), M^-1 r, (AC)^T u
        flops += 18 * nb + 4 * n + 6 * n + 6 * n + 2 * n * nc
        byts += 76 * nb + 4 * (nodes + 1) + precond_bytes_per_dof * n + 8 * n * nc + 48 * n
        if j < m - 1:
            # P4-P7: s = G^-1 t, z = u - C s, (r,z), g = (AW)^T z, w = z - W g
            flops += 2 * nc * nc + 2 * n * nc + 2 * n + 4 * n * (j + 1)
            byts += 8 * n * nc + 16 * n * (j + 1) + 16 * n
    return flops, byts


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


def profiled_traffic(precision="fp64"):
    """DRAM bytes per launch from the committed ncu summary of that precision's persistent
    kernel, if it was taken on the current kernel sources (else None)."""
    path = PROFILE_SUMMARY.get(precision)
    if not path or not os.path.exists(path):
        return None, None
    txt = open(path).read()
    vals = {}
    for line in txt.splitlines():
        item = line.strip().lstrip("-* ").strip()  # markdown list items "- key: `value`"
        if ":" in item and item.startswith(("traffic_bytes_per_launch", "algorithmic_bytes_per_launch",
                                            "csrc_sha256")):
            k, v = item.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("csrc_sha256") != csrc_digest():
        return None, None
    try:
        return float(vals["traffic_bytes_per_launch"]), float(vals["algorithmic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None, None


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


# ----------------------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------------------

def run_krs(args, rank, world, local):
    import torch
    from paper_1301_7530_gb300 import binding as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    mats, bs = workload(args.N, args.systems, rank, args.problem)
    b = bs[0]
    n = mats[0].n
    # device-resident inputs
    dmats = []
    for A in mats:
        dmats.append({"row_ptr": torch.as_tensor(A.row_ptr, device=dev),
                      "col_idx": torch.as_tensor(A.col_idx, device=dev),
                      "values": torch.as_tensor(A.vals, device=dev).reshape(-1)})
    b_ds = [torch.as_tensor(bk, device=dev) for bk in bs]
    x_d = torch.zeros(n, dtype=torch.float64, device=dev)
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                        max_aug=args.max_aug, max_iter=args.max_iter, exec=args.exec, precision=args.precision,
                        reselect=args.reselect)
    seq = B.Sequence(n, device=local, stream=stream)

    def one_step(record=None, lat=None):
        seq.import_space(np.zeros((n, 0)))
        for k, Ad in enumerate(dmats):
            t0 = time.perf_counter()
            ver = 1 if args.problem == "inclusions" else k + 1  # the inclusion cube keeps its A
            _, st = seq.solve(Ad, b_ds[k], TOL, pol, x=x_d, version=ver)
            if lat is not None:
                lat.append((time.perf_counter() - t0) * 1e3)
            if st["status"] != 0:
                raise RuntimeError(f"solve {k} failed: {st}")
            if record is not None:
                record.append(st)

    def timed(steps, warmup, record, lat):
        """warm-up steps, then `steps` steps bracketed by a barrier and synchronisation on both
        sides, CUDA events on the library's stream; returns (ms, clocks)"""
        for _ in range(warmup):
            one_step()
        barrier(world)
        torch.cuda.synchronize()
        clocks = ClockSampler(gpu_index, enabled=not args.no_clocks)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            one_step(record, lat)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return ev0.elapsed_time(ev1), clocks.stop()

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except (ValueError, IndexError):
            gpu_index = local
    stats, lat = [], []
    ms, clk = timed(args.steps, args.warmup, stats, lat)
    ms_max = all_max(ms, world)
    solves = args.steps * args.systems
    total_solves = all_sum(solves, world)
    value = total_solves / (ms_max / 1e3)

    # roofline of the dominant kernel (persistent iteration kernel)
    flops = byts = t_iter = 0.0
    for st in stats:
        f, bb = alg_counts(args.N, 24, st["m"], st["n_c"])
        flops += f
        byts += bb
        t_iter += st["t_iter_ms"]
    launches = sum(1 for st in stats if st["m"] > 0)
    achieved_tflops = flops / (t_iter / 1e3) / 1e12
    achieved_gbs = byts / (t_iter / 1e3) / 1e9
    hbm_peak, hbm_kind = measured_peaks()
    traffic, traffic_alg = profiled_traffic(args.precision)
    iter_share = t_iter / ms

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = []
        for A in mats:
            rp = torch.as_tensor(A.row_ptr).pin_memory()
            ci = torch.as_tensor(A.col_idx).pin_memory()
            vv = torch.as_tensor(A.vals).pin_memory()
            pin.append(P.BSR3(rp.numpy(), ci.numpy(), vv.numpy()))
        b_hs = [torch.as_tensor(bk).pin_memory().numpy() for bk in bs]
        x_h = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
        seq2 = B.Sequence(n, device=local, stream=stream)

        def host_step():
            seq2.import_space(np.zeros((n, 0)))
            for k, A in enumerate(pin):
                ver = 1 if args.problem == "inclusions" else k + 1
                _, st = seq2.solve(A, b_hs[k], TOL, pol, x=x_h, version=ver)
                if st["status"] != 0:
                    raise RuntimeError(f"e2e solve {k} failed: {st}")

        host_step()  # warm-up (allocations)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            host_step()
        torch.cuda.synchronize()
        e_ms = all_max((time.perf_counter() - t0) * 1e3, world)
        e_solves = all_sum(args.e2e_steps * args.systems, world)
        s0 = P.sizes(args.N)
        if args.problem == "inclusions":  # one A for the whole sequence: uploaded before the timed region
            h2d = 8 * n * len(mats)
        else:
            h2d = sum(4 * (A.n_block_rows + 1) + 4 * A.nnzb + 72 * A.nnzb + 8 * n for A in mats)
        d2h = 8 * n * len(mats)
        e2e = {"value": e_solves / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps, "n": s0["n"]}
        seq2.close()

    # the same workload with double-float search directions and matrix values (FP32 pipes)
    variant = None
    if args.precision == "fp64" and not args.no_variant:
        pol = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                            max_aug=args.max_aug, max_iter=args.max_iter, exec=args.exec,
                            precision="double_float", reselect=args.reselect)
        vstats, vlat = [], []
        vms, vclk = timed(args.steps, args.warmup, vstats, vlat)
        vms_max = all_max(vms, world)
        vflops = vbyts = vt_iter = 0.0
        for st in vstats:
            f, bb = alg_counts(args.N, 24, st["m"], st["n_c"])
            vflops += f
            vbyts += bb
            vt_iter += st["t_iter_ms"]
        vgbs = vbyts / (vt_iter / 1e3) / 1e9
        vtraffic, vtraffic_alg = profiled_traffic("double_float")
        variant = {
            "precision": "double_float", "dtype": dtype_of("double_float"),
            "value": all_sum(args.steps * args.systems, world) / (vms_max / 1e3), "unit": UNIT,
            "ms_per_step": vms_max / args.steps,
            "latency_ms": {"p50": float(np.percentile(vlat, 50)), "p99": float(np.percentile(vlat, 99))},
            "m_mean": float(np.mean([st["m"] for st in vstats])),
            "true_rel_res_max": float(max(st["true_rel_res"] for st in vstats)),
            "roofline": {"kernel": "k_apcg_persistent<PrecE>", "bound": "hbm", "achieved": vgbs, "peak": hbm_peak,
                         "unit": "GB/s", "frac": vgbs / hbm_peak, "peak_kind": hbm_kind,
                         "traffic": vtraffic, "traffic_alg_bytes": vtraffic_alg,
                         "share_of_step_time": vt_iter / vms},
            "gpu_launches": int(sum(st["kernel_launches"] for st in vstats)),
            "clocks": vclk,
            "what": "the same 20-system sequence, same warm-up and timing, precision KRS_DOUBLE_FLOAT "
                    "(FP64 recurrences, projection and coarse solve; double-float directions and matrix values)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mats, b)

    mat_bytes = sum(76 * A.nnzb + 4 * (A.n_block_rows + 1) for A in (mats if args.problem == "damage" else mats[:1]))
    l2_note = (f"inputs larger than L2: {len(mats) if args.problem == 'damage' else 1} resident matrices, "
               f"{mat_bytes / 1e9:.2f} GB, plus the direction storage streamed every iteration")
    if rank == 0:
        ms_per_step = ms_max / args.steps
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(args.precision), "data": "synthetic",
            "config": {
                "workload": (f"{args.N}^3 Q1 elasticity damage sequence, {args.systems} systems per step, SRKS"
                             if args.problem == "damage" else
                             f"{args.N}^3 Q1 elasticity with stiff spherical inclusions (5 %, contrast 1e3), "
                             f"{args.systems} traction systems per step, SRKS"),
                "precision": args.precision, "reselect": args.reselect,
                "n": n, "nnzb": mats[0].nnzb, "systems_per_step": args.systems, "precond": "block_jacobi3",
                "recycle": "srks", "ritz_eps": args.ritz_eps, "theta_frac": args.theta_frac,
                "max_aug": args.max_aug, "tol": TOL, "exec": args.exec, "reorth": "full",
                "parallelism": f"{world} independent sequence(s), one per GPU",
                "l2": l2_note},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat))},
            "solves": {"m_mean": float(np.mean([s["m"] for s in stats])),
                       "n_c_mean": float(np.mean([s["n_c"] for s in stats])),
                       "n_c_max": int(max(s["n_c_after"] for s in stats)),
                       "true_rel_res_max": float(max(s["true_rel_res"] for s in stats)),
                       "t_setup_ms_mean": float(np.mean([s["t_setup_ms"] for s in stats])),
                       "t_iter_ms_mean": float(np.mean([s["t_iter_ms"] for s in stats])),
                       "t_recycle_ms_mean": float(np.mean([s["t_recycle_ms"] for s in stats]))},
            "roofline": ({"kernel": "k_apcg_persistent", "bound": "alu", "achieved": achieved_tflops,
                          "flops": "FP64 algorithmic flops of the iterations" if args.precision == "fp64" else
                                   "FP64-equivalent flops of the iterations (mixed-precision passes)",
                          "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                          "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                          "traffic": traffic, "traffic_alg_bytes": traffic_alg,
                          "launches": launches, "share_of_step_time": iter_share}
                         if args.precision != "double_float" else
                         # the reorthogonalisation streams run on the FP32 pipes: memory-bound
                         {"kernel": "k_apcg_persistent<PrecE>", "bound": "hbm", "achieved": achieved_gbs,
                          "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                          "peak_kind": hbm_kind, "what": "algorithmic bytes of the iterations / iteration kernel time",
                          "traffic": traffic, "traffic_alg_bytes": traffic_alg,
                          "launches": launches, "share_of_step_time": iter_share,
                          "fp64_view": {"achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                        "what": "FP64-equivalent algorithmic flops / time (part of them on FP32 pipes)"}}),
            "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                    "peak_kind": hbm_kind, "what": "algorithmic bytes of the iteration kernel / its time"},
            "e2e": e2e,
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if variant is not None:
            out["double_float"] = variant
        print(json.dumps(out))
    seq.close()


# ----------------------------------------------------------------------------------------
# the oracle: cpu_baseline of the GPU arm, and the reference arm
# ----------------------------------------------------------------------------------------

def oracle_one_solve(mats, b):
    import oracle as O
    s = O.Sequence(mats[0].n)
    pol = O.make_policy("srks", "block_jacobi3", ritz_eps=1e-6, theta_frac=0.1, max_aug=200, max_iter=2000)
    t0 = time.perf_counter()
    x, st = s.solve(mats[0], b, TOL, pol)
    return time.perf_counter() - t0, st


def cpu_baseline(mats, b):
    sec, st = oracle_one_solve(mats, b)
    return {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one oracle solve (system 0 of the sequence, empty C, m = {st['m']}) "
                      f"timed single-threaded: {sec:.2f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    mats, bs = workload(args.N, 1, 0, args.problem)
    b = bs[0]
    for _ in range(args.warmup):
        oracle_one_solve(mats, b)
    t0 = time.perf_counter()
    ms_list = []
    for _ in range(args.steps):
        sec, st = oracle_one_solve(mats, b)
        ms_list.append(sec * 1e3)
    total = time.perf_counter() - t0
    value = args.steps / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.N}^3 Q1 elasticity damage sequence, {args.systems} systems per step, SRKS",
                   "n": mats[0].n, "tol": TOL, "precond": "block_jacobi3", "recycle": "srks"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: one FP64 oracle solve of system 0 (empty C, m = {st['m']}), "
                                   "single-threaded"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": float(np.percentile(ms_list, 50)), "p99": float(np.percentile(ms_list, 99))},
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


def _flops_of(reqs, Ns):
    f = 0.0
    for r in reqs:
        if r.m > 0:
            f += alg_counts(int(Ns[r.cid]), 24, r.m, r.n_c)[0]
    return f


def _reset(clients):
    for c in clients:
        c.seq.import_space(np.zeros((c.n, 0)))
        c.m_prev = 0


def run_many(args, kind):
    import torch
    from paper_1301_7530_gb300 import binding as B
    from paper_1301_7530_gb300 import serve as S
    Ns, systems, clients = _many(args, kind)
    B.lib()
    pol = B.make_policy("srks", "block_jacobi3", ritz_eps=args.ritz_eps, theta_frac=args.theta_frac,
                        max_aug=100, max_iter=1000 if args.precision in ("fp64", "double_float") else 800,
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
    byts = sum(alg_counts(int(Ns[r.cid]), 24, r.m, r.n_c)[1] for r in reqs if r.m > 0)
    hbm_peak, hbm_kind = measured_peaks()
    gbs = 0.5 * byts / (kern_ms / 1e3) / 1e9 if kern_ms > 0 else 0.0
    value = len(reqs) / wall
    srv.close()
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
        cpu = {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one oracle solve of the smallest sequence's first system (n = {c0.n}, m = {st['m']}), "
                         f"single-threaded: {sec:.2f} s"}
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


def main():
    args = parse_args()
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
