"""Continuous batching of solve requests over the batched engine (host scheduler).

Clients are sequences of systems (one recycled space each).  A client's request k can
start only after its request k - 1 has returned, because the space it solves with is the
one that solve produced (Algorithms 2 and 3).  The scheduler

  * admits requests into the engine as device memory allows (an estimate of what the solve
    will allocate, against a byte budget that also counts every space held on the device),
  * steps the engine: one launch runs every in-flight solve for at most `quantum`
    iterations, then finished solves are returned and waiting requests admitted, so new
    work joins while other solves are in the middle of their iterations,
  * frees a finished solve's direction storage at once (its space stays resident), and
  * under memory pressure evicts idle clients' spaces to host memory
    (krs_export_space + krs_release) and re-imports them at the client's next request.

Latency of a request = time its result was returned - its arrival time (host clock).
Every solve itself runs in the CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Request:
    cid: int
    k: int
    arrival: float
    t_submit: float = -1.0
    t_done: float = -1.0
    status: int = -1
    m: int = 0
    n_c: int = 0
    true_rel_res: float = float("nan")
    launches: int = 0     # kernels the library launched for this solve outside the batched kernel
    x: object = None
    passes: int = 1       # refinement passes (FP32 inner solves) and the sum of their lengths squared
    m2: float = 0.0
    vals: object = None  # the request's matrix values (device), alive while in flight


class Client:
    """One sequence: its matrices A^(k) = A_out + d_k A_in (device), right-hand side and
    library sequence handle."""

    def __init__(self, cid, A_out, vals_in, b, dks, device=0):
        import torch
        self.cid = cid
        self.n = A_out.n
        self.nbr = A_out.n_block_rows
        self.nnzb = A_out.nnzb
        dev = torch.device("cuda", device)
        self.rp = torch.as_tensor(A_out.row_ptr, dtype=torch.int32, device=dev)
        self.ci = torch.as_tensor(A_out.col_idx, dtype=torch.int32, device=dev)
        self.vals_out = torch.as_tensor(A_out.vals.reshape(-1), dtype=torch.float64, device=dev)
        self.vals_in = torch.as_tensor(np.ascontiguousarray(vals_in).reshape(-1), dtype=torch.float64, device=dev)
        self.b = torch.as_tensor(b, dtype=torch.float64, device=dev)
        self.dks = [float(d) for d in dks]
        self.seq = B.Sequence(self.n, device=device)
        self.queue = collections.deque()
        self.inflight = None
        self.evicted = None  # host copy of the space while evicted
        self.last_done = 0.0
        self.m_prev = 0
        self.nc = 0

    def matrix(self, k):
        vals = self.vals_out + self.dks[k] * self.vals_in
        return {"row_ptr": self.rp, "col_idx": self.ci, "values": vals}, vals

    def close(self):
        self.seq.close()


def _round_up(v, m):
    return (v + m - 1) // m * m


class Server:
    def __init__(self, clients, policy, tol=1e-8, budget_bytes=150 << 30, group_ctas=0, quantum=32,
                 release_scratch=True, device=0, group_scale=0):
        self.clients = clients
        self.policy = policy
        self.tol = float(tol)
        self.budget = int(budget_bytes)
        self.release_scratch = release_scratch
        self.engine = B.Batch(device=device, group_ctas=group_ctas, quantum=quantum, group_scale=group_scale)
        self.evictions = 0
        self.reimports = 0
        self.steps = 0
        self.peak_held = 0
        self._version = 1 << 40

    # ---- memory accounting
    def estimate(self, c: Client) -> int:
        """Bytes the next solve of c adds: direction storage (FP64 / double-float: W, AW and the
        coefficient rows at 1.25x the previous iteration count, as the engine sizes it; FP32
        refinement: W32, AW32, Z32 for max_iter inner iterations), growth of the space, the
        request's matrix values, and the space itself if it has to be re-imported."""
        ld = _round_up(c.n, 32)
        m = c.m_prev if c.m_prev > 0 else 12.0 * c.n ** (1.0 / 3.0)
        cap = _round_up(int(1.25 * m) + 48, 32)
        room = self.policy.max_aug if self.policy.max_aug > 0 else cap
        if self.policy.precision == 1:  # refinement: FP32 storage for max_iter inner iterations
            wi = _round_up(self.policy.max_iter + 1, 32)
            est = ld * (4 * 3 * wi + 4 * 2 * room + 8 * 2 * room + 40) + (72 + 36) * c.nnzb
        else:
            est = 8 * ld * (2 * cap + 1 + 2 * room) + 4 * cap * cap + 72 * c.nnzb
        if c.evicted is not None:
            est += 16 * ld * c.evicted.shape[1]
        return est

    def held(self) -> int:
        tot = 0
        for c in self.clients:
            tot += c.seq.device_bytes()
            if c.inflight is not None:
                tot += 72 * c.nnzb
        return tot

    def _evict_one(self, now) -> bool:
        idle = [c for c in self.clients if c.inflight is None and c.evicted is None and c.seq.device_bytes() > 0]
        if not idle:
            return False
        # least recently used first; clients with nothing queued before those waiting
        idle.sort(key=lambda c: (len(c.queue) > 0, c.last_done))
        c = idle[0]
        c.evicted = c.seq.export_space()
        c.seq.release(B.RELEASE_SCRATCH | B.RELEASE_SPACE | B.RELEASE_MATRIX)
        self.evictions += 1
        return True

    # ---- request flow
    def _submit(self, c: Client, now):
        r = c.queue.popleft()
        if c.evicted is not None:
            c.seq.import_space(c.evicted)
            c.evicted = None
            self.reimports += 1
        A, vals = c.matrix(r.k)
        r.vals = vals
        r.x = c.b.new_zeros(c.n)
        self._version += 1
        r.t_submit = now
        c.inflight = r
        self.engine.submit(c.seq, A, c.b, self.tol, self.policy, tag=c.cid, x=r.x, version=self._version)

    def _admit(self, now):
        waiting = [c for c in self.clients if c.queue and c.inflight is None]
        waiting.sort(key=lambda c: c.queue[0].arrival)
        held = self.held()
        for c in waiting:
            need = self.estimate(c)
            while held + need > self.budget and self._evict_one(now):
                held = self.held()
            if held + need > self.budget and any(x.inflight is not None for x in self.clients):
                break  # wait for memory to come back
            self._submit(c, now)
            held = self.held()
            self.peak_held = max(self.peak_held, held)

    def _complete(self, cid, status, now, closed_loop, n_systems, out):
        c = self.clients[cid]
        r = c.inflight
        c.inflight = None
        st = c.seq.stats()
        r.t_done = now
        r.status = status
        r.m = st["m"]
        r.n_c = st["n_c"]
        r.true_rel_res = st["true_rel_res"]
        r.launches = st["kernel_launches"]
        r.passes = max(1, st["outer_iters"])
        r.m2 = st["inner_m2"]
        r.vals = None
        c.m_prev = st["m"] if st["m"] > 0 else c.m_prev
        c.last_done = now
        if self.release_scratch:
            c.seq.release(B.RELEASE_SCRATCH)
        out.append(r)
        if closed_loop and r.k + 1 < n_systems:
            c.queue.append(Request(cid, r.k + 1, now))

    def run(self, arrivals, closed_loop=False, n_systems=None, clock=time.perf_counter):
        """Serve `arrivals` = [(time, cid, k)] sorted by time (closed_loop: each return
        of (cid, k) issues (cid, k + 1) at once, up to n_systems).  Returns the requests in
        completion order."""
        import torch
        arrivals = sorted(arrivals)
        total = len(arrivals) if not closed_loop else len(self.clients) * n_systems
        out = []
        i = 0
        t0 = clock()
        while len(out) < total:
            now = clock() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                t, cid, k = arrivals[i]
                self.clients[cid].queue.append(Request(cid, k, t))
                i += 1
            self._admit(now)
            if any(c.inflight is not None for c in self.clients):
                done = self.engine.step()
                self.steps += 1
                now = clock() - t0
                for cid, status, _x in done:
                    self._complete(cid, status, now, closed_loop, n_systems, out)
            elif i < len(arrivals):
                time.sleep(max(0.0, arrivals[i][0] - (clock() - t0)))
            else:
                break
        torch.cuda.synchronize()
        return out

    def close(self):
        self.engine.close()


def poisson_arrivals(n_clients, n_systems, rate, seed):
    """Each client issues n_systems requests as a Poisson process of rate rate / n_clients
    (so the total offered rate is `rate`); returns [(time, cid, k)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    per = rate / n_clients
    for cid in range(n_clients):
        t = 0.0
        for k in range(n_systems):
            t += rng.exponential(1.0 / per)
            out.append((t, cid, k))
    out.sort()
    return out


def latency_summary(reqs):
    lat = np.array([r.t_done - r.arrival for r in reqs])
    if lat.size == 0:
        return {}
    t_first = min(r.arrival for r in reqs)
    t_last = max(r.t_done for r in reqs)
    return {"solves": int(lat.size), "solves_per_s": lat.size / max(t_last - t_first, 1e-9),
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean()), "max_ms": 1e3 * float(lat.max()),
            "failed": int(sum(r.status != 0 for r in reqs)),
            "max_true_rel_res": float(max(r.true_rel_res for r in reqs))}


def make_clients(Ns, n_systems, seed, device=0, pool=None):
    """Damage-sequence clients: client i has cube size Ns[i], ellipsoid seed seed + i,
    traction seed seed + 10000 + i, d_k falling geometrically from 1 to 0.05."""
    from . import problems as P
    dks = P.damage_factors(n_systems)
    args = [(int(N), seed + i, seed + 10000 + i) for i, N in enumerate(Ns)]
    parts = pool.starmap(P.damage_parts, args) if pool is not None else [P.damage_parts(*a) for a in args]
    return [Client(i, A_out, vin, b, dks, device) for i, (A_out, vin, b) in enumerate(parts)]


def solve_alone(clients, policy, tol, per_solve=True, release_scratch=True):
    """Reference path: every request of every client solved one at a time with krs_solve
    (each a full-device persistent launch).  Returns (elapsed seconds, requests)."""
    import torch
    out = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ver = 1 << 50
    for c in clients:
        for k in range(len(c.dks)):
            A, vals = c.matrix(k)
            x = c.b.new_zeros(c.n)
            ver += 1
            _, st = c.seq.solve(A, c.b, tol, policy, x=x, version=ver, raise_on_error=False)
            out.append(Request(c.cid, k, 0.0, 0.0, time.perf_counter() - t0, st["status"], st["m"], st["n_c"],
                               st["true_rel_res"], st["kernel_launches"], x))
            if release_scratch:
                c.seq.release(B.RELEASE_SCRATCH)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out
