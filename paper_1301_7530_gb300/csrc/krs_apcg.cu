// krs_apcg.cu -- the APCG iteration on the GPU (Algorithm 1 with full
// reorthogonalisation), in two execution modes that share every arithmetic routine:
//   * persistent: one cooperative kernel runs the whole iteration loop of a solve; the
//     phases are separated by bounded grid barriers;
//   * kernels:    one kernel launch per phase (the launch boundary is the barrier).
// Both use the same CTA partition and the same reduction order, so they produce the same
// bits.  Everything is templated on the value type T of the vectors, multi-vectors and
// matrix: T = double for the FP64 solve, T = float for the inner solve of the
// mixed-precision refinement.  Scalars (alpha, gamma, rho, the coarse coefficients) and
// every partial sum that crosses CTAs are doubles in both.
//
// One iteration j (literal order of Algorithm 1 with the readings: z_j = P M^-1 r_j, the
// Gram-Schmidt beta computed before use, classical Gram-Schmidt over all stored
// directions):
//   P1  q = A w_j (stored as AW[:, j]); partials (w_j, q), (r_j, w_j)
//   P2  gamma_j, alpha_j = (r_j, w_j)/gamma_j; x += alpha w_j; r -= alpha q; (r, r);
//       u = M^-1 r; partials t = (AC)^T u
//   P3  convergence ||r||^2 <= tol^2 ||b||^2; t reduced (slice, or whole when n_c is small)
//   P4  slice of s = (C^T A C)^-1 t (only when n_c is not small)
//   P5  z = u - C s (Z[:, j+1], or the single z column); partials (r, z), g = (AW)^T z
//   P6  rho_{j+1} = (r, z); slice of g_i / gamma_i (also kept in the packed coefficient
//       rows U when z is not stored: z_{j+1} = w_{j+1} + sum_i g_i w_i)
//   P7  w_{j+1} = z - W g (stored as W[:, j+1])
// The projection P u = u - C (C^T A C)^-1 (AC)^T u is the projector of Eq. 5; its two
// block products and the coarse solve are the items of Section 2.3.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#include <mutex>
#include <type_traits>

#include "krs_device.cuh"
#include "krs_internal.h"

namespace krs {

// Precision of a solve: V = vectors x, r, u (and q in PrecP / PrecE), M = the search
// directions W, AW, Z, MC = the augmentation space C, AC, A = matrix values and M^-1.
// Partial sums that cross CTAs and every scalar are doubles in all four.
//   PrecD  FP64 throughout;
//   PrecF  FP32 throughout (inner solves of the mixed-precision refinement);
//   PrecP  FP64 operator product, preconditioner, x and r recurrences; FP32 projection and
//          reorthogonalisation (C, AC, W, AW, Z stored and combined in FP32);
//   PrecE  FP64 preconditioner, recurrences and projection (C, AC); double-float search
//          directions W, AW, Z and matrix values (48-bit significand), so that the operator
//          product and the reorthogonalisation run on the FP32 pipes.  The operator product
//          writes q in FP64 (its double-float copy goes to AW); x, (w, q) and (r, w) use the
//          FP64 copy wv of w_j.
struct PrecD { using V = double; using M = double; using MC = double; using A = double; static constexpr int id = 0; };
struct PrecF { using V = float;  using M = float;  using MC = float;  using A = float;  static constexpr int id = 1; };
struct PrecP { using V = double; using M = float;  using MC = float;  using A = double; static constexpr int id = 2; };
struct PrecE { using V = double; using M = dfl;    using MC = double; using A = double; static constexpr int id = 3; };

template <typename Pr>
struct ApcgCtx {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using MC = typename Pr::MC;
  using A = typename Pr::A;
  int64_t n, ld;       // order, leading dimension of multi-vectors and vector padding
  int nbr, npc, P;     // block rows, nodes per CTA, CTAs of this problem's group
  int cta0;            // first CTA of the group in a batched launch (0 otherwise)
  int lb;              // this CTA's index within its group (set on kernel entry)
  int nc, ldg;         // columns of C, leading dimension of Ginv
  int nc_dense;        // columns [0, nc_dense) use Ginv; columns [nc_dense, nc) are mutually
                       // A-conjugate directions whose coarse block is diag(dinv)
  int max_iter, reorth_full, precond;
  int jcap;            // iterations j >= jcap do not start in this launch (direction storage)
  double tol2;         // tol^2 * ||b||^2
  long long spin_limit;
  const double* dinv;  // 1/(w_i, A w_i) of the tail columns
  const int* rp;
  const int* ci;
  const A* vals;
  const A* minv;
  const MC* C;
  const MC* AC;
  const double* Ginv;
  M* W;
  M* AW;
  M* Z;                // z_j: column j at Z + j * zld (zld = 0: one column, reused)
  int64_t zld;
  double* ucoef;       // zld = 0: packed reorthogonalisation coefficients, row j at
                       // j (j - 1) / 2 holding g_i of w_j = z_j - sum_{i<j} g_i w_i
  V* x;
  V* r;
  V* u;
  V* q;                // PrecP, PrecE: the FP64 operator product A w_j (AW keeps its copy)
  V* wv;               // PrecE: the FP64 search direction w_j (W keeps its double-float copy)
  const dfl* valsd;    // PrecE: the matrix values as double-float (the operator product)
  double* alpha;
  double* gamma;
  double* rho;
  double* tfull;
  double* sfull;
  double* gfull;
  double* part;        // [P * PS_STRIDE]
  double* vpart;       // [P * vld]  partials of t = (AC)^T u
  double* gpart;       // [P * vld]  partials of g = (AW)^T z (separate: no phase overlap hazard)
  int64_t vld;
  int* ctrl;           // this solve's status / done / iteration words
  int* bctrl;          // status / abort words the barrier watches (== ctrl for one solve)
  int* gstop;          // batched: the group's drain word (nullptr for one solve)
  const int* idle;     // batched: groups that found their queue empty
  int drain_at;        // batched: drain once this many groups are idle (0: never)
  int stall_win;       // > 0: end with status 7 when ||r||^2 fell < 4x over stall_win iterations
  double stall_rr;     //   once ||r||^2 is below this (the test is off on the way down)
  double* rrh;         // ||r_j||^2 history for the stall test
  unsigned long long* bar;
};

// shared-memory layout (in doubles): su[ROW_CHUNK] | red[4*TPB] | sv[kmax]
// (su and sv hold values of the direction type M; svc is sv seen as the type MC of the
// augmentation space, for the coarse coefficients s)
template <typename Pr>
struct Smem {
  typename Pr::M* su;
  double* red;
  typename Pr::M* sv;
  typename Pr::MC* svc;
};

template <typename Pr>
__device__ __forceinline__ Smem<Pr> smem_layout(double* base) {
  static_assert(sizeof(typename Pr::M) <= sizeof(double) && sizeof(typename Pr::MC) <= sizeof(double),
                "shared-memory slots hold one double");
  Smem<Pr> s;
  s.su = reinterpret_cast<typename Pr::M*>(base);
  s.red = base + ROW_CHUNK;
  s.sv = reinterpret_cast<typename Pr::M*>(base + ROW_CHUNK + 4 * TPB);
  s.svc = reinterpret_cast<typename Pr::MC*>(base + ROW_CHUNK + 4 * TPB);
  return s;
}

enum PhaseResult { PH_CONTINUE = 0, PH_STOP = 1 };

template <typename Pr>
__device__ __forceinline__ void finish(const ApcgCtx<Pr>& c, int status, int m) {
  if (c.lb == 0 && threadIdx.x == 0) {
    if (status) atomicCAS(c.ctrl + CTRL_STATUS, 0, status);
    c.ctrl[CTRL_M] = m;
    c.ctrl[CTRL_DONE] = 1;
  }
}

// Reduce a scalar partial over all CTAs (warp 0, fixed order) and broadcast it.
__device__ __forceinline__ double grid_scalar(const double* part, int P, int slot, double* red) {
  if (threadIdx.x < 32) {
    double v = warp_sum_strided(part + slot, P, PS_STRIDE);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  double v = red[0];
  __syncthreads();
  return v;
}

// Two scalars at once (warps 0 and 1 in parallel).
__device__ __forceinline__ void grid_scalar2(const double* part, int P, int slot_a, int slot_b, double* red,
                                             double& va, double& vb) {
  const int warp = threadIdx.x >> 5;
  if (warp < 2) {
    const double v = warp_sum_strided(part + (warp == 0 ? slot_a : slot_b), P, PS_STRIDE);
    if ((threadIdx.x & 31) == 0) red[warp] = v;
  }
  __syncthreads();
  va = red[0];
  vb = red[1];
  __syncthreads();
}

// Augmentation sizes up to this are reduced by every CTA redundantly (no extra barriers).
constexpr int SMALL_NC = 16;

// s[col] = (G^-1 t)[col]: the dense block G^-1 (nc_dense x nc_dense) for the first columns,
// 1/(w, Aw) for the tail of mutually A-conjugate directions.  Computed by one warp; the
// result is returned to every lane.
__device__ __forceinline__ double coarse_coef(const double* Ginv, int ldg, int nc_dense, const double* dinv, int col,
                                              const double* t) {
  const int lane = threadIdx.x & 31;
  if (col >= nc_dense) return t[col] * dinv[col - nc_dense];
  const double* g = Ginv + (int64_t)col * ldg;
  double s = 0.0;
  for (int k = lane; k < nc_dense; k += 32) s += g[k] * t[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <typename Pr>
__device__ __forceinline__ void phase1(const ApcgCtx<Pr>& c, int j, Smem<Pr>& sm) {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using A = typename Pr::A;
  int64_t r0, r1;
  cta_rows(c.nbr, c.npc, c.lb, r0, r1);
  const M* w = c.W + (int64_t)j * c.ld;
  M* aw = c.AW + (int64_t)j * c.ld;
  double wq = 0.0, rw = 0.0;
  if constexpr (Pr::id == 2)  // q in FP64 for the recurrences, its FP32 copy into AW
    cta_spmv<A, M, V, V>(c.rp, c.ci, c.vals, w, c.q, c.r, r0, r1, wq, rw, aw);
  else if constexpr (Pr::id == 3)  // double-float A and w_j on the FP32 pipes; q in FP64 and into AW
    cta_spmv_df(c.rp, c.ci, c.valsd, w, c.wv, c.q, aw, c.r, r0, r1, wq, rw);
  else
    cta_spmv<A, M, M, V>(c.rp, c.ci, c.vals, w, aw, c.r, r0, r1, wq, rw);
  block_sum2(wq, rw, sm.red);
  if (threadIdx.x == 0) {
    c.part[c.lb * PS_STRIDE + PS_WQ] = wq;
    c.part[c.lb * PS_STRIDE + PS_RW] = rw;
  }
}

template <typename Pr>
__device__ __forceinline__ int phase2(const ApcgCtx<Pr>& c, int j, Smem<Pr>& sm) {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using A = typename Pr::A;
  double gam, rws;
  grid_scalar2(c.part, c.P, PS_WQ, PS_RW, sm.red, gam, rws);
  if (!(gam > 0.0)) {
    finish(c, 2 /* KRS_ERR_NOT_SPD */, j);
    return PH_STOP;
  }
  const double al = rws / gam;
  if (c.lb == 0 && threadIdx.x == 0) {
    c.alpha[j] = al;
    c.gamma[j] = gam;
  }
  const V alT = (V)al;
  int64_t r0, r1;
  cta_rows(c.nbr, c.npc, c.lb, r0, r1);
  using WT = typename std::conditional<Pr::id == 3, V, M>::type;
  const WT* w;
  if constexpr (Pr::id == 3) w = c.wv;
  else w = c.W + (int64_t)j * c.ld;
  const V* q;
  if constexpr (Pr::id == 2 || Pr::id == 3) q = c.q;
  else q = c.AW + (int64_t)j * c.ld;
  double rr = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) {
    c.x[row] += alT * (V)w[row];
    const V rn = c.r[row] - alT * q[row];
    c.r[row] = rn;
    rr += (double)rn * (double)rn;
  }
  __syncthreads();
  for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB)
    c.u[row] = precond_row<A, V>(c.precond, c.minv, c.r, row);
  rr = block_sum(rr, sm.red);
  if (threadIdx.x == 0) c.part[c.lb * PS_STRIDE + PS_RR] = rr;
  if (c.nc > 0)
    cta_gemv_t<true, typename Pr::MC, V>(c.AC, c.ld, c.nc, c.u, r0, r1, c.vpart + c.lb * c.vld,
                                         reinterpret_cast<typename Pr::MC*>(sm.su), sm.red);
  return PH_CONTINUE;
}

// Slice [a, b) of the k reduced columns owned by this CTA.
__device__ __forceinline__ void col_slice(int k, int P, int b, int& a, int& e) {
  const int per = (k + P - 1) / P;
  a = min(k, b * per);
  e = min(k, a + per);
}

template <typename Pr>
__device__ __forceinline__ int phase3(const ApcgCtx<Pr>& c, int j, Smem<Pr>& sm) {
  using MC = typename Pr::MC;
  const double rr = grid_scalar(c.part, c.P, PS_RR, sm.red);
  if (rr <= c.tol2) {
    finish(c, 0, j + 1);
    return PH_STOP;
  }
  if (c.stall_win > 0) {
    // the history entry stall_win iterations back was written before many grid barriers,
    // so every CTA reads the same value and takes the same decision
    if (c.lb == 0 && threadIdx.x == 0) c.rrh[j] = rr;
    if (j >= c.stall_win && rr < c.stall_rr && rr > 0.25 * c.rrh[j - c.stall_win]) {
      finish(c, 7 /* KRS_STALLED */, j + 1);
      return PH_STOP;
    }
  }
  if (j + 1 >= c.max_iter) {
    finish(c, 3 /* KRS_ERR_NO_CONVERGENCE */, j + 1);
    return PH_STOP;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c.nc > SMALL_NC) {
    // slice of t reduced here; s follows in phase 4 after a barrier
    int a, e;
    col_slice(c.nc, c.P, c.lb, a, e);
    for (int col = a + warp; col < e; col += TPB / 32) {
      const double v = warp_sum_strided(c.vpart + col, c.P, c.vld);
      if (lane == 0) c.tfull[col] = v;
    }
  } else if (c.nc > 0) {
    // every CTA: t = sum of all partials (fixed order), s = Ginv t into shared memory
    for (int col = warp; col < c.nc; col += TPB / 32) {
      const double v = warp_sum_strided(c.vpart + col, c.P, c.vld);
      if (lane == 0) sm.red[col] = v;
    }
    __syncthreads();
    for (int col = warp; col < c.nc; col += TPB / 32) {
      const double sacc = coarse_coef(c.Ginv, c.ldg, c.nc_dense, c.dinv, col, sm.red);
      if (lane == 0) {
        sm.svc[col] = (MC)sacc;
        if (c.lb == 0) c.sfull[col] = sacc;  // for the per-phase kernel mode
      }
    }
    __syncthreads();
  }
  return PH_CONTINUE;
}

template <typename Pr>
__device__ __forceinline__ void phase4(const ApcgCtx<Pr>& c) {
  int a, e;
  col_slice(c.nc, c.P, c.lb, a, e);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int col = a + warp; col < e; col += TPB / 32) {
    const double s = coarse_coef(c.Ginv, c.ldg, c.nc_dense, c.dinv, col, c.tfull);
    if (lane == 0) c.sfull[col] = s;
  }
}

// s_in_smem: s = Ginv t is already in sm.sv (small-augmentation path of phase 3 in the
// same kernel); otherwise it is read from sfull.
template <typename Pr>
__device__ __forceinline__ void phase5(const ApcgCtx<Pr>& c, int j, Smem<Pr>& sm, bool s_in_smem) {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using MC = typename Pr::MC;
  int64_t r0, r1;
  cta_rows(c.nbr, c.npc, c.lb, r0, r1);
  M* z = c.Z + (int64_t)(j + 1) * c.zld;
  if (c.nc > 0) {
    if (!s_in_smem) {
      for (int k = threadIdx.x; k < c.nc; k += TPB) sm.svc[k] = (MC)c.sfull[k];
    }
    __syncthreads();
    cta_gemv_n<true, MC, V, M>(c.C, c.ld, c.nc, sm.svc, MC(-1), c.u, z, r0, r1, sm.red);
  } else {
    for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) z[row] = (M)c.u[row];
    __syncthreads();
  }
  double rz = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) rz += (double)c.r[row] * (double)z[row];
  rz = block_sum(rz, sm.red);
  if (threadIdx.x == 0) c.part[c.lb * PS_STRIDE + PS_RZ] = rz;
  const int base = c.reorth_full ? 0 : j;
  const int kk = j + 1 - base;
  cta_gemv_t<false, M, M>(c.AW + (int64_t)base * c.ld, c.ld, kk, z, r0, r1, c.gpart + c.lb * c.vld,
                          sm.su, sm.red);
}

template <typename Pr>
__device__ __forceinline__ int phase6(const ApcgCtx<Pr>& c, int j, Smem<Pr>& sm) {
  const double rz = grid_scalar(c.part, c.P, PS_RZ, sm.red);
  if (!(rz > 0.0)) {
    finish(c, 2 /* KRS_ERR_NOT_SPD */, j + 1);
    return PH_STOP;
  }
  if (c.lb == 0 && threadIdx.x == 0) c.rho[j + 1] = rz;
  const int base = c.reorth_full ? 0 : j;
  const int kk = j + 1 - base;
  int a, e;
  col_slice(kk, c.P, c.lb, a, e);
  const int warp = threadIdx.x >> 5;
  double* urow = c.ucoef ? c.ucoef + (int64_t)(j + 1) * j / 2 + base : nullptr;  // row j + 1 of U
  for (int col = a + warp; col < e; col += TPB / 32) {
    const double v = warp_sum_strided(c.gpart + col, c.P, c.vld);
    if ((threadIdx.x & 31) == 0) {
      const double g = v / c.gamma[base + col];
      c.gfull[col] = g;
      if (urow) urow[col] = g;
    }
  }
  return PH_CONTINUE;
}

template <typename Pr>
__device__ __forceinline__ void phase7(const ApcgCtx<Pr>& c, int j, Smem<Pr>& sm) {
  using M = typename Pr::M;
  int64_t r0, r1;
  cta_rows(c.nbr, c.npc, c.lb, r0, r1);
  const int base = c.reorth_full ? 0 : j;
  const int kk = j + 1 - base;
  for (int k = threadIdx.x; k < kk; k += TPB) sm.sv[k] = (M)c.gfull[k];
  __syncthreads();
  const M* z = c.Z + (int64_t)(j + 1) * c.zld;
  M* wn = c.W + (int64_t)(j + 1) * c.ld;
  double* wv = nullptr;
  if constexpr (Pr::id == 3) wv = c.wv;  // the FP64 copy of w_{j+1} for the next operator product
  cta_gemv_n<false, M, M, M>(c.W + (int64_t)base * c.ld, c.ld, kk, sm.sv, M(-1.0), z, wn, r0, r1, sm.red, wv);
}

// ------------------------------------------------------------------------------------
// persistent kernel: the whole iteration loop of one solve
// ------------------------------------------------------------------------------------
enum LoopResult { LOOP_ENDED = 0, LOOP_SUSPENDED = 1, LOOP_ABORTED = 2, LOOP_DRAINED = 3 };

// The iteration loop of one solve from iteration j0, run by the CTAs of one group: at most
// `quantum` iterations, after which the solve is suspended with CTRL_J = the next iteration
// (every value the loop carries from one iteration to the next is in global memory).
// `target` is the CTA's running count for the group's barrier counter.
// Drain (batched launches): at the end of each iteration the group's first CTA compares
// the launch's idle-group count with drain_at and publishes the outcome in the group's
// drain word before the iteration's last barrier; every CTA of the group reads that word
// after the barrier, so all of them suspend at the same iteration.
template <typename Pr>
__device__ __forceinline__ int apcg_loop(const ApcgCtx<Pr>& c, Smem<Pr>& sm, int j0, int quantum,
                                         unsigned long long& target) {
  const int TO = 6;  // KRS_ERR_TIMEOUT
#define KRS_SYNC()                                                                         \
  do {                                                                                     \
    if (!grid_barrier(c.bar, target, (unsigned)c.P, c.bctrl, c.spin_limit, TO)) return LOOP_ABORTED; \
  } while (0)
  for (int j = j0;; j++) {
    if (j - j0 >= quantum || j >= c.jcap) {
      if (c.lb == 0 && threadIdx.x == 0) c.ctrl[CTRL_J] = j;
      return LOOP_SUSPENDED;
    }
    if (c.gstop && *((volatile int*)c.gstop)) {
      if (c.lb == 0 && threadIdx.x == 0) c.ctrl[CTRL_J] = j;
      return LOOP_DRAINED;
    }
    phase1(c, j, sm);
    KRS_SYNC();
    if (phase2(c, j, sm) == PH_STOP) return LOOP_ENDED;
    KRS_SYNC();
    if (phase3(c, j, sm) == PH_STOP) return LOOP_ENDED;
    if (c.nc > SMALL_NC) {
      KRS_SYNC();
      phase4(c);
      KRS_SYNC();
      phase5(c, j, sm, false);
    } else {
      phase5(c, j, sm, true);  // nothing written in phase 3 is read by another CTA here
    }
    KRS_SYNC();
    if (phase6(c, j, sm) == PH_STOP) return LOOP_ENDED;
    KRS_SYNC();
    phase7(c, j, sm);
    if (c.gstop && c.drain_at > 0 && c.lb == 0 && threadIdx.x == 0 && *((volatile const int*)c.idle) >= c.drain_at)
      *((volatile int*)c.gstop) = 1;
    KRS_SYNC();
  }
#undef KRS_SYNC
}

// persistent kernel: one solve, all CTAs in one group
template <typename Pr>
__global__ void __launch_bounds__(TPB, 1) k_apcg_persistent(ApcgCtx<Pr> c) {
  extern __shared__ double4_32a smem_raw4[];
  Smem<Pr> sm = smem_layout<Pr>(reinterpret_cast<double*>(smem_raw4));
  c.lb = blockIdx.x;
  unsigned long long target = 0;
  apcg_loop(c, sm, 0, 0x7fffffff, target);
}

// Batched persistent kernel: many independent solves in one cooperative launch.  The grid
// is cut into groups of CTAs; groups of the same size form a class with its own work
// queue.  A group takes the next solve from its class's queue, runs its iterations (at
// most `quantum` of them) with the group's own barrier counter and partial-sum buffers,
// and takes the next, until the queue is empty.  Solves of uneven sizes and iteration
// counts therefore never wait for each other, a group that finishes early picks up queued
// work at once, and a large solve can run on a larger group than a small one.  A solve is
// queued only in the class whose group size its context was prepared for, so its
// arithmetic (the partition and the order of every reduction) depends on its group size
// only -- not on which group runs it or on which other solves share the launch.
template <typename Pr>
struct BatchArgs {
  const ApcgCtx<Pr>* ctxs;   // one per solve in the table
  const int* queue;         // per class, indices into ctxs in the order groups take them
  const int* qoff;          // [classes + 1] offsets of the classes' queues
  int* heads;               // [classes] queue positions (zero at launch)
  const int* cta_group;     // [CTAs] group of each CTA
  const int* grp_cta0;      // [groups + 1] first CTA of each group (groups are contiguous)
  const int* grp_class;     // [groups] class (queue) of each group
  int quantum;              // iteration limit per solve in this launch
  int drain_at;             // suspend every solve once this many groups are idle (0: never)
  int* idle;                // idle-group counter (zero at launch)
  int* gstop;               // [groups] drain words (zero at launch)
  int* mail;                // [groups * 2] solve index handed from the group's first CTA
  unsigned long long* gbar; // [groups * 16] barrier counters (one 128-byte line each)
  double* gpart;            // [CTAs * PS_STRIDE], a group uses the rows of its CTAs
  double* gvpart;           // [CTAs * vld]
  double* ggpart;           // [CTAs * vld]
  int64_t vld;
  long long spin_limit;
  int* bctrl;               // launch-wide status / abort words
};

template <typename Pr>
__global__ void __launch_bounds__(TPB, 1) k_apcg_batched(BatchArgs<Pr> B) {
  extern __shared__ double4_32a smem_raw4[];
  Smem<Pr> sm = smem_layout<Pr>(reinterpret_cast<double*>(smem_raw4));
  const int group = B.cta_group[blockIdx.x];
  const int c0 = B.grp_cta0[group];
  const int g = B.grp_cta0[group + 1] - c0;
  const int lb = (int)blockIdx.x - c0;
  const int cls = B.grp_class[group];
  const int q0 = B.qoff[cls], qlen = B.qoff[cls + 1] - q0;
  unsigned long long* bar = B.gbar + (int64_t)group * 16;
  unsigned long long target = 0;
  __shared__ ApcgCtx<Pr> s_ctx;
  __shared__ int s_j0;
  for (int round = 0;; round++) {
    int* box = B.mail + 2 * group + (round & 1);
    if (lb == 0 && threadIdx.x == 0) {
      const int k = atomicAdd(B.heads + cls, 1);
      *box = k < qlen ? B.queue[q0 + k] : -1;
      if (k >= qlen) atomicAdd(B.idle, 1);
    }
    if (!grid_barrier(bar, target, (unsigned)g, B.bctrl, B.spin_limit, 6)) return;
    const int idx = *((volatile int*)box);
    if (idx < 0) return;
    // the solve's context lives in shared memory (the kernel-parameter copy of the
    // single-solve kernel has no per-solve equivalent; registers would spill)
    __syncthreads();  // every thread is done with the previous solve's context
    if (threadIdx.x == 0) {
      ApcgCtx<Pr> c = B.ctxs[idx];
      c.lb = lb;
      c.P = g;
      c.bar = bar;
      c.bctrl = B.bctrl;
      c.part = B.gpart + (int64_t)c0 * PS_STRIDE;
      c.vpart = B.gvpart + (int64_t)c0 * B.vld;
      c.gpart = B.ggpart + (int64_t)c0 * B.vld;
      c.vld = B.vld;
      c.gstop = B.gstop + group;
      c.idle = B.idle;
      c.drain_at = B.drain_at;
      s_ctx = c;
      s_j0 = *((volatile int*)(c.ctrl + CTRL_J));
    }
    __syncthreads();
    const ApcgCtx<Pr>& c = s_ctx;
    const int j0 = s_j0;
    const int res = apcg_loop(c, sm, j0, B.quantum, target);
    if (res == LOOP_ABORTED || res == LOOP_DRAINED) return;
  }
}

// ------------------------------------------------------------------------------------
// per-phase kernels (kernels mode).  Each returns at once when the solve has ended.
// ------------------------------------------------------------------------------------
template <typename Pr>
__device__ __forceinline__ bool ended(const ApcgCtx<Pr>& c) {
  return *((volatile int*)(c.ctrl + CTRL_DONE)) != 0;
}

#define KRS_PHASE_KERNEL(NAME, BODY)                                          \
  template <typename Pr>                                                       \
  __global__ void __launch_bounds__(TPB, 1) NAME(ApcgCtx<Pr> c, int j) {      \
    extern __shared__ double4_32a smem_raw4[];                                \
    Smem<Pr> sm = smem_layout<Pr>(reinterpret_cast<double*>(smem_raw4));       \
    c.lb = blockIdx.x;                                                        \
    if (ended(c)) return;                                                     \
    (void)sm;                                                                 \
    BODY;                                                                     \
  }

KRS_PHASE_KERNEL(k_phase1, phase1(c, j, sm))
KRS_PHASE_KERNEL(k_phase2, phase2(c, j, sm))
KRS_PHASE_KERNEL(k_phase3, phase3(c, j, sm))
KRS_PHASE_KERNEL(k_phase4, phase4(c))
KRS_PHASE_KERNEL(k_phase5, phase5(c, j, sm, false))
KRS_PHASE_KERNEL(k_phase6, phase6(c, j, sm))
KRS_PHASE_KERNEL(k_phase7, phase7(c, j, sm))

// ------------------------------------------------------------------------------------
// set-up: x_0, r_0 = P^T b, z_0 = P M^-1 r_0, w_0 = z_0, rho_0 (Algorithm 1, steps 1-3)
// ------------------------------------------------------------------------------------

// partial t = V^T y over the CTA's rows (y global)
template <typename TM, typename TU>
__global__ void __launch_bounds__(TPB, 1) k_gemv_t_part(const TM* V, int64_t ld, int k, const TU* y, int nbr,
                                                        int npc, double* vpart, int64_t vld) {
  extern __shared__ double4_32a smem_raw4[];
  double* base = reinterpret_cast<double*>(smem_raw4);
  int64_t r0, r1;
  cta_rows(nbr, npc, blockIdx.x, r0, r1);
  cta_gemv_t<false, TM, TU>(V, ld, k, y, r0, r1, vpart + blockIdx.x * vld, reinterpret_cast<TM*>(base),
                            base + ROW_CHUNK);
}

// out[c] = sum_b vpart[b*vld + c]  (c < k)
__global__ void k_reduce_cols(const double* vpart, int64_t vld, int P, int k, double* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= k) return;
  const double v = warp_sum_strided(vpart + warp, P, vld);
  if ((threadIdx.x & 31) == 0) out[warp] = v;
}

__global__ void k_small_gemv(const double* G, int ldg, int k, int k_dense, const double* dinv, const double* t,
                             double* s) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= k) return;
  const double a = coarse_coef(G, ldg, k_dense, dinv, warp, t);
  if (lane == 0) s[warp] = a;
}

// x = C s, r = b - AC s (or x = 0, r = b when k == 0); partials (b, b) and (r, r)
template <typename TC, typename TV>
__global__ void __launch_bounds__(TPB, 1) k_init_xr(const TC* C, const TC* AC, int64_t ld, int k, const double* s,
                                                    const TV* b, TV* x, TV* r, int nbr, int npc, double* part) {
  extern __shared__ double4_32a smem_raw4[];
  double* base = reinterpret_cast<double*>(smem_raw4);
  double* red = base + ROW_CHUNK;
  TC* sv = reinterpret_cast<TC*>(base + ROW_CHUNK + 4 * TPB);
  int64_t r0, r1;
  cta_rows(nbr, npc, blockIdx.x, r0, r1);
  if (k > 0) {
    for (int i = threadIdx.x; i < k; i += TPB) sv[i] = (TC)s[i];
    __syncthreads();
    cta_gemv_n<false, TC, TV, TV>(C, ld, k, sv, TC(1), nullptr, x, r0, r1, red);
    cta_gemv_n<false, TC, TV, TV>(AC, ld, k, sv, TC(-1), b, r, r0, r1, red);
  } else {
    for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) {
      x[row] = TV(0);
      r[row] = b[row];
    }
    __syncthreads();
  }
  double bb = 0.0, rr = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) {
    bb += (double)b[row] * (double)b[row];
    rr += (double)r[row] * (double)r[row];
  }
  block_sum2(bb, rr, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * PS_STRIDE + 0] = bb;
    part[blockIdx.x * PS_STRIDE + 1] = rr;
  }
}

// u = M^-1 r
template <typename TA, typename TV>
__global__ void k_precond_rows(int kind, const TA* minv, const TV* r, TV* u, int64_t n) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < n) u[row] = precond_row<TA, TV>(kind, minv, r, row);
}

// z0 = u - C s (or u), stored as TZ: W[:,0] = Z[:,0] = z0, partial (r, z0) of the stored z0;
// wv (optional): z0 = w0 also as a double
template <typename TC, typename TV, typename TZ>
__global__ void __launch_bounds__(TPB, 1) k_init_z(const TC* C, int64_t ld, int k, const double* s, const TV* u,
                                                   const TV* r, TZ* Z, TZ* W, int nbr, int npc, double* part,
                                                   double* wv) {
  extern __shared__ double4_32a smem_raw4[];
  double* base = reinterpret_cast<double*>(smem_raw4);
  double* red = base + ROW_CHUNK;
  TC* sv = reinterpret_cast<TC*>(base + ROW_CHUNK + 4 * TPB);
  int64_t r0, r1;
  cta_rows(nbr, npc, blockIdx.x, r0, r1);
  if (k > 0) {
    for (int i = threadIdx.x; i < k; i += TPB) sv[i] = (TC)s[i];
    __syncthreads();
    cta_gemv_n<false, TC, TV, TZ>(C, ld, k, sv, TC(-1), u, Z, r0, r1, red, wv);
  } else {
    for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) {
      Z[row] = (TZ)u[row];
      if (wv) wv[row] = (double)u[row];
    }
    __syncthreads();
  }
  double rz = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) {
    W[row] = Z[row];
    rz += (double)r[row] * (double)Z[row];
  }
  rz = block_sum(rz, red);
  if (threadIdx.x == 0) part[blockIdx.x * PS_STRIDE + 2] = rz;
}

// scal[0] = bb, scal[1] = rr0, rho[0] = rho0 (all from partial slots 0, 1, 2)
__global__ void k_init_finish(const double* part, int P, double* scal, double* rho) {
  const int warp = threadIdx.x >> 5;
  if (warp < 3) {
    const double v = warp_sum_strided(part + warp, P, PS_STRIDE);
    if ((threadIdx.x & 31) == 0) {
      if (warp < 2) scal[warp] = v;
      else rho[0] = v;
    }
  }
}

// ------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------
size_t apcg_smem_bytes(int kmax) {
  return sizeof(double) * (size_t)(ROW_CHUNK + 4 * TPB + ((kmax + 3) & ~3));
}

template <typename Pr>
static ApcgCtx<Pr> make_ctx(const IterArgs& a) {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using A = typename Pr::A;
  ApcgCtx<Pr> c;
  c.n = a.n; c.ld = a.ld; c.nbr = a.nbr; c.npc = a.npc; c.P = a.P;
  c.nc = a.nc; c.ldg = a.ldg; c.max_iter = a.max_iter; c.reorth_full = a.reorth_full;
  c.nc_dense = a.nc_dense; c.dinv = a.dinv;
  c.cta0 = 0; c.lb = 0; c.jcap = a.jcap > 0 ? a.jcap : 0x7fffffff;
  c.precond = a.precond; c.tol2 = a.tol2; c.spin_limit = a.spin_limit;
  c.rp = a.rp; c.ci = a.ci;
  c.vals = static_cast<const A*>(a.vals); c.minv = static_cast<const A*>(a.minv);
  c.C = static_cast<const typename Pr::MC*>(a.C); c.AC = static_cast<const typename Pr::MC*>(a.AC);
  c.Ginv = a.Ginv;
  c.W = static_cast<M*>(a.W); c.AW = static_cast<M*>(a.AW); c.Z = static_cast<M*>(a.Z);
  c.zld = a.zld; c.ucoef = a.zld == 0 ? a.ucoef : nullptr;
  c.x = static_cast<V*>(a.x); c.r = static_cast<V*>(a.r); c.u = static_cast<V*>(a.u);
  c.q = static_cast<V*>(a.q);
  c.wv = static_cast<V*>(a.wv);
  c.valsd = static_cast<const dfl*>(a.vals_df);
  c.alpha = a.alpha; c.gamma = a.gamma; c.rho = a.rho;
  c.tfull = a.tfull; c.sfull = a.sfull; c.gfull = a.gfull;
  c.part = a.part; c.vpart = a.vpart; c.gpart = a.gpart; c.vld = a.vld; c.ctrl = a.ctrl; c.bar = a.bar;
  c.bctrl = a.ctrl;
  c.gstop = nullptr;
  c.idle = nullptr;
  c.drain_at = 0;
  c.stall_win = a.stall_win;
  c.stall_rr = a.stall_rr;
  c.rrh = a.rrh;
  return c;
}

// init element types: the init stage of PrecP works from the FP64 C and AC (x_0 and r_0 in
// FP64, consistent with the FP64 recurrences) and stores z_0 in FP32; PrecE's C and AC are
// FP64 and it stores z_0 in double-float
template <typename Pr>
struct InitTypes {
  using TC = typename std::conditional<Pr::id == 2, double, typename Pr::MC>::type;
};

template <typename Pr>
static cudaError_t prepare_attributes_t(size_t sm) {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using TC = typename InitTypes<Pr>::TC;
  // the init kernels over C and AC of type TC, and (PrecP's restarted passes, PrecF) of type M
  using TM = typename std::conditional<Pr::id == 3, double, M>::type;
  const void* fns[] = {(const void*)k_apcg_persistent<Pr>, (const void*)k_phase1<Pr>, (const void*)k_phase2<Pr>,
                       (const void*)k_phase3<Pr>, (const void*)k_phase4<Pr>, (const void*)k_phase5<Pr>,
                       (const void*)k_phase6<Pr>, (const void*)k_phase7<Pr>, (const void*)k_gemv_t_part<TC, V>,
                       (const void*)k_init_xr<TC, V>, (const void*)k_init_z<TC, V, M>,
                       (const void*)k_gemv_t_part<TM, V>, (const void*)k_init_xr<TM, V>, (const void*)k_init_z<TM, V, M>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Dispatch on the precision id of IterArgs (0 PrecD, 1 PrecF, 2 PrecP, 3 PrecE).
#define KRS_DISPATCH(prec, CALL)           \
  do {                                     \
    if ((prec) == 1) {                     \
      using PR = PrecF;                    \
      CALL;                                \
    } else if ((prec) == 2) {              \
      using PR = PrecP;                    \
      CALL;                                \
    } else if ((prec) == 3) {              \
      using PR = PrecE;                    \
      CALL;                                \
    } else {                               \
      using PR = PrecD;                    \
      CALL;                                \
    }                                      \
  } while (0)

// The dynamic shared-memory limit is a per-function attribute of the device: it only ever
// grows here, so a launch prepared for one solve stays valid after another solve (of a
// smaller kmax) prepared the same kernels.
cudaError_t apcg_prepare_attributes(int kmax, int prec) {
  static std::mutex mu;
  static size_t set_bytes[64][4] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || prec < 0 || prec > 3) return cudaErrorInvalidValue;
  const size_t sm = apcg_smem_bytes(kmax);
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = set_bytes[dev][prec];
  if (sm <= cur) return cudaSuccess;
  KRS_DISPATCH(prec, e = prepare_attributes_t<PR>(sm));
  if (e == cudaSuccess) cur = sm;
  return e;
}

cudaError_t apcg_max_coresident(int kmax, int prec, int* blocks_per_sm) {
  cudaError_t e = cudaSuccess;
  KRS_DISPATCH(prec, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_apcg_persistent<PR>, TPB,
                                                                       apcg_smem_bytes(kmax)));
  return e;
}

template <typename Pr, typename TC>
static cudaError_t launch_init_t(const IterArgs& a, const void* bv, double* scal, cudaStream_t st,
                                 int64_t* launches) {
  using V = typename Pr::V;
  using M = typename Pr::M;
  using A = typename Pr::A;
  const size_t sm = apcg_smem_bytes(a.kmax);
  const int k = a.nc;
  const V* b = static_cast<const V*>(bv);
  const TC* C = static_cast<const TC*>(a.Ci ? a.Ci : a.C);
  const TC* AC = static_cast<const TC*>(a.ACi ? a.ACi : a.AC);
  V* x = static_cast<V*>(a.x);
  V* r = static_cast<V*>(a.r);
  V* u = static_cast<V*>(a.u);
  if (k > 0) {
    k_gemv_t_part<TC, V><<<a.P, TPB, sm, st>>>(C, a.ld, k, b, a.nbr, a.npc, a.vpart, a.vld);
    k_reduce_cols<<<(k * 32 + 255) / 256, 256, 0, st>>>(a.vpart, a.vld, a.P, k, a.tfull);
    k_small_gemv<<<(k * 32 + 255) / 256, 256, 0, st>>>(a.Ginv, a.ldg, k, a.nc_dense, a.dinv, a.tfull, a.sfull);
    *launches += 3;
  }
  k_init_xr<TC, V><<<a.P, TPB, sm, st>>>(C, AC, a.ld, k, a.sfull, b, x, r, a.nbr, a.npc, a.part);
  k_precond_rows<A, V><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a.precond, static_cast<const A*>(a.minv), r,
                                                                        u, a.n);
  *launches += 2;
  if (k > 0) {
    k_gemv_t_part<TC, V><<<a.P, TPB, sm, st>>>(AC, a.ld, k, u, a.nbr, a.npc, a.vpart, a.vld);
    k_reduce_cols<<<(k * 32 + 255) / 256, 256, 0, st>>>(a.vpart, a.vld, a.P, k, a.tfull);
    k_small_gemv<<<(k * 32 + 255) / 256, 256, 0, st>>>(a.Ginv, a.ldg, k, a.nc_dense, a.dinv, a.tfull, a.sfull);
    *launches += 3;
  }
  k_init_z<TC, V, M><<<a.P, TPB, sm, st>>>(C, a.ld, k, a.sfull, u, r, static_cast<M*>(a.Z), static_cast<M*>(a.W),
                                           a.nbr, a.npc, a.part, Pr::id == 3 ? static_cast<double*>(a.wv) : nullptr);
  k_init_finish<<<1, 96, 0, st>>>(a.part, a.P, scal, a.rho);
  *launches += 2;
  return cudaGetLastError();
}

// Set-up of x_0, r_0, z_0, w_0, rho_0, ||b||^2, ||r_0||^2 (scal[0..1]).  Counts launches.
cudaError_t apcg_launch_init(const IterArgs& a, const void* b, double* scal, cudaStream_t st, int64_t* launches) {
  // PrecP's first pass works from the FP64 C and AC (x_0, r_0 consistent with the FP64
  // recurrences); restarted passes use the FP32 copies that also hold the earlier passes'
  // directions
  if (a.prec == 2)
    return a.init32 ? launch_init_t<PrecP, float>(a, b, scal, st, launches)
                    : launch_init_t<PrecP, double>(a, b, scal, st, launches);
  if (a.prec == 1) return launch_init_t<PrecF, float>(a, b, scal, st, launches);
  if (a.prec == 3) return launch_init_t<PrecE, double>(a, b, scal, st, launches);
  return launch_init_t<PrecD, double>(a, b, scal, st, launches);
}

template <typename Pr>
static cudaError_t launch_persistent_t(const IterArgs& a, cudaStream_t st) {
  ApcgCtx<Pr> c = make_ctx<Pr>(a);
  void* args[] = {&c};
  return cudaLaunchCooperativeKernel((const void*)k_apcg_persistent<Pr>, dim3(a.P), dim3(TPB), args,
                                     apcg_smem_bytes(a.kmax), st);
}

cudaError_t apcg_launch_persistent(const IterArgs& a, cudaStream_t st, int64_t* launches) {
  *launches += 1;
  cudaError_t e = cudaSuccess;
  KRS_DISPATCH(a.prec, e = launch_persistent_t<PR>(a, st));
  return e;
}

size_t apcg_ctx_bytes() {
  static_assert(sizeof(ApcgCtx<PrecD>) == sizeof(ApcgCtx<PrecP>) && sizeof(ApcgCtx<PrecD>) == sizeof(ApcgCtx<PrecF>) &&
                    sizeof(ApcgCtx<PrecD>) == sizeof(ApcgCtx<PrecE>),
                "one context size for every precision");
  return sizeof(ApcgCtx<PrecD>);
}

void apcg_fill_ctx(const IterArgs& a, void* dst) {
  KRS_DISPATCH(a.prec, {
    ApcgCtx<PR> c = make_ctx<PR>(a);
    memcpy(dst, &c, sizeof(c));
  });
}

cudaError_t apcg_batched_coresident(int kmax, int prec, int* blocks_per_sm) {
  const size_t sm = apcg_smem_bytes(kmax);
  cudaError_t e = cudaSuccess;
  KRS_DISPATCH(prec, {
    e = cudaFuncSetAttribute((const void*)k_apcg_batched<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_apcg_batched<PR>, TPB, sm);
  });
  return e;
}

// out[4 p + w] = word w (status, done, m, j) of solve p's control block (the control
// pointer sits at the same offset in every precision's context)
__global__ void k_gather_ctrl(const ApcgCtx<PrecD>* __restrict__ ctxs, int count, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 4 * count) out[i] = *((volatile const int*)(ctxs[i >> 2].ctrl + (i & 3)));
}

cudaError_t apcg_gather_ctrl(const void* ctxs, int count, int* out, cudaStream_t st) {
  static_assert(offsetof(ApcgCtx<PrecD>, ctrl) == offsetof(ApcgCtx<PrecP>, ctrl) &&
                    offsetof(ApcgCtx<PrecD>, ctrl) == offsetof(ApcgCtx<PrecF>, ctrl) &&
                    offsetof(ApcgCtx<PrecD>, ctrl) == offsetof(ApcgCtx<PrecE>, ctrl),
                "control pointer at one offset");
  if (count <= 0) return cudaSuccess;
  k_gather_ctrl<<<(4 * count + 255) / 256, 256, 0, st>>>(static_cast<const ApcgCtx<PrecD>*>(ctxs), count, out);
  return cudaGetLastError();
}

template <typename Pr>
static cudaError_t launch_batched_t(const BatchLaunch& L, cudaStream_t st) {
  BatchArgs<Pr> B;
  B.ctxs = static_cast<const ApcgCtx<Pr>*>(L.ctxs);
  B.queue = L.queue;
  B.qoff = L.qoff;
  B.heads = L.heads;
  B.cta_group = L.cta_group;
  B.grp_cta0 = L.grp_cta0;
  B.grp_class = L.grp_class;
  B.quantum = L.quantum > 0 ? L.quantum : 0x7fffffff;
  B.drain_at = L.drain_at;
  B.idle = L.idle;
  B.gstop = L.gstop;
  B.mail = L.mail;
  B.gbar = L.gbar;
  B.gpart = L.gpart;
  B.gvpart = L.gvpart;
  B.ggpart = L.ggpart;
  B.vld = L.vld;
  B.spin_limit = L.spin_limit;
  B.bctrl = L.bctrl;
  void* args[] = {&B};
  return cudaLaunchCooperativeKernel((const void*)k_apcg_batched<Pr>, dim3(L.ctas), dim3(TPB), args,
                                     apcg_smem_bytes(L.kmax), st);
}

cudaError_t apcg_launch_batched(const BatchLaunch& L, int prec, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  KRS_DISPATCH(prec, e = launch_batched_t<PR>(L, st));
  return e;
}

template <typename Pr>
static cudaError_t launch_phases_t(const IterArgs& a, int j0, int j1, cudaStream_t st, int64_t* launches) {
  ApcgCtx<Pr> c = make_ctx<Pr>(a);
  const size_t sm = apcg_smem_bytes(a.kmax);
  for (int j = j0; j < j1; j++) {
    k_phase1<Pr><<<a.P, TPB, sm, st>>>(c, j);
    k_phase2<Pr><<<a.P, TPB, sm, st>>>(c, j);
    k_phase3<Pr><<<a.P, TPB, sm, st>>>(c, j);
    if (a.nc > SMALL_NC) {
      k_phase4<Pr><<<a.P, TPB, sm, st>>>(c, j);
      *launches += 1;
    }
    k_phase5<Pr><<<a.P, TPB, sm, st>>>(c, j);
    k_phase6<Pr><<<a.P, TPB, sm, st>>>(c, j);
    k_phase7<Pr><<<a.P, TPB, sm, st>>>(c, j);
    *launches += 6;
  }
  return cudaGetLastError();
}

// Launch the phases of iterations [j0, j1) (kernels mode).
cudaError_t apcg_launch_phases(const IterArgs& a, int j0, int j1, cudaStream_t st, int64_t* launches) {
  cudaError_t e = cudaSuccess;
  KRS_DISPATCH(a.prec, e = launch_phases_t<PR>(a, j0, j1, st, launches));
  return e;
}

}  // namespace krs
