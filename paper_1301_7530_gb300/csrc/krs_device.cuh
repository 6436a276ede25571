// krs_device.cuh -- device building blocks shared by the solve kernels.
//
// Partition.  A grid of P CTAs owns the block rows (nodes) in contiguous ranges of `npc`
// nodes (npc a multiple of 4), so every CTA's first scalar row 3*node0 is a multiple of 4
// and its multi-vector rows start 32-byte aligned (leading dimensions are multiples of
// 32 elements).  Every phase of an iteration works on the same CTA-local rows, so the
// per-CTA partial sums are formed in the same order whatever the execution mode.
//
// FP64 cost model (GB300, sm_103a): the FP64 pipe retires about 2 lane-operations per
// clock per SM, so one warp-wide FP64 instruction costs ~16 SM clocks whatever its
// active mask.  Inner loops therefore accumulate in registers (thread per column for
// V^T u, thread per row for V s) and only the per-CTA results are combined, once,
// through shared memory; no FP64 warp-shuffle trees run inside the streaming loops.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef KRS_TPB
#define KRS_TPB 512
#endif

namespace krs {

__host__ __device__ __forceinline__ int64_t kmin64(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr int TPB = KRS_TPB;
constexpr int ROW_CHUNK = 2048;     // rows staged in shared memory per pass

// control block (device int32 / int64 words)
enum Ctrl {
  CTRL_STATUS = 0,     // krs_status of the running solve (0 = running/ok)
  CTRL_DONE = 1,       // 1 once the iteration loop has terminated
  CTRL_M = 2,          // iterations completed
  CTRL_J = 3,          // current iteration index (multi-kernel mode)
  CTRL_ABORT = 4,      // set when a CTA gave up waiting: everyone leaves
  CTRL_WORDS = 8
};

// scalar partial slots per CTA
enum PartSlot { PS_WQ = 0, PS_RW = 1, PS_RR = 2, PS_RZ = 3, PS_STRIDE = 4 };

__device__ __forceinline__ void cta_rows(int nbr, int npc, int b, int64_t& r0, int64_t& r1) {
  int64_t n0 = (int64_t)b * npc;
  if (n0 > nbr) n0 = nbr;
  int64_t n1 = n0 + npc;
  if (n1 > nbr) n1 = nbr;
  r0 = 3 * n0;
  r1 = 3 * n1;
}

// ------------------------------------------------------------------------------------
// Block-wide sum of one double per thread (result valid in every thread).  The 512
// partials are folded by 4 warps (one per SM sub-partition, so their FP64 work runs in
// parallel) into 128 values, then by one warp.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red /* >= TPB + 1 doubles */) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  if (t < 128) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < TPB / 128; k++) s += red[t + 128 * k];
    red[t] = s;  // each t < 128 reads only indices congruent to t mod 128
  }
  __syncthreads();
  if (t < 32) {
    double s = red[t] + red[t + 32] + red[t + 64] + red[t + 96];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (t == 0) red[TPB] = s;
  }
  __syncthreads();
  double r = red[TPB];
  __syncthreads();
  return r;
}

// Same for two values at once.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red /* 2*TPB+2 */) {
  const int t = threadIdx.x;
  red[t] = a;
  red[TPB + t] = b;
  __syncthreads();
  if (t < 256) {
    const int base = (t < 128) ? 0 : TPB;
    const int tt = t & 127;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < TPB / 128; k++) s += red[base + tt + 128 * k];
    red[base + tt] = s;
  }
  __syncthreads();
  if (t < 64) {
    const int base = (t < 32) ? 0 : TPB;
    const int tt = t & 31;
    double s = red[base + tt] + red[base + tt + 32] + red[base + tt + 64] + red[base + tt + 96];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tt == 0) red[2 * TPB + (t >> 5)] = s;
  }
  __syncthreads();
  a = red[2 * TPB];
  b = red[2 * TPB + 1];
  __syncthreads();
}

// Sum of `cnt` doubles at p[0], p[stride], ... by one warp, fixed order (lane-strided,
// then a butterfly); the result is returned to every lane of the warp.
__device__ __forceinline__ double warp_sum_strided(const double* p, int cnt, int64_t stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < cnt; i += 32) s += p[(int64_t)i * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// ------------------------------------------------------------------------------------
// Grid barrier for the persistent (cooperative) kernel.  A monotone 64-bit arrival
// counter: barrier number k completes when the counter reaches k * P.  The wait is
// bounded: after `spin_limit` polls the CTA records KRS_ERR_TIMEOUT and the abort flag,
// and every CTA that sees the abort flag leaves.  Returns false when the CTA must exit.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(unsigned long long* counter, unsigned long long& target,
                                             unsigned P, int* ctrl, long long spin_limit,
                                             int timeout_code) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    target += P;
    int ok = 1;
    __threadfence();
    atomicAdd(counter, 1ull);
    long long spins = 0;
    for (;;) {
      unsigned long long v = *((volatile unsigned long long*)counter);
      if (v >= target) break;
      if (*((volatile int*)(ctrl + CTRL_ABORT)) != 0) { ok = 0; break; }
      if (++spins > spin_limit) {
        atomicCAS(ctrl + CTRL_STATUS, 0, timeout_code);
        atomicExch(ctrl + CTRL_ABORT, 1);
        ok = 0;
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------------------------
// Tall-skinny kernels on one CTA's rows [r0, r1) (r0 a multiple of 4).
// V: column-major, leading dimension ld (multiple of 4), rows >= n padded with zeros.
// ------------------------------------------------------------------------------------

// Load of data that is read-only for the whole kernel (NC = true: non-coherent path) or
// that other CTAs of the same (persistent) kernel may have written (NC = false).
template <bool NC>
__device__ __forceinline__ double4_32a ld4(const double* p) {
  if (NC) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    return make_double4_32a(a.x, a.y, b.x, b.y);
  }
  return *reinterpret_cast<const double4_32a*>(p);
}

// out[c] = sum_{i in [r0, r1)} V[c*ld + i] * u[i], c in [0, k).  Thread per column:
// each thread streams its column with 32-byte loads and keeps one accumulator; several
// row groups share the columns when k < TPB and are combined in shared memory.
// u: global vector (zero padded past n).  su: shared (ROW_CHUNK doubles); red: shared
// (TPB doubles).
template <bool NC>
__device__ __forceinline__ void cta_gemv_t(const double* __restrict__ V, int64_t ld, int k,
                                           const double* __restrict__ u, int64_t r0, int64_t r1,
                                           double* __restrict__ out, double* su, double* red) {
  const int t = threadIdx.x;
  const int64_t rows4 = ((r1 - r0) + 3) & ~int64_t(3);  // padded to a multiple of 4
  for (int cb = 0; cb < k; cb += TPB) {
    const int kc = min(k - cb, TPB);
    const int G = TPB / kc;  // row groups
    const int c = t % kc;
    const int g = t / kc;
    double acc = 0.0;
    for (int64_t ch = 0; ch < rows4; ch += ROW_CHUNK) {
      const int len = (int)kmin64(ROW_CHUNK, rows4 - ch);
      __syncthreads();
      for (int i = t; i < len; i += TPB) su[i] = u[r0 + ch + i];
      __syncthreads();
      if (g < G) {
        const int q4 = len >> 2;
        const int qa = (int)((int64_t)q4 * g / G), qb = (int)((int64_t)q4 * (g + 1) / G);
        const double* col = V + (int64_t)(cb + c) * ld + r0 + ch;
        const double4_32a* s4 = reinterpret_cast<const double4_32a*>(su);
        int q = qa;
        for (; q + 2 <= qb; q += 2) {
          const double4_32a a0 = ld4<NC>(col + 4 * q), a1 = ld4<NC>(col + 4 * q + 4);
          const double4_32a b0 = s4[q], b1 = s4[q + 1];
          acc += a0.x * b0.x; acc += a0.y * b0.y; acc += a0.z * b0.z; acc += a0.w * b0.w;
          acc += a1.x * b1.x; acc += a1.y * b1.y; acc += a1.z * b1.z; acc += a1.w * b1.w;
        }
        for (; q < qb; q++) {
          const double4_32a a0 = ld4<NC>(col + 4 * q), b0 = s4[q];
          acc += a0.x * b0.x; acc += a0.y * b0.y; acc += a0.z * b0.z; acc += a0.w * b0.w;
        }
      }
    }
    __syncthreads();
    if (g < G) red[g * kc + c] = acc;
    __syncthreads();
    if (t < kc) {
      double sum = red[t];
      for (int gg = 1; gg < G; gg++) sum += red[gg * kc + t];
      out[cb + t] = sum;
    }
  }
  __syncthreads();
}

// z[i] = u[i] + sgn * sum_{c<k} V[c*ld + i] * s[c] for i in [r0, r1) (u == nullptr: 0).
// Thread per 4 rows; when the CTA has few rows, column groups split the k columns and
// are combined in shared memory.  s: shared (k doubles).  red: shared (4*TPB doubles).
template <bool NC>
__device__ __forceinline__ void cta_gemv_n(const double* __restrict__ V, int64_t ld, int k,
                                           const double* s, double sgn, const double* u,
                                           double* z, int64_t r0, int64_t r1, double* red) {
  const int t = threadIdx.x;
  const int64_t L = r1 - r0;
  const int64_t q4 = (L + 3) >> 2;
  for (int64_t qb0 = 0; qb0 < q4; qb0 += TPB) {
    const int nq = (int)kmin64(TPB, q4 - qb0);
    const int G = (k > 0) ? max(1, min(TPB / nq, k)) : 1;  // column groups
    const int q = t % nq;
    const int g = t / nq;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (g < G && k > 0) {
      const int ca = (int)((int64_t)k * g / G), cbnd = (int)((int64_t)k * (g + 1) / G);
      const int64_t row = r0 + 4 * (qb0 + q);
      int c = ca;
      for (; c + 2 <= cbnd; c += 2) {
        const double4_32a v0 = ld4<NC>(V + (int64_t)c * ld + row);
        const double4_32a v1 = ld4<NC>(V + (int64_t)(c + 1) * ld + row);
        const double s0 = s[c], s1 = s[c + 1];
        a0 += v0.x * s0; a1 += v0.y * s0; a2 += v0.z * s0; a3 += v0.w * s0;
        a0 += v1.x * s1; a1 += v1.y * s1; a2 += v1.z * s1; a3 += v1.w * s1;
      }
      for (; c < cbnd; c++) {
        const double4_32a v0 = ld4<NC>(V + (int64_t)c * ld + row);
        const double s0 = s[c];
        a0 += v0.x * s0; a1 += v0.y * s0; a2 += v0.z * s0; a3 += v0.w * s0;
      }
    }
    if (G > 1) {
      __syncthreads();
      double4_32a* r4 = reinterpret_cast<double4_32a*>(red);
      if (g < G) r4[g * nq + q] = make_double4_32a(a0, a1, a2, a3);
      __syncthreads();
      if (t < nq) {
        double4_32a acc = r4[t];
        for (int gg = 1; gg < G; gg++) {
          const double4_32a v = r4[gg * nq + t];
          acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        a0 = acc.x; a1 = acc.y; a2 = acc.z; a3 = acc.w;
      }
    }
    if (t < nq) {
      const int64_t row = r0 + 4 * (qb0 + t);
      const double aa[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        if (row + e < r1) z[row + e] = (u ? u[row + e] : 0.0) + sgn * aa[e];
      }
    }
  }
  __syncthreads();
}

// q = A w on one CTA's nodes (thread per scalar row: 3 FMAs per stored block, no
// reduction), adds the thread's (w, q) and (r, w) contributions to wq / rw.  The matrix
// is read through the non-coherent path; w (written by other CTAs of a persistent kernel)
// is not.
__device__ __forceinline__ void cta_spmv(const int* __restrict__ rp, const int* __restrict__ ci,
                                         const double* __restrict__ vals,
                                         const double* __restrict__ w, double* __restrict__ q,
                                         const double* __restrict__ r, int64_t r0, int64_t r1,
                                         double& wq, double& rw) {
  for (int64_t row = r0 + threadIdx.x; row < r1; row += TPB) {
    const int64_t node = row / 3;
    const int d = (int)(row - 3 * node);
    const int ka = __ldg(rp + node), kb = __ldg(rp + node + 1);
    double acc = 0.0;
    for (int k = ka; k < kb; k++) {
      const int64_t cc = 3 * (int64_t)__ldg(ci + k);
      const double* a = vals + 9 * (int64_t)k + 3 * d;
      acc += __ldg(a + 0) * w[cc + 0];
      acc += __ldg(a + 1) * w[cc + 1];
      acc += __ldg(a + 2) * w[cc + 2];
    }
    q[row] = acc;
    const double wr = w[row];
    wq += wr * acc;
    if (r) rw += r[row] * wr;
  }
}

// u = M^-1 r on the CTA's rows (r read from global; Jacobi: minv[row]; block Jacobi:
// minv[9*node + 3*d + e]; identity: copy).
__device__ __forceinline__ double precond_row(int kind, const double* __restrict__ minv,
                                              const double* __restrict__ r, int64_t row) {
  if (kind == 0) return minv[row] * r[row];
  if (kind == 1) {
    const int64_t node = row / 3;
    const int d = (int)(row - 3 * node);
    const double* m = minv + 9 * node + 3 * d;
    return m[0] * r[3 * node] + m[1] * r[3 * node + 1] + m[2] * r[3 * node + 2];
  }
  return r[row];
}

}  // namespace krs
