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
// active mask.  Inner loops therefore accumulate in registers (a warp per 8-column block
// for V^T u, thread per row quad for V s) and partial sums are combined once per column
// block or per CTA; no FP64 warp-shuffle trees run inside the streaming loops.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
    // release: this CTA's writes (ordered before by __syncthreads) become visible with the
    // arrival; acquire on the polls: the other CTAs' writes are visible after the exit
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(counter), "l"(1ull) : "memory");
    long long spins = 0;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(counter) : "memory");
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
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------------------------
// Double-float numbers (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2): a value hi + lo held as
// two FP32 numbers with |lo| <= ulp(hi) / 2, i.e. a 48-bit significand in 8 bytes.  On
// GB300 an FP64 instruction retires 2 lanes per clock per SM against 128 for FP32, so a
// tall-skinny product over double-float storage runs on the FP32 pipes (about 12 FP32
// operations per element) and is bound by memory, not by the FP64 pipe.  Conversions
// to and from double use FP64 arithmetic and appear only O(n) times per iteration.
// Range: FP32 exponents (|values| within about 1e-30 .. 1e38 keep the full significand).
// ------------------------------------------------------------------------------------
struct __align__(8) dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ __forceinline__ explicit dfl(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);  // d - hi is exact in double
  }
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) dfl4 { dfl x, y, z, w; };
struct __align__(16) dfl2 { dfl x, y; };

// Running sum of products in double-float form: s + c, with every product x * y taken
// exactly to 2^-48 relative (error-free FP32 product of the high parts by FMA, plus the
// two cross terms) and added to s by an error-free two-sum whose error goes to c.
struct dacc {
  float s, c;
};
__device__ __forceinline__ void dacc_add(dacc& a, float p, float e) {
  const float s = __fadd_rn(a.s, p);
  const float bp = __fsub_rn(s, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  a.c = __fadd_rn(a.c, __fadd_rn(err, e));
  a.s = s;
}

// Accumulator of a product stream over values of type T: T itself for double and float
// (a += x * y, one FMA), dacc for double-float.  out(): the accumulated value as the type
// the per-thread results are combined in (T, or double for double-float).
template <typename T>
struct Acc {
  using type = T;
  using out_t = T;
  __device__ static __forceinline__ T zero() { return T(0); }
  __device__ static __forceinline__ void mac(T& a, T x, T y) { a += x * y; }
  __device__ static __forceinline__ T out(T a) { return a; }
  __device__ static __forceinline__ double fold4(T a0, T a1, T a2, T a3) { return (double)((a0 + a1) + (a2 + a3)); }
};
template <>
struct Acc<dfl> {
  using type = dacc;
  using out_t = double;
  __device__ static __forceinline__ dacc zero() { return dacc{0.f, 0.f}; }
  __device__ static __forceinline__ void mac(dacc& a, dfl x, dfl y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    dacc_add(a, p, e);
  }
  __device__ static __forceinline__ double out(dacc a) { return (double)a.s + (double)a.c; }
  __device__ static __forceinline__ double fold4(dacc a0, dacc a1, dacc a2, dacc a3) {
    return (out(a0) + out(a1)) + (out(a2) + out(a3));
  }
};

// ------------------------------------------------------------------------------------
// Value types.  The FP64 path instantiates everything with T = double; the inner solve of
// the mixed-precision refinement with T = float (storage and arithmetic), while every
// partial sum that crosses CTAs is a double.  Double-float storage (T = dfl) holds the
// search directions of the double-float precision.
// ------------------------------------------------------------------------------------
template <typename T>
struct VT;
template <>
struct VT<double> {
  using V4 = double4_32a;  // four rows, 32 bytes
  using V2 = double2;      // 16 bytes
  __device__ static __forceinline__ V4 make4(double a, double b, double c, double d) {
    return make_double4_32a(a, b, c, d);
  }
};
template <>
struct VT<float> {
  using V4 = float4;  // four rows, 16 bytes
  using V2 = float2;  // 8 bytes
  __device__ static __forceinline__ V4 make4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <>
struct VT<dfl> {
  using V4 = dfl4;  // four rows, 32 bytes
  using V2 = dfl2;
  __device__ static __forceinline__ V4 make4(dfl a, dfl b, dfl c, dfl d) { return dfl4{a, b, c, d}; }
};

// Load of four consecutive rows of data that is read-only for the whole kernel (NC = true:
// non-coherent path) or that other CTAs of the same (persistent) kernel may have written
// (NC = false).
template <bool NC, typename T>
__device__ __forceinline__ typename VT<T>::V4 ld4(const T* p);

template <>
__device__ __forceinline__ double4_32a ld4<true, double>(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  return make_double4_32a(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ double4_32a ld4<false, double>(const double* p) {
  return *reinterpret_cast<const double4_32a*>(p);
}
template <>
__device__ __forceinline__ float4 ld4<true, float>(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ float4 ld4<false, float>(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
template <>
__device__ __forceinline__ dfl4 ld4<true, dfl>(const dfl* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p + 2));
  dfl4 v;
  v.x.hi = a.x; v.x.lo = a.y; v.y.hi = a.z; v.y.lo = a.w;
  v.z.hi = b.x; v.z.lo = b.y; v.w.hi = b.z; v.w.lo = b.w;
  return v;
}
template <>
__device__ __forceinline__ dfl4 ld4<false, dfl>(const dfl* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 2);
  dfl4 v;
  v.x.hi = a.x; v.x.lo = a.y; v.y.hi = a.z; v.y.lo = a.w;
  v.z.hi = b.x; v.z.lo = b.y; v.w.hi = b.z; v.w.lo = b.w;
  return v;
}

// Four consecutive rows of a vector of type TU, as the four-row vector of type T.
template <typename T, typename TU>
__device__ __forceinline__ typename VT<T>::V4 load4_as(const TU* p) {
  const typename VT<TU>::V4 y = *reinterpret_cast<const typename VT<TU>::V4*>(p);
  return VT<T>::make4((T)y.x, (T)y.y, (T)y.z, (T)y.w);
}

// ------------------------------------------------------------------------------------
// Tall-skinny kernels on one CTA's rows [r0, r1) (r0 a multiple of 4).
// V: column-major, leading dimension ld (multiple of 4), rows >= n padded with zeros.
// ------------------------------------------------------------------------------------

// Few columns (k <= TPB/32): warps instead of threads own the columns -- Gw = (TPB/32)/k
// warps per column split the rows, lanes read consecutive four-row pieces of the column
// (contiguous per warp load), each warp folds its lanes with one shuffle tree, and the Gw
// warp partials are summed in a fixed order.  Used by cta_gemv_t.
template <bool NC, typename T, typename TU>
__device__ __forceinline__ void cta_gemv_t_few(const T* __restrict__ V, int64_t ld, int k,
                                               const TU* __restrict__ u, int64_t r0, int64_t r1,
                                               double* __restrict__ out, double* red) {
  using V4 = typename VT<T>::V4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int W = TPB / 32;
  const int Gw = W / k;
  const int q4 = (int)(((r1 - r0) + 3) >> 2);
  if (warp < Gw * k) {
    const int c = warp / Gw, g = warp % Gw;
    const int qa = (int)((int64_t)q4 * g / Gw), qb = (int)((int64_t)q4 * (g + 1) / Gw);
    const T* col = V + (int64_t)c * ld + r0;
    const TU* uu = u + r0;
    using AC = Acc<T>;
    typename AC::type a0 = AC::zero(), a1 = AC::zero(), a2 = AC::zero(), a3 = AC::zero();
    for (int q = qa + lane; q < qb; q += 32) {
      const V4 x = ld4<NC, T>(col + 4 * q);
      const V4 y = load4_as<T, TU>(uu + 4 * q);
      AC::mac(a0, x.x, y.x); AC::mac(a1, x.y, y.y); AC::mac(a2, x.z, y.z); AC::mac(a3, x.w, y.w);
    }
    double v = AC::fold4(a0, a1, a2, a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = red[threadIdx.x * Gw];
    for (int g = 1; g < Gw; g++) s += red[threadIdx.x * Gw + g];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// Tall-skinny layouts that favour long contiguous runs per column:
//   cta_gemv_t_wb (V^T u; double-float, and FP64 as cta_gemv_t selects): a warp takes
//     a block of 8 columns over a range of row pairs; lane l reads row pairs l, l + 32, ...
//     of all 8 columns (512 contiguous bytes of each column per warp load), accumulates per
//     column, and the 8 x 32 lane sums are folded once per block by a transposed shuffle
//     reduction (4 + 2 + 1 + 1 + 1 adds per lane for 8 columns).  Units (column block, row
//     range) are spread over the 16 warps.  A thread per column (the older layout) reads
//     32 separate 128-byte runs per warp load: it streamed 2.9-3.7 TB/s at 696 rows per CTA
//     and 1.7 TB/s at 5,340 (the 64^3 cube), against 4.7-5.3 TB/s for this layout.
//   cta_gemv_n_df (u - V s, double-float): thread per row quad; G = floor(TPB / quads)
//     column groups so that one pass covers every quad; 8-column unroll (256 bytes in flight
//     per thread).
// Row pairs / quads past r1 read the zero padding of the columns (r0 is a multiple of 4;
// a column holds ld >= n + 1 values when n is odd).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ dacc dacc_sum(dacc a, dacc b) {
  dacc_add(a, b.s, b.c);
  return a;
}
__device__ __forceinline__ dacc dacc_shfl(dacc a, int m) {
  return dacc{__shfl_xor_sync(0xffffffffu, a.s, m), __shfl_xor_sync(0xffffffffu, a.c, m)};
}

// Per-type pieces of the warp-block layout of V^T u: a row pair of a column (16 bytes), a
// multiply-add of two row pairs into the accumulator, and the lane combination.
template <typename T>
struct WB;
template <>
struct WB<double> {
  using acc = double;
  using P2 = double2;
  __device__ static __forceinline__ acc zero() { return 0.0; }
  template <bool NC>
  __device__ static __forceinline__ P2 load(const double* p) {
    return NC ? __ldg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
  }
  __device__ static __forceinline__ P2 none() { return make_double2(0.0, 0.0); }
  __device__ static __forceinline__ void mac2(acc& a, P2 x, P2 y) {
    a += x.x * y.x;
    a += x.y * y.y;
  }
  __device__ static __forceinline__ acc add(acc a, acc b) { return a + b; }
  __device__ static __forceinline__ acc shfl(acc a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
  __device__ static __forceinline__ double out(acc a) { return a; }
};
template <>
struct WB<dfl> {
  using acc = dacc;
  using P2 = float4;  // (hi, lo) of two rows
  __device__ static __forceinline__ acc zero() { return dacc{0.f, 0.f}; }
  template <bool NC>
  __device__ static __forceinline__ P2 load(const dfl* p) {
    return NC ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
  }
  __device__ static __forceinline__ P2 none() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static __forceinline__ void mac2(acc& a, P2 x, P2 y) {
    dfl x0, x1, y0, y1;
    x0.hi = x.x; x0.lo = x.y; x1.hi = x.z; x1.lo = x.w;
    y0.hi = y.x; y0.lo = y.y; y1.hi = y.z; y1.lo = y.w;
    Acc<dfl>::mac(a, x0, y0);
    Acc<dfl>::mac(a, x1, y1);
  }
  __device__ static __forceinline__ acc add(acc a, acc b) { return dacc_sum(a, b); }
  __device__ static __forceinline__ acc shfl(acc a, int m) { return dacc_shfl(a, m); }
  __device__ static __forceinline__ double out(acc a) { return Acc<dfl>::out(a); }
};

// Row ranges per 8-column block: split only when there are fewer blocks than warps (every
// warp then gets a unit).  Splitting further to fill a last, partial wave of units was
// measured slower (shorter per-lane runs, more lane reductions).
__device__ __forceinline__ int wb_row_ranges(int nblk) {
  constexpr int NW = TPB / 32;
  return nblk >= NW ? 1 : (NW + nblk - 1) / nblk;
}

// out[c] = sum_{i in [r0, r1)} V[c*ld + i] u[i] (c < k), V and u of type T (double or
// double-float), as doubles: the warp-block layout above.  red: shared, >= 256 doubles
// (row-range partials).  The summation order depends only on k and the rows.
template <bool NC, typename T>
__device__ __forceinline__ void cta_gemv_t_wb(const T* __restrict__ V, int64_t ld, int k, const T* __restrict__ u,
                                              int64_t r0, int64_t r1, double* __restrict__ out, double* red) {
  using W = WB<T>;
  using A = typename W::acc;
  using P2 = typename W::P2;
  constexpr int CB = 8;
  constexpr int NW = TPB / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t pairs = ((r1 - r0) + 1) >> 1;
  const int nblk = (k + CB - 1) / CB;
  const int Rg = wb_row_ranges(nblk);  // when Rg > 1: Rg * k <= (16 / nblk + 1) * 8 nblk <= 248
  const int units = nblk * Rg;
  const T* u2 = u + r0;
  for (int un = warp; un < units; un += NW) {
    const int blk = un / Rg, rg = un - blk * Rg;
    const int c0 = blk * CB;
    const int nc = min(CB, k - c0);
    const int64_t pa = pairs * rg / Rg, pb = pairs * (rg + 1) / Rg;
    A acc[CB];
#pragma unroll
    for (int c = 0; c < CB; c++) acc[c] = W::zero();
    const T* col0 = V + (int64_t)c0 * ld + r0;
    for (int64_t p = pa + lane; p < pb; p += 32) {
      P2 x[CB];
#pragma unroll
      for (int c = 0; c < CB; c++) x[c] = c < nc ? W::template load<NC>(col0 + (int64_t)c * ld + 2 * p) : W::none();
      const P2 y = W::template load<false>(u2 + 2 * p);
#pragma unroll
      for (int c = 0; c < CB; c++) W::mac2(acc[c], x[c], y);
    }
    // transposed reduction: after it, lane 4c holds column c0 + c (sum over all 32 lanes)
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    A v4[4];
#pragma unroll
    for (int i = 0; i < 4; i++) v4[i] = W::add(b4 ? acc[4 + i] : acc[i], W::shfl(b4 ? acc[i] : acc[4 + i], 16));
    A v2[2];
#pragma unroll
    for (int i = 0; i < 2; i++) v2[i] = W::add(b3 ? v4[2 + i] : v4[i], W::shfl(b3 ? v4[i] : v4[2 + i], 8));
    A v1 = W::add(b2 ? v2[1] : v2[0], W::shfl(b2 ? v2[0] : v2[1], 4));
    v1 = W::add(v1, W::shfl(v1, 1));
    v1 = W::add(v1, W::shfl(v1, 2));
    if ((lane & 3) == 0 && (lane >> 2) < nc) {
      const double r = W::out(v1);
      if (Rg == 1) out[c0 + (lane >> 2)] = r;
      else red[rg * k + c0 + (lane >> 2)] = r;
    }
  }
  if (Rg > 1) {  // fixed-order sum of the row ranges
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += TPB) {
      double s = red[c];
      for (int g = 1; g < Rg; g++) s += red[g * k + c];
      out[c] = s;
    }
  }
  __syncthreads();
}

// z[i] = u[i] + sgn * sum_{c<k} V[c*ld + i] * s[c] for i in [r0, r1), double-float V and s
// (shared); u of type TU (nullptr: 0); z of type TZ; z2 (optional): the result as a double.
// red: shared, TPB four-row double vectors.
template <bool NC, typename TU, typename TZ>
__device__ __forceinline__ void cta_gemv_n_df(const dfl* __restrict__ V, int64_t ld, int k, const dfl* s, double sgn,
                                              const TU* u, TZ* z, int64_t r0, int64_t r1, void* red, double* z2) {
  constexpr int CU = 8;
  const int t = threadIdx.x;
  const int64_t q4 = ((r1 - r0) + 3) >> 2;
  for (int64_t qb0 = 0; qb0 < q4; ) {
    const int64_t remq = q4 - qb0;
    int G = remq >= TPB ? 1 : (int)(TPB / remq);  // column groups (one pass over the quads)
    if (G > k) G = k > 0 ? k : 1;
    const int nq = (int)kmin64(remq, TPB / G);
    const int q = t % nq, g = t / nq;
    dacc a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
    if (g < G && k > 0) {
      const int ca = (int)((int64_t)k * g / G), cb = (int)((int64_t)k * (g + 1) / G);
      const int64_t row = r0 + 4 * (qb0 + q);
      int c = ca;
      for (; c + CU <= cb; c += CU) {
        dfl4 v[CU];
#pragma unroll
        for (int e = 0; e < CU; e++) v[e] = ld4<NC, dfl>(V + (int64_t)(c + e) * ld + row);
#pragma unroll
        for (int e = 0; e < CU; e++) {
          const dfl se = s[c + e];
          Acc<dfl>::mac(a0, v[e].x, se); Acc<dfl>::mac(a1, v[e].y, se);
          Acc<dfl>::mac(a2, v[e].z, se); Acc<dfl>::mac(a3, v[e].w, se);
        }
      }
      for (; c < cb; c++) {
        const dfl4 v0 = ld4<NC, dfl>(V + (int64_t)c * ld + row);
        const dfl se = s[c];
        Acc<dfl>::mac(a0, v0.x, se); Acc<dfl>::mac(a1, v0.y, se);
        Acc<dfl>::mac(a2, v0.z, se); Acc<dfl>::mac(a3, v0.w, se);
      }
    }
    double f0 = Acc<dfl>::out(a0), f1 = Acc<dfl>::out(a1), f2 = Acc<dfl>::out(a2), f3 = Acc<dfl>::out(a3);
    if (G > 1) {
      __syncthreads();
      double4_32a* r4 = reinterpret_cast<double4_32a*>(red);
      if (g < G) r4[g * nq + q] = make_double4_32a(f0, f1, f2, f3);
      __syncthreads();
      for (int st = 1; st < G; st <<= 1) {  // pairwise tree over the column groups (fixed order)
        if (g < G && (g % (2 * st)) == 0 && g + st < G) {
          const double4_32a v = r4[(g + st) * nq + q];
          double4_32a acc = r4[g * nq + q];
          acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
          r4[g * nq + q] = acc;
        }
        __syncthreads();
      }
      if (t < nq) {
        const double4_32a acc = r4[t];
        f0 = acc.x; f1 = acc.y; f2 = acc.z; f3 = acc.w;
      }
    }
    if (t < nq) {
      const int64_t row = r0 + 4 * (qb0 + t);
      const double ff[4] = {f0, f1, f2, f3};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        if (row + e < r1) {
          const double v = (u ? (double)u[row + e] : 0.0) + sgn * ff[e];
          z[row + e] = (TZ)v;
          if (z2) z2[row + e] = v;
        }
      }
    }
    qb0 += nq;
  }
  __syncthreads();
}

// out[c] = sum_{i in [r0, r1)} V[c*ld + i] * u[i], c in [0, k), as doubles.  Thread per
// column: each thread streams its column with four-row vector loads into four independent
// accumulators (no dependent FMA chain).  Columns are taken in blocks of kc with
// G = ceil(TPB / rem) row groups each (kc = TPB / G), so that all threads stay busy
// whatever k is; the groups are combined by a pairwise tree in a fixed order.  Double-float,
// and FP64 with 17..256 columns or more than ROW_CHUNK rows, take the warp-block layout
// (cta_gemv_t_wb).
// u: global vector (zero padded past n).  su: shared (ROW_CHUNK values of T); red: shared
// (4 * TPB doubles).
template <bool NC, typename T, typename TU = T>
__device__ __forceinline__ void cta_gemv_t(const T* __restrict__ V, int64_t ld, int k,
                                           const TU* __restrict__ u, int64_t r0, int64_t r1,
                                           double* __restrict__ out, T* su, double* red) {
  using V4 = typename VT<T>::V4;
  if constexpr (std::is_same<T, dfl>::value) {
    static_assert(std::is_same<TU, dfl>::value, "double-float V^T u takes a double-float u");
    cta_gemv_t_wb<NC, dfl>(V, ld, k, u, r0, r1, out, red);
    return;
  }
  if constexpr (std::is_same<T, double>::value && std::is_same<TU, double>::value) {
    // FP64: the warp-block layout up to 256 columns, and at any width once a CTA owns more
    // rows than one staging chunk; thread per column streamed faster at ~700 rows per CTA and
    // 400 columns (3.7 against 3.4 TB/s), far slower at 5,340 rows (1.7 against 4.8 TB/s)
    if (k > TPB / 32 && (k <= 256 || r1 - r0 > ROW_CHUNK)) {
      cta_gemv_t_wb<NC, double>(V, ld, k, u, r0, r1, out, red);
      return;
    }
  }
  if (k <= TPB / 32) {
    cta_gemv_t_few<NC, T, TU>(V, ld, k, u, r0, r1, out, red);
    return;
  }
  const int t = threadIdx.x;
  const int64_t rows4 = ((r1 - r0) + 3) & ~int64_t(3);  // padded to a multiple of 4
  const bool one_chunk = rows4 <= ROW_CHUNK;
  if (one_chunk) {
    __syncthreads();
    for (int i = t; i < (int)rows4; i += TPB) su[i] = (T)u[r0 + i];
    __syncthreads();
  }
  int cb = 0;
  while (cb < k) {
    const int rem = k - cb;
    const int G = (rem >= TPB) ? 1 : (TPB + rem - 1) / rem;  // row groups
    const int kc = min(rem, TPB / G);
    const int c = t % kc;
    const int g = t / kc;
    using AC = Acc<T>;
    typename AC::type a0 = AC::zero(), a1 = AC::zero(), a2 = AC::zero(), a3 = AC::zero();
    for (int64_t ch = 0; ch < rows4; ch += ROW_CHUNK) {
      const int len = (int)kmin64(ROW_CHUNK, rows4 - ch);
      if (!one_chunk) {
        __syncthreads();
        for (int i = t; i < len; i += TPB) su[i] = (T)u[r0 + ch + i];
        __syncthreads();
      }
      if (g < G) {
        const int q4 = len >> 2;
        const int qa = (int)((int64_t)q4 * g / G), qb = (int)((int64_t)q4 * (g + 1) / G);
        const T* col = V + (int64_t)(cb + c) * ld + r0 + ch;
        const V4* s4 = reinterpret_cast<const V4*>(su);
        int q = qa;
        for (; q + 4 <= qb; q += 4) {
          const V4 x0 = ld4<NC, T>(col + 4 * q), x1 = ld4<NC, T>(col + 4 * q + 4);
          const V4 x2 = ld4<NC, T>(col + 4 * q + 8), x3 = ld4<NC, T>(col + 4 * q + 12);
          const V4 y0 = s4[q], y1 = s4[q + 1], y2 = s4[q + 2], y3 = s4[q + 3];
          AC::mac(a0, x0.x, y0.x); AC::mac(a1, x0.y, y0.y); AC::mac(a2, x0.z, y0.z); AC::mac(a3, x0.w, y0.w);
          AC::mac(a0, x1.x, y1.x); AC::mac(a1, x1.y, y1.y); AC::mac(a2, x1.z, y1.z); AC::mac(a3, x1.w, y1.w);
          AC::mac(a0, x2.x, y2.x); AC::mac(a1, x2.y, y2.y); AC::mac(a2, x2.z, y2.z); AC::mac(a3, x2.w, y2.w);
          AC::mac(a0, x3.x, y3.x); AC::mac(a1, x3.y, y3.y); AC::mac(a2, x3.z, y3.z); AC::mac(a3, x3.w, y3.w);
        }
        for (; q < qb; q++) {
          const V4 x0 = ld4<NC, T>(col + 4 * q), y0 = s4[q];
          AC::mac(a0, x0.x, y0.x); AC::mac(a1, x0.y, y0.y); AC::mac(a2, x0.z, y0.z); AC::mac(a3, x0.w, y0.w);
        }
      }
    }
    __syncthreads();
    if (g < G) red[g * kc + c] = AC::fold4(a0, a1, a2, a3);
    __syncthreads();
    // combine the G row groups: pairwise tree (fixed order), log2(G) parallel rounds
    for (int st = 1; st < G; st <<= 1) {
      if (g < G && (g % (2 * st)) == 0 && g + st < G) red[g * kc + c] += red[(g + st) * kc + c];
      __syncthreads();
    }
    if (t < kc) out[cb + t] = red[t];
    cb += kc;
  }
  __syncthreads();
}

// z[i] = u[i] + sgn * sum_{c<k} V[c*ld + i] * s[c] for i in [r0, r1) (u == nullptr: 0).
// Thread per 4 rows (four independent accumulators), four-column unroll; quads are taken
// in blocks of qc with G = ceil(TPB / remaining quads) column groups each (qc = TPB / G),
// combined by a pairwise tree in a fixed order.  s: shared (k values of T).  red: shared
// scratch of TPB four-row vectors of T (32 bytes each for double-float).  Double-float
// V: the column sums are formed in double-float and combined in double.  z2 (optional):
// the same result also stored as a double.
template <bool NC, typename T, typename TU = T, typename TZ = T>
__device__ __forceinline__ void cta_gemv_n(const T* __restrict__ V, int64_t ld, int k, const T* s, T sgn,
                                           const TU* u, TZ* z, int64_t r0, int64_t r1, void* red,
                                           double* z2 = nullptr) {
  if constexpr (std::is_same<T, dfl>::value) {
    cta_gemv_n_df<NC, TU, TZ>(V, ld, k, s, (double)sgn, u, z, r0, r1, red, z2);
    return;
  }
  using V4 = typename VT<T>::V4;
  using AC = Acc<T>;
  using FT = typename AC::out_t;          // type the column groups are combined in
  using F4 = typename VT<FT>::V4;
  const int t = threadIdx.x;
  const int64_t L = r1 - r0;
  const int64_t q4 = (L + 3) >> 2;
  int64_t qb0 = 0;
  while (qb0 < q4) {
    const int64_t remq = q4 - qb0;
    int G = (remq >= TPB) ? 1 : (int)((TPB + remq - 1) / remq);  // column groups
    if (G > k) G = (k > 0) ? k : 1;
    const int nq = (int)kmin64(remq, TPB / G);
    const int q = t % nq;
    const int g = t / nq;
    typename AC::type a0 = AC::zero(), a1 = AC::zero(), a2 = AC::zero(), a3 = AC::zero();
    if (g < G && k > 0) {
      const int ca = (int)((int64_t)k * g / G), cbnd = (int)((int64_t)k * (g + 1) / G);
      const int64_t row = r0 + 4 * (qb0 + q);
      int c = ca;
      for (; c + 4 <= cbnd; c += 4) {
        const V4 v0 = ld4<NC, T>(V + (int64_t)c * ld + row);
        const V4 v1 = ld4<NC, T>(V + (int64_t)(c + 1) * ld + row);
        const V4 v2 = ld4<NC, T>(V + (int64_t)(c + 2) * ld + row);
        const V4 v3 = ld4<NC, T>(V + (int64_t)(c + 3) * ld + row);
        const T s0 = s[c], s1 = s[c + 1], s2 = s[c + 2], s3 = s[c + 3];
        AC::mac(a0, v0.x, s0); AC::mac(a1, v0.y, s0); AC::mac(a2, v0.z, s0); AC::mac(a3, v0.w, s0);
        AC::mac(a0, v1.x, s1); AC::mac(a1, v1.y, s1); AC::mac(a2, v1.z, s1); AC::mac(a3, v1.w, s1);
        AC::mac(a0, v2.x, s2); AC::mac(a1, v2.y, s2); AC::mac(a2, v2.z, s2); AC::mac(a3, v2.w, s2);
        AC::mac(a0, v3.x, s3); AC::mac(a1, v3.y, s3); AC::mac(a2, v3.z, s3); AC::mac(a3, v3.w, s3);
      }
      for (; c < cbnd; c++) {
        const V4 v0 = ld4<NC, T>(V + (int64_t)c * ld + row);
        const T s0 = s[c];
        AC::mac(a0, v0.x, s0); AC::mac(a1, v0.y, s0); AC::mac(a2, v0.z, s0); AC::mac(a3, v0.w, s0);
      }
    }
    FT f0 = AC::out(a0), f1 = AC::out(a1), f2 = AC::out(a2), f3 = AC::out(a3);
    if (G > 1) {
      __syncthreads();
      F4* r4 = reinterpret_cast<F4*>(red);
      if (g < G) r4[g * nq + q] = VT<FT>::make4(f0, f1, f2, f3);
      __syncthreads();
      // pairwise tree over the G column groups (fixed order), log2(G) parallel rounds
      for (int st = 1; st < G; st <<= 1) {
        if (g < G && (g % (2 * st)) == 0 && g + st < G) {
          const F4 v = r4[(g + st) * nq + q];
          F4 acc = r4[g * nq + q];
          acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
          r4[g * nq + q] = acc;
        }
        __syncthreads();
      }
      if (t < nq) {
        const F4 acc = r4[t];
        f0 = acc.x; f1 = acc.y; f2 = acc.z; f3 = acc.w;
      }
    }
    if (t < nq) {
      const int64_t row = r0 + 4 * (qb0 + t);
      const FT ff[4] = {f0, f1, f2, f3};
      const FT sg = (FT)sgn;
#pragma unroll
      for (int e = 0; e < 4; e++) {
        if (row + e < r1) {
          const FT v = (u ? (FT)u[row + e] : FT(0)) + sg * ff[e];
          z[row + e] = (TZ)v;
          if (z2) z2[row + e] = (double)v;
        }
      }
    }
    qb0 += nq;
  }
  __syncthreads();
}

// q = A w on one CTA's nodes [r0/3, r1/3).  Two threads per node: each takes half of the
// node's blocks and all three rows (three independent accumulators, 9 FMAs per block),
// the odd thread's partial sums reach its even neighbour by register shuffle, and the
// even thread writes q and adds its nodes' (w, q) and (r, w) terms to wq / rw (doubles).
// Every thread gets ~half a node, so the FP64 pipe is not idled by uneven rows per thread.
// Blocks are read in pairs starting at an even block index, 18 values as nine two-value
// loads (16-byte loads for FP64 values: 16-byte aligned values and 8-byte aligned col_idx
// required).  The matrix goes through the non-coherent path; w (written by other CTAs of a
// persistent kernel) does not.  qw (optional): a second copy of q, of type TQW.
template <typename T, typename TW = T, typename TQ = T, typename TR = T, typename TQW = TW>
__device__ __forceinline__ void cta_spmv(const int* __restrict__ rp, const int* __restrict__ ci,
                                         const T* __restrict__ vals, const TW* __restrict__ w,
                                         TQ* __restrict__ q, const TR* __restrict__ r, int64_t r0, int64_t r1,
                                         double& wq, double& rw, TQW* __restrict__ qw = nullptr) {
  using V2 = typename VT<T>::V2;
  const int64_t n0 = r0 / 3;
  const int64_t items = 2 * ((r1 - r0) / 3);
  for (int64_t base = 0; base < items; base += TPB) {
    const int64_t it = base + threadIdx.x;
    T a0 = 0, a1 = 0, a2 = 0;
    const bool active = it < items;
    int64_t node = 0;
    if (active) {
      node = n0 + (it >> 1);
      const int ka = __ldg(rp + node), kb = __ldg(rp + node + 1);
      const int mid = ka + ((kb - ka) >> 1);
      const int kbeg = (it & 1) ? mid : ka, kend = (it & 1) ? kb : mid;
      int k = kbeg;
      if ((k & 1) && k < kend) {  // a leading odd block alone (not aligned for pair loads)
        const int64_t cc = 3 * (int64_t)__ldg(ci + k);
        const T* v = vals + 9 * (int64_t)k;
        const T w0 = (T)w[cc], w1 = (T)w[cc + 1], w2 = (T)w[cc + 2];
        a0 += __ldg(v + 0) * w0; a1 += __ldg(v + 3) * w0; a2 += __ldg(v + 6) * w0;
        a0 += __ldg(v + 1) * w1; a1 += __ldg(v + 4) * w1; a2 += __ldg(v + 7) * w1;
        a0 += __ldg(v + 2) * w2; a1 += __ldg(v + 5) * w2; a2 += __ldg(v + 8) * w2;
        k++;
      }
      // block pairs (k even): nine two-value loads; the next pair's indices and values are
      // loaded before the current pair is used (two-stage software pipeline)
      if (k + 2 <= kend) {
        int2 cp = __ldg(reinterpret_cast<const int2*>(ci + k));
        const V2* v2 = reinterpret_cast<const V2*>(vals + 9 * (int64_t)k);
        V2 p0 = __ldg(v2 + 0), p1 = __ldg(v2 + 1), p2 = __ldg(v2 + 2), p3 = __ldg(v2 + 3);
        V2 p4 = __ldg(v2 + 4), p5 = __ldg(v2 + 5), p6 = __ldg(v2 + 6), p7 = __ldg(v2 + 7);
        V2 p8 = __ldg(v2 + 8);
#pragma unroll 1
        for (; k + 2 <= kend; k += 2) {
          const int64_t c0 = 3 * (int64_t)cp.x, c1 = 3 * (int64_t)cp.y;
          const T x0 = (T)w[c0], x1 = (T)w[c0 + 1], x2 = (T)w[c0 + 2];
          const T y0 = (T)w[c1], y1 = (T)w[c1 + 1], y2 = (T)w[c1 + 2];
          const V2 q0 = p0, q1 = p1, q2 = p2, q3 = p3, q4 = p4, q5 = p5, q6 = p6, q7 = p7, q8 = p8;
          if (k + 4 <= kend) {
            cp = __ldg(reinterpret_cast<const int2*>(ci + k + 2));
            const V2* n2 = reinterpret_cast<const V2*>(vals + 9 * (int64_t)(k + 2));
            p0 = __ldg(n2 + 0); p1 = __ldg(n2 + 1); p2 = __ldg(n2 + 2); p3 = __ldg(n2 + 3);
            p4 = __ldg(n2 + 4); p5 = __ldg(n2 + 5); p6 = __ldg(n2 + 6); p7 = __ldg(n2 + 7);
            p8 = __ldg(n2 + 8);
          }
          // block k: (q0.x q0.y q1.x / q1.y q2.x q2.y / q3.x q3.y q4.x); block k+1: q4.y ... q8.y
          a0 += q0.x * x0; a1 += q1.y * x0; a2 += q3.x * x0;
          a0 += q0.y * x1; a1 += q2.x * x1; a2 += q3.y * x1;
          a0 += q1.x * x2; a1 += q2.y * x2; a2 += q4.x * x2;
          a0 += q4.y * y0; a1 += q6.x * y0; a2 += q7.y * y0;
          a0 += q5.x * y1; a1 += q6.y * y1; a2 += q8.x * y1;
          a0 += q5.y * y2; a1 += q7.x * y2; a2 += q8.y * y2;
        }
      }
      if (k < kend) {  // a trailing single block
        const int64_t cc = 3 * (int64_t)__ldg(ci + k);
        const T* v = vals + 9 * (int64_t)k;
        const T w0 = (T)w[cc], w1 = (T)w[cc + 1], w2 = (T)w[cc + 2];
        a0 += __ldg(v + 0) * w0; a1 += __ldg(v + 3) * w0; a2 += __ldg(v + 6) * w0;
        a0 += __ldg(v + 1) * w1; a1 += __ldg(v + 4) * w1; a2 += __ldg(v + 7) * w1;
        a0 += __ldg(v + 2) * w2; a1 += __ldg(v + 5) * w2; a2 += __ldg(v + 8) * w2;
      }
    }
    // pairs (2i, 2i+1) share a warp (TPB and base are even); every lane takes part
    const T b0 = __shfl_xor_sync(0xffffffffu, a0, 1);
    const T b1 = __shfl_xor_sync(0xffffffffu, a1, 1);
    const T b2 = __shfl_xor_sync(0xffffffffu, a2, 1);
    if (active && !(it & 1)) {
      const T q0 = a0 + b0, q1 = a1 + b1, q2 = a2 + b2;
      const int64_t row = 3 * node;
      q[row] = (TQ)q0;
      q[row + 1] = (TQ)q1;
      q[row + 2] = (TQ)q2;
      if (qw) {
        qw[row] = (TQW)q0;
        qw[row + 1] = (TQW)q1;
        qw[row + 2] = (TQW)q2;
      }
      const T w0 = (T)w[row], w1 = (T)w[row + 1], w2 = (T)w[row + 2];
      wq += (double)w0 * (double)q0;
      wq += (double)w1 * (double)q1;
      wq += (double)w2 * (double)q2;
      if (r) {
        rw += (double)r[row] * (double)w0;
        rw += (double)r[row + 1] * (double)w1;
        rw += (double)r[row + 2] * (double)w2;
      }
    }
  }
}

// q = A w on one CTA's nodes with double-float matrix values and w: the layout of cta_spmv
// (two threads per node, block pairs as nine 16-byte loads, two-stage software pipeline)
// with each row accumulated in double-float on the FP32 pipes.  q is written as a double
// (qd) and as double-float (qw); (w, q) and (r, w) are formed in FP64 from wv, the FP64
// copy of w.
__device__ __forceinline__ dfl dfl_of(float hi, float lo) {
  dfl v;
  v.hi = hi;
  v.lo = lo;
  return v;
}
__device__ __forceinline__ void spmv_df_block(const dfl* __restrict__ v, dfl w0, dfl w1, dfl w2, dacc& a0, dacc& a1,
                                              dacc& a2) {
  const float2* f = reinterpret_cast<const float2*>(v);
  dfl m[9];
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const float2 t = __ldg(f + e);
    m[e] = dfl_of(t.x, t.y);
  }
  using AC = Acc<dfl>;
  AC::mac(a0, m[0], w0); AC::mac(a1, m[3], w0); AC::mac(a2, m[6], w0);
  AC::mac(a0, m[1], w1); AC::mac(a1, m[4], w1); AC::mac(a2, m[7], w1);
  AC::mac(a0, m[2], w2); AC::mac(a1, m[5], w2); AC::mac(a2, m[8], w2);
}
__device__ __forceinline__ void cta_spmv_df(const int* __restrict__ rp, const int* __restrict__ ci,
                                            const dfl* __restrict__ vals, const dfl* __restrict__ w,
                                            const double* __restrict__ wv, double* __restrict__ qd,
                                            dfl* __restrict__ qw, const double* __restrict__ r, int64_t r0,
                                            int64_t r1, double& wq, double& rw) {
  using AC = Acc<dfl>;
  const int64_t n0 = r0 / 3;
  const int64_t items = 2 * ((r1 - r0) / 3);
  for (int64_t base = 0; base < items; base += TPB) {
    const int64_t it = base + threadIdx.x;
    dacc a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f};
    const bool active = it < items;
    int64_t node = 0;
    if (active) {
      node = n0 + (it >> 1);
      const int ka = __ldg(rp + node), kb = __ldg(rp + node + 1);
      const int mid = ka + ((kb - ka) >> 1);
      const int kbeg = (it & 1) ? mid : ka, kend = (it & 1) ? kb : mid;
      int k = kbeg;
      if ((k & 1) && k < kend) {  // a leading odd block alone (not aligned for pair loads)
        const int64_t cc = 3 * (int64_t)__ldg(ci + k);
        spmv_df_block(vals + 9 * (int64_t)k, w[cc], w[cc + 1], w[cc + 2], a0, a1, a2);
        k++;
      }
      if (k + 2 <= kend) {
        int2 cp = __ldg(reinterpret_cast<const int2*>(ci + k));
        const float4* v4 = reinterpret_cast<const float4*>(vals + 9 * (int64_t)k);
        float4 p[9];
#pragma unroll
        for (int e = 0; e < 9; e++) p[e] = __ldg(v4 + e);
#pragma unroll 1
        for (; k + 2 <= kend; k += 2) {
          const int64_t c0 = 3 * (int64_t)cp.x, c1 = 3 * (int64_t)cp.y;
          const dfl x0 = w[c0], x1 = w[c0 + 1], x2 = w[c0 + 2];
          const dfl y0 = w[c1], y1 = w[c1 + 1], y2 = w[c1 + 2];
          float4 q[9];
#pragma unroll
          for (int e = 0; e < 9; e++) q[e] = p[e];
          if (k + 4 <= kend) {
            cp = __ldg(reinterpret_cast<const int2*>(ci + k + 2));
            const float4* n4 = reinterpret_cast<const float4*>(vals + 9 * (int64_t)(k + 2));
#pragma unroll
            for (int e = 0; e < 9; e++) p[e] = __ldg(n4 + e);
          }
          // value e of the pair (0..17) is half (e & 1) of q[e >> 1]; block k: values 0..8,
          // block k + 1: values 9..17, each row-major
#define KRS_DFV(e) ((((e) & 1) == 0) ? dfl_of(q[(e) >> 1].x, q[(e) >> 1].y) : dfl_of(q[(e) >> 1].z, q[(e) >> 1].w))
          AC::mac(a0, KRS_DFV(0), x0); AC::mac(a1, KRS_DFV(3), x0); AC::mac(a2, KRS_DFV(6), x0);
          AC::mac(a0, KRS_DFV(1), x1); AC::mac(a1, KRS_DFV(4), x1); AC::mac(a2, KRS_DFV(7), x1);
          AC::mac(a0, KRS_DFV(2), x2); AC::mac(a1, KRS_DFV(5), x2); AC::mac(a2, KRS_DFV(8), x2);
          AC::mac(a0, KRS_DFV(9), y0); AC::mac(a1, KRS_DFV(12), y0); AC::mac(a2, KRS_DFV(15), y0);
          AC::mac(a0, KRS_DFV(10), y1); AC::mac(a1, KRS_DFV(13), y1); AC::mac(a2, KRS_DFV(16), y1);
          AC::mac(a0, KRS_DFV(11), y2); AC::mac(a1, KRS_DFV(14), y2); AC::mac(a2, KRS_DFV(17), y2);
#undef KRS_DFV
        }
      }
      if (k < kend) {  // a trailing single block
        const int64_t cc = 3 * (int64_t)__ldg(ci + k);
        spmv_df_block(vals + 9 * (int64_t)k, w[cc], w[cc + 1], w[cc + 2], a0, a1, a2);
      }
    }
    // pairs (2i, 2i+1) share a warp (TPB and base are even); every lane takes part
    const dacc b0 = dacc_shfl(a0, 1), b1 = dacc_shfl(a1, 1), b2 = dacc_shfl(a2, 1);
    if (active && !(it & 1)) {
      const double q0 = AC::out(dacc_sum(a0, b0)), q1 = AC::out(dacc_sum(a1, b1)), q2 = AC::out(dacc_sum(a2, b2));
      const int64_t row = 3 * node;
      qd[row] = q0;
      qd[row + 1] = q1;
      qd[row + 2] = q2;
      qw[row] = dfl(q0);
      qw[row + 1] = dfl(q1);
      qw[row + 2] = dfl(q2);
      const double w0 = wv[row], w1 = wv[row + 1], w2 = wv[row + 2];
      wq += w0 * q0;
      wq += w1 * q1;
      wq += w2 * q2;
      rw += r[row] * w0;
      rw += r[row + 1] * w1;
      rw += r[row + 2] * w2;
    }
  }
}

// u = M^-1 r for one row (Jacobi: minv[row]; block Jacobi: minv[9*node + 3*d + e];
// identity: r).
template <typename T, typename TV = T>
__device__ __forceinline__ TV precond_row(int kind, const T* __restrict__ minv, const TV* __restrict__ r,
                                          int64_t row) {
  if (kind == 0) return (TV)(minv[row] * (T)r[row]);
  if (kind == 1) {
    const int64_t node = row / 3;
    const int d = (int)(row - 3 * node);
    const T* m = minv + 9 * node + 3 * d;
    return (TV)(m[0] * (T)r[3 * node] + m[1] * (T)r[3 * node + 1] + m[2] * (T)r[3 * node + 2]);
  }
  return r[row];
}

}  // namespace krs
