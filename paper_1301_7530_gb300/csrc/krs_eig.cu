// krs_eig.cu -- the between-solve SRKS step on the GPU (Section 4, Algorithm 3):
//   * H_m = tridiag(eta_{j-1}, delta_j, eta_j) from the CG coefficients (Section 4.1):
//     beta~_j = rho_{j+1}/rho_j, delta_0 = 1/alpha_0,
//     delta_j = 1/alpha_j + beta~_{j-1}/alpha_{j-1}, eta_j = sqrt(beta~_j)/alpha_j;
//   * its eigenvalues and those of H_{m-1} by multisection on Sturm counts (a group of
//     L lanes per eigenvalue tests L points per round, so an interval shrinks (L+1)x);
//   * the stagnation selection of Eq. 16 (union of both tests), the optional
//     theta < theta_frac * theta_max filter, ascending-theta order, the cap;
//   * eigenvectors of the selected values by inverse iteration (a lane per vector,
//     partial-pivoting LU of T - theta I), orthogonalised inside clusters;
//   * Ritz vectors y = V q / sqrt(theta), V = [(-1)^j z_j / sqrt(rho_j)] (Eq. 17).
// The eigenvalue arithmetic is FP64 throughout.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>

#include "krs_device.cuh"
#include "krs_internal.h"

namespace krs {

__global__ void k_lanczos(int m, const double* alpha, const double* rho, double* delta, double* eta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double d = 1.0 / alpha[j];
  if (j > 0) d += (rho[j] / rho[j - 1]) / alpha[j - 1];
  delta[j] = d;
  if (j < m - 1) eta[j] = sqrt(rho[j + 1] / rho[j]) / alpha[j];
}

cudaError_t launch_lanczos(int m, const double* alpha, const double* rho, double* delta, double* eta,
                           cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_lanczos<<<(m + 127) / 128, 128, 0, st>>>(m, alpha, rho, delta, eta);
  return cudaGetLastError();
}

// Number of eigenvalues of T (order m, diagonal d, squared off-diagonal e2) below x: the
// number of negative pivots q_i of T - x I = L D L^T.  The pivots are taken as ratios of
// consecutive leading principal minors, p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2} (p_{-1} = 1),
// which needs no division: after every step the pair (p_{i-1}, p_i) is rescaled by the power
// of two that brings |p_i| into [1, 2) (exact), so the minors stay in range.  A pivot at or
// below pivmin counts as negative, and one within pivmin of zero is replaced by -pivmin.
// With pivmin >= 2^-900 max(1, max e2) the rescaled p_{i-1} stays below 2^901 / max(1, e2), so
// no product overflows.  (A division per step made each count a chain of slow FP64
// divisions on GB300; this chain is one fused multiply-add, one multiply and integer work.)
__device__ __forceinline__ int sturm_count(int m, const double* d, const double* e2, double x,
                                           double pivmin) {
  int cnt = 0;
  double a = 1.0;       // p_{i-1}, rescaled
  double b = d[0] - x;  // p_i, rescaled (p_{-1} = 1, so q_0 = p_0)
  if (b <= pivmin) {
    cnt++;
    b = fmin(b, -pivmin);
  }
  for (int i = 1; i <= m; i++) {
    // rescale the pair so that |b| is in [1, 2): s = 2^(1023 - biased exponent of b)
    const long long bits = __double_as_longlong(b);
    const int ex = (int)((bits >> 52) & 0x7ff);
    const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
    a *= sc;
    b *= sc;
    if (i == m) break;
    double p = (d[i] - x) * b - e2[i - 1] * a;
    // q_i = p / b <= pivmin  <=>  p sgn(b) <= pivmin |b|
    const double ab = fabs(b);
    const double ps = (b > 0.0) ? p : -p;
    const double lim = pivmin * ab;
    if (ps <= lim) {
      cnt++;
      if (ps > -lim) p = -pivmin * b;  // q_i := -pivmin
    }
    a = b;
    b = p;
  }
  return cnt;
}

// Multisection over lane groups.  Each eigenvalue (a "job") gets a group of L lanes of a
// warp (L a power of two); every round the L lanes evaluate Sturm counts at L interior
// points of the job's interval, which shrinks (L + 1)-fold.  GB300's FP64 units cost the
// same per warp instruction whatever the number of active lanes, so the cost of a job is
// rounds x m and a warp holds 32 / L jobs: the launcher picks L so that the warps about
// fill one warp per SM sub-partition (four-warp CTAs).
// Job index q in [0, m + m1): q < m is eigenvalue q (descending) of T_m, else eigenvalue
// q - m of T_{m1} (leading block).  Output: theta_m[m], theta_m1[m1], descending.
constexpr int BISECT_WARPS = 4;  // one warp per SM sub-partition

// SM: the tridiagonal is staged in shared memory (2m + 1 doubles); otherwise (an order too
// large for shared memory) it is read from global memory, `eta` then holding the squared
// off-diagonal (k_square below).
template <bool SM>
__global__ void __launch_bounds__(32 * BISECT_WARPS) k_bisect(int m, int m1, int L, const double* __restrict__ delta,
                                                              const double* __restrict__ eta, double* theta_m,
                                                              double* theta_m1) {
  extern __shared__ double sh[];
  const double* d;
  const double* e2;
  if constexpr (SM) {
    double* ds = sh;
    double* es = sh + m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      ds[i] = delta[i];
      if (i < m - 1) es[i] = eta[i] * eta[i];
    }
    __syncthreads();
    d = ds;
    e2 = es;
  } else {
    d = delta;
    e2 = eta;
  }
  const int lane = threadIdx.x & 31;
  const int per_warp = 32 / L;
  const int grp = lane / L, sub = lane % L;
  const int job = (blockIdx.x * BISECT_WARPS + (int)(threadIdx.x >> 5)) * per_warp + grp;
  const bool active = job < m + m1;
  const int order = !active ? m : (job < m ? m : m1);
  const int idx_desc = !active ? 0 : (job < m ? job : job - m);
  const int k = order - 1 - idx_desc;  // ascending index
  // Gershgorin interval of the order-`order` leading block
  double lo = d[0], hi = d[0], emax = 0.0;
  for (int i = 0; i < order; i++) {
    const double el = (i > 0) ? sqrt(e2[i - 1]) : 0.0;
    const double er = (i < order - 1) ? sqrt(e2[i]) : 0.0;
    lo = fmin(lo, d[i] - el - er);
    hi = fmax(hi, d[i] + el + er);
    if (i < order - 1) emax = fmax(emax, e2[i]);
  }
  const double tnorm = fmax(fabs(lo), fabs(hi));
  const double pivmin = 0x1p-900 * fmax(1.0, emax);
  lo -= 2.0 * DBL_EPSILON * tnorm + pivmin;
  hi += 2.0 * DBL_EPSILON * tnorm + pivmin;
  const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (grp * L));
  bool done = !active;
  // invariant: count(lo) <= k < count(hi)
  for (int round = 0; round < 400; round++) {
    if (!done) {
      const double width = hi - lo;
      if (width <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) done = true;
    }
    if (!__any_sync(0xffffffffu, !done)) break;
    const double x = lo + (hi - lo) * ((double)(sub + 1) / (double)(L + 1));
    const int c = done ? 0 : sturm_count(order, d, e2, x, pivmin);
    const unsigned above = __ballot_sync(0xffffffffu, !done && c > k) & gmask;
    const int first = above ? (__ffs(above) - 1) - grp * L : L;  // first point above, in the group
    const double xF = __shfl_sync(0xffffffffu, x, grp * L + (first < L ? first : 0));
    const double xFm = __shfl_sync(0xffffffffu, x, grp * L + (first > 0 ? first - 1 : 0));
    if (!done) {
      const double nhi = (first < L) ? xF : hi;
      const double nlo = (first > 0) ? xFm : lo;
      if (nhi == hi && nlo == lo) done = true;  // no representable progress
      lo = nlo;
      hi = nhi;
    }
  }
  if (active && sub == 0) {
    const double v = 0.5 * (lo + hi);
    if (job < m) theta_m[idx_desc] = v;
    else theta_m1[idx_desc] = v;
  }
}

__global__ void k_square(const double* __restrict__ v, double* __restrict__ out, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = v[i] * v[i];
}

cudaError_t launch_tridiag_eigvals2(int m, int m1, const double* delta, const double* eta, double* theta_m,
                                    double* theta_m1, cudaStream_t st, double* e2_scratch) {
  if (m <= 0) return cudaSuccess;
  const int jobs = m + m1;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // lanes per job: the largest power of two whose warps (32 / L jobs each) still fit one
  // warp per SM sub-partition (an FP64 warp instruction occupies its sub-partition's FP64
  // unit; a lone warp per SM leaves three of them idle)
  int L = 32;
  while (L > 1 && (int64_t)jobs * L > 32 * (int64_t)BISECT_WARPS * sms) L >>= 1;
  const int per_warp = 32 / L;
  const int per_cta = per_warp * BISECT_WARPS;
  const size_t sm = sizeof(double) * (size_t)(2 * m + 1);
  int sm_max = 0;
  cudaDeviceGetAttribute(&sm_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const unsigned grid = (unsigned)((jobs + per_cta - 1) / per_cta);
  if (sm <= (size_t)sm_max) {
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute((const void*)k_bisect<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_bisect<true><<<grid, 32 * BISECT_WARPS, sm, st>>>(m, m1, L, delta, eta, theta_m, theta_m1);
  } else {
    // too long for shared memory: the squared off-diagonal in the caller's scratch (m doubles)
    if (!e2_scratch) return cudaErrorInvalidValue;
    k_square<<<(m + 255) / 256, 256, 0, st>>>(eta, e2_scratch, m - 1);
    k_bisect<false><<<grid, 32 * BISECT_WARPS, 0, st>>>(m, m1, L, delta, e2_scratch, theta_m, theta_m1);
  }
  return cudaGetLastError();
}

cudaError_t launch_tridiag_eigvals(int m, const double* delta, const double* eta, double* theta,
                                   cudaStream_t st) {
  return launch_tridiag_eigvals2(m, 0, delta, eta, theta, nullptr, st, nullptr);
}

// ------------------------------------------------------------------------------------
// selection (one thread; O(m))
// ------------------------------------------------------------------------------------
// Cluster reselection on the s preselected values (ascending) v[0..s): the three-piece
// least-squares fit of the gaps d_i = v_{i+1} - v_i (pieces [0, a), [a, b], (b, s-2]),
// central piece = values v_a .. v_{b+1}, at least max(2, ceil(s/5)) of them; the values of
// the central piece are dropped when it is strictly denser (smaller mean gap) than every
// non-empty outer piece and an outer piece exists.  Piece sums come from prefix sums of d
// and d^2; the warp's lanes split the a range, ties go to the smallest (a, b).
// keep[k] = 0 for a dropped value.  P1, P2: s doubles each (scratch).
__device__ void cluster_reselect_warp(int s, const double* v, double* P1, double* P2, unsigned char* keep) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < s; k += 32) keep[k] = 1;
  __syncwarp();
  if (s < 3) return;
  const int ng = s - 1;
  int minsize = (s + 4) / 5;
  if (minsize < 2) minsize = 2;
  if (lane == 0) {
    double a1 = 0.0, a2 = 0.0;
    P1[0] = 0.0;
    P2[0] = 0.0;
    for (int i = 0; i < ng; i++) {
      const double d = v[i + 1] - v[i];
      a1 += d;
      a2 += d * d;
      P1[i + 1] = a1;
      P2[i + 1] = a2;
    }
  }
  __syncwarp();
  auto sse = [&](int lo, int hi, double* mean) -> double {  // gaps [lo, hi], empty if hi < lo
    if (hi < lo) {
      *mean = 0.0;
      return 0.0;
    }
    const double len = (double)(hi - lo + 1);
    const double s1 = P1[hi + 1] - P1[lo], s2 = P2[hi + 1] - P2[lo];
    *mean = s1 / len;
    const double e = s2 - s1 * s1 / len;
    return e > 0.0 ? e : 0.0;
  };
  double best = -1.0;
  int ba = ng, bb = ng;
  for (int a = lane; a < ng; a += 32) {
    for (int b = a; b < ng; b++) {
      if (b - a + 2 < minsize) continue;
      double m0, m1, m2;
      const double e = sse(0, a - 1, &m0) + sse(a, b, &m1) + sse(b + 1, ng - 1, &m2);
      if (best < 0.0 || e < best) {  // within a lane, (a, b) increase: the first minimum stays
        best = e;
        ba = a;
        bb = b;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double e2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int a2 = __shfl_xor_sync(0xffffffffu, ba, o), b2 = __shfl_xor_sync(0xffffffffu, bb, o);
    const bool take = (e2 >= 0.0) && (best < 0.0 || e2 < best || (e2 == best && (a2 < ba || (a2 == ba && b2 < bb))));
    if (take) {
      best = e2;
      ba = a2;
      bb = b2;
    }
  }
  if (lane == 0 && best >= 0.0) {
    double m0, m1, m2;
    sse(0, ba - 1, &m0);
    sse(ba, bb, &m1);
    sse(bb + 1, ng - 1, &m2);
    const bool left = ba > 0, right = bb < ng - 1;
    const bool denser = (left || right) && (!left || m1 < m0) && (!right || m1 < m2);
    if (denser)
      for (int i = ba; i <= bb + 1; i++) keep[i] = 0;
  }
  __syncwarp();
}

// Selection (one warp).  scratch: 4m doubles after the m selected values in tsel:
// [m, 2m) flags (bytes), [2m, 3m) ascending preselected values, [3m, 5m) prefix sums.
__global__ void k_srks_select(int m, const double* tm, const double* tm1, double eps, double theta_frac,
                              int reselect, int room, int* sel, int* count, double* tsel) {
  if (blockIdx.x != 0) return;
  unsigned char* flag = reinterpret_cast<unsigned char*>(tsel + m);
  double* v = tsel + 2 * (size_t)m;
  double* P1 = tsel + 3 * (size_t)m;
  double* P2 = tsel + 4 * (size_t)m;
  unsigned char* keep = reinterpret_cast<unsigned char*>(sel);  // sel is rewritten below
  const int lane = threadIdx.x & 31;
  const bool run = m >= 2 && room > 0 && eps > 0.0;
  __shared__ int s_cnt;
  if (lane == 0) {
    s_cnt = 0;
    if (run) {
      for (int i = 0; i < m; i++) flag[i] = 0;
      for (int j = 1; j <= m - 1; j++) {  // paper's 1-based j
        const double a = tm[j - 1], b = tm1[j - 1], c = tm[j];
        if (fabs(a - b) <= eps * fabs(a)) flag[j - 1] = 1;
        if (fabs(c - b) <= eps * fabs(c)) flag[j] = 1;
      }
      if (theta_frac > 0.0) {
        const double lim = theta_frac * tm[0];
        for (int i = 0; i < m; i++)
          if (flag[i] && !(tm[i] < lim)) flag[i] = 0;
      }
      if (reselect == 1) {
        int c = 0;
        for (int i = m - 1; i >= 0; i--)
          if (flag[i]) v[c++] = tm[i];
        s_cnt = c;
      }
    }
  }
  __syncwarp();
  if (run && reselect == 1) {
    const int s = s_cnt;
    cluster_reselect_warp(s, v, P1, P2, keep);
    if (lane == 0) {
      int c = 0;
      for (int i = m - 1; i >= 0; i--)
        if (flag[i]) {
          if (!keep[c]) flag[i] = 0;
          c++;
        }
    }
    __syncwarp();
  }
  if (lane == 0) {
    int cnt = 0;
    if (run) {
      for (int i = m - 1; i >= 0 && cnt < room; i--) {
        if (flag[i]) {
          sel[cnt] = i;
          tsel[cnt] = tm[i];
          cnt++;
        }
      }
    }
    *count = cnt;
  }
}

cudaError_t launch_srks_select(int m, const double* theta_m, const double* theta_m1, double eps,
                               double theta_frac, int reselect, int room, int* sel, int* count, double* tsel,
                               cudaStream_t st) {
  k_srks_select<<<1, 32, 0, st>>>(m, theta_m, theta_m1, eps, theta_frac, reselect, room, sel, count, tsel);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// eigenvectors by inverse iteration
// ------------------------------------------------------------------------------------
constexpr int INV_ITERS = 3;
constexpr int VEC_TPB = 256;

size_t eigvecs_work_doubles(int m, int k) { return (size_t)5 * m * k + 64; }

// Sum over the VEC_TPB threads of a block (warp butterflies, then warp 0); all threads get it.
__device__ __forceinline__ double vec_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < VEC_TPB / 32; w++) t += red[w];
  __syncthreads();
  return t;
}

// One CTA; thread c < k owns eigenvector c.  Work layout: [array][i][c] (arrays: d, du1,
// du2, l, piv) so that lanes touch consecutive addresses.
__global__ void __launch_bounds__(VEC_TPB) k_tridiag_eigvecs(int m, const double* __restrict__ delta,
                                                             const double* __restrict__ eta, int k,
                                                             const double* __restrict__ theta,
                                                             double* __restrict__ Q, double* __restrict__ work) {
  __shared__ double red[VEC_TPB / 32];
  // ||T||_1 bound for tiny-pivot replacement and cluster detection
  double tn = 0.0;
  for (int i = 0; i < m; i++) {
    const double a = fabs(delta[i]) + (i > 0 ? fabs(eta[i - 1]) : 0.0) + (i < m - 1 ? fabs(eta[i]) : 0.0);
    tn = fmax(tn, a);
  }
  const double tiny = DBL_EPSILON * tn;
  const double ortol = 1e-6 * tn;
  double* D = work;
  double* U1 = work + (size_t)m * k;
  double* U2 = work + 2 * (size_t)m * k;
  double* Lm = work + 3 * (size_t)m * k;
  double* PV = work + 4 * (size_t)m * k;
  for (int c0 = 0; c0 < k; c0 += VEC_TPB) {
    const int c = c0 + threadIdx.x;
    if (c < k) {
      const double th = theta[c];
      // LU with partial pivoting of T - th I
      double cd = delta[0] - th;
      double cu1 = (m > 1) ? eta[0] : 0.0;
      for (int i = 0; i < m - 1; i++) {
        const double sub = eta[i];
        const double nd = delta[i + 1] - th;
        const double nu = (i + 1 < m - 1) ? eta[i + 1] : 0.0;
        const size_t at = (size_t)i * k + c;
        if (fabs(cd) >= fabs(sub)) {
          if (cd == 0.0) cd = tiny;
          const double mult = sub / cd;
          D[at] = cd; U1[at] = cu1; U2[at] = 0.0; Lm[at] = mult; PV[at] = 0.0;
          cd = nd - mult * cu1;
          cu1 = nu;
        } else {
          const double mult = cd / sub;
          D[at] = sub; U1[at] = nd; U2[at] = nu; Lm[at] = mult; PV[at] = 1.0;
          cd = cu1 - mult * nd;
          cu1 = -mult * nu;
        }
      }
      if (cd == 0.0) cd = tiny;
      D[(size_t)(m - 1) * k + c] = cd;
      // start vector: deterministic, distinct per vector
      for (int i = 0; i < m; i++) {
        const unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)((c + 1) * 40503u);
        Q[(size_t)c * m + i] = 1.0 + 0.25 * (double)((h >> 8) & 1023) / 1024.0;
      }
    }
  }
  __syncthreads();
  for (int it = 0; it < INV_ITERS; it++) {
    for (int c0 = 0; c0 < k; c0 += VEC_TPB) {
      const int c = c0 + threadIdx.x;
      if (c < k) {
        double* v = Q + (size_t)c * m;
        // forward: apply the row operations
        for (int i = 0; i < m - 1; i++) {
          const size_t at = (size_t)i * k + c;
          if (PV[at] != 0.0) {
            const double t = v[i];
            v[i] = v[i + 1];
            v[i + 1] = t - Lm[at] * v[i];
          } else {
            v[i + 1] -= Lm[at] * v[i];
          }
        }
        // backward substitution with U (three diagonals), tracking the largest entry
        double x2 = 0.0, x1 = 0.0, mx = 0.0;
        for (int i = m - 1; i >= 0; i--) {
          const size_t at = (size_t)i * k + c;
          const double xi = (v[i] - U1[at] * x1 - U2[at] * x2) / D[at];
          v[i] = xi;
          mx = fmax(mx, fabs(xi));
          x2 = x1;
          x1 = xi;
        }
        // scale by the largest entry (no overflow), then to unit 2-norm
        const double s = (mx > 0.0) ? 1.0 / mx : 1.0;
        double nrm = 0.0;
        for (int i = 0; i < m; i++) {
          const double t = v[i] * s;
          v[i] = t;
          nrm += t * t;
        }
        const double inv = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 1.0;
        for (int i = 0; i < m; i++) v[i] *= inv;
      }
    }
    __syncthreads();
    // orthogonalise inside clusters (theta ascending on input; a cluster is a chain of
    // consecutive values closer than ortol), modified Gram-Schmidt, then renormalise
    for (int c = 1; c < k; c++) {
      if (!(fabs(theta[c] - theta[c - 1]) <= ortol)) continue;
      double* v = Q + (size_t)c * m;
      int p0 = c - 1;  // first member of c's cluster
      while (p0 > 0 && fabs(theta[p0] - theta[p0 - 1]) <= ortol) p0--;
      for (int p = c - 1; p >= p0; p--) {
        const double* w = Q + (size_t)p * m;
        double sdot = 0.0;
        for (int i = threadIdx.x; i < m; i += VEC_TPB) sdot += w[i] * v[i];
        const double dp = vec_block_sum(sdot, red);
        for (int i = threadIdx.x; i < m; i += VEC_TPB) v[i] -= dp * w[i];
        __syncthreads();
      }
      double sn = 0.0;
      for (int i = threadIdx.x; i < m; i += VEC_TPB) sn += v[i] * v[i];
      const double nn = vec_block_sum(sn, red);
      const double sc = (nn > 0.0) ? 1.0 / sqrt(nn) : 1.0;
      for (int i = threadIdx.x; i < m; i += VEC_TPB) v[i] *= sc;
      __syncthreads();
    }
  }
  // sign: largest-magnitude component positive (owner thread)
  for (int c0 = 0; c0 < k; c0 += VEC_TPB) {
    const int c = c0 + threadIdx.x;
    if (c < k) {
      double* v = Q + (size_t)c * m;
      double best = 0.0;
      int bi = 0;
      for (int i = 0; i < m; i++)
        if (fabs(v[i]) > best) { best = fabs(v[i]); bi = i; }
      if (v[bi] < 0.0)
        for (int i = 0; i < m; i++) v[i] = -v[i];
    }
  }
}

cudaError_t launch_tridiag_eigvecs(int m, const double* delta, const double* eta, int k,
                                   const double* theta_sel, double* Q, double* work, cudaStream_t st) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  k_tridiag_eigvecs<<<1, VEC_TPB, 0, st>>>(m, delta, eta, k, theta_sel, Q, work);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Ritz vectors: F[j][c] = (-1)^j Q[j, c] / sqrt(rho_j) / sqrt|theta_c|, Y = Z F
// ------------------------------------------------------------------------------------
__global__ void k_ritz_coeffs(int m, int k, const double* Q, const double* rho, const double* tsel, double* F) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int j = e % m, c = e / m;
  const double sgn = (j & 1) ? -1.0 : 1.0;
  F[(size_t)j * k + c] = sgn * Q[(size_t)c * m + j] / sqrt(rho[j]) / sqrt(fabs(tsel[c]));
}

constexpr int RITZ_COLS = 8;
constexpr int RITZ_JCHUNK = 256;

template <typename TZ>
__global__ void __launch_bounds__(256) k_ritz_gemm(int64_t n, int64_t ld, int m, int k, const TZ* __restrict__ Z,
                                                   const double* __restrict__ F, double* __restrict__ Y) {
  __shared__ double sF[RITZ_JCHUNK][RITZ_COLS];
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int cb = blockIdx.y * RITZ_COLS;
  const int nk = min(RITZ_COLS, k - cb);
  double acc[RITZ_COLS];
#pragma unroll
  for (int q = 0; q < RITZ_COLS; q++) acc[q] = 0.0;
  for (int j0 = 0; j0 < m; j0 += RITZ_JCHUNK) {
    const int jl = min(RITZ_JCHUNK, m - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < jl * RITZ_COLS; e += blockDim.x) {
      const int jj = e / RITZ_COLS, q = e % RITZ_COLS;
      sF[jj][q] = (q < nk) ? F[(size_t)(j0 + jj) * k + cb + q] : 0.0;
    }
    __syncthreads();
    if (row < n) {
      for (int jj = 0; jj < jl; jj++) {
        const double z = (double)Z[(int64_t)(j0 + jj) * ld + row];
#pragma unroll
        for (int q = 0; q < RITZ_COLS; q++) acc[q] += z * sF[jj][q];
      }
    }
  }
  if (row < n) {
#pragma unroll
    for (int q = 0; q < RITZ_COLS; q++)
      if (q < nk) Y[(int64_t)(cb + q) * ld + row] = acc[q];
  }
}

template <typename TZ>
static cudaError_t ritz_vectors_t(int64_t n, int64_t ld, int m, int k, const TZ* Z, const double* rho, const double* Q,
                                  const double* tsel, double* F, double* Y, cudaStream_t st) {
  if (k <= 0 || m <= 0) return cudaSuccess;
  k_ritz_coeffs<<<(m * k + 255) / 256, 256, 0, st>>>(m, k, Q, rho, tsel, F);
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((k + RITZ_COLS - 1) / RITZ_COLS));
  k_ritz_gemm<TZ><<<grid, 256, 0, st>>>(n, ld, m, k, Z, F, Y);
  return cudaGetLastError();
}

// Ritz vectors from single-precision z_j (inner solve of the mixed-precision refinement);
// accumulated and stored in FP64.
cudaError_t launch_ritz_vectors_f(int64_t n, int64_t ld, int m, int k, const float* Z, const double* rho,
                                  const double* Q, const double* tsel, double* F, double* Y, cudaStream_t st) {
  return ritz_vectors_t<float>(n, ld, m, k, Z, rho, Q, tsel, F, Y, st);
}

// ------------------------------------------------------------------------------------
// The z_j of a solve that kept only its reorthogonalisation coefficients: w_j = z_j -
// sum_{i<j} g_i^(j) w_i, so z_j = w_j + sum_{i<j} U[i, j] w_i with U[i, j] = g_i^(j) (packed
// rows: row j at j (j - 1) / 2).  Then sum_j z_j F[j, c] = sum_i w_i F2[i, c] with
// F2[i, c] = F[i, c] + sum_{j>i} U[i, j] F[j, c]: the Ritz vectors are formed from W.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double u_entry(const double* __restrict__ U, int full, int i, int j) {
  // U[i, j] for i < j (full == 0: classical CG, only the previous direction is used)
  return (full || i == j - 1) ? U[(int64_t)j * (j - 1) / 2 + i] : 0.0;
}

__global__ void k_ritz_fold(int m, int k, const double* __restrict__ U, int full, const double* __restrict__ F,
                            double* __restrict__ F2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * k) return;
  const int i = (int)(e % m), c = (int)(e / m);
  double acc = F[(size_t)i * k + c];
  const int jend = full ? m : min(m, i + 2);
  for (int j = i + 1; j < jend; j++) acc += u_entry(U, full, i, j) * F[(size_t)j * k + c];
  F2[(size_t)i * k + c] = acc;
}

// Ud[i, c] (row-major, m x m) = coefficient of w_i in z_c: 1 on the diagonal, U above it
__global__ void k_dense_u(int m, const double* __restrict__ U, int full, double* __restrict__ Ud) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int i = (int)(e / m), c = (int)(e % m);
  Ud[e] = (i == c) ? 1.0 : (i < c ? u_entry(U, full, i, c) : 0.0);
}

cudaError_t launch_ritz_vectors_wu(int64_t n, int64_t ld, int m, int k, const void* W, bool w_df, const double* ucoef,
                                   int full, const double* rho, const double* Q, const double* tsel, double* F,
                                   double* F2, double* Y, cudaStream_t st) {
  if (k <= 0 || m <= 0) return cudaSuccess;
  k_ritz_coeffs<<<(m * k + 255) / 256, 256, 0, st>>>(m, k, Q, rho, tsel, F);
  k_ritz_fold<<<(unsigned)(((int64_t)m * k + 255) / 256), 256, 0, st>>>(m, k, ucoef, full, F, F2);
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((k + RITZ_COLS - 1) / RITZ_COLS));
  if (w_df)
    k_ritz_gemm<dfl><<<grid, 256, 0, st>>>(n, ld, m, k, static_cast<const dfl*>(W), F2, Y);
  else
    k_ritz_gemm<double><<<grid, 256, 0, st>>>(n, ld, m, k, static_cast<const double*>(W), F2, Y);
  return cudaGetLastError();
}

cudaError_t launch_z_from_wu(int64_t n, int64_t ld, int m, const void* W, bool w_df, const double* ucoef, int full,
                             double* Ud, double* Y, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_dense_u<<<(unsigned)(((int64_t)m * m + 255) / 256), 256, 0, st>>>(m, ucoef, full, Ud);
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((m + RITZ_COLS - 1) / RITZ_COLS));
  if (w_df)
    k_ritz_gemm<dfl><<<grid, 256, 0, st>>>(n, ld, m, m, static_cast<const dfl*>(W), Ud, Y);
  else
    k_ritz_gemm<double><<<grid, 256, 0, st>>>(n, ld, m, m, static_cast<const double*>(W), Ud, Y);
  return cudaGetLastError();
}


}  // namespace krs
