// krs_kernels.cu -- single kernels: the operator product, the preconditioner, the coarse
// set-up of the augmentation (A C, C^T A C, its Cholesky factor and inverse; Section 2.3
// items (i)-(iii)), the true residual, and stand-alone launches of the tall-skinny and
// vector kernels used by the iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "krs_device.cuh"
#include "krs_internal.h"

namespace krs {

// ------------------------------------------------------------------------------------
// y = A x, thread per scalar row (stand-alone product: set-up, true residual)
// ------------------------------------------------------------------------------------
__global__ void k_spmv(int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= 3 * (int64_t)nbr) return;
  const int64_t node = row / 3;
  const int d = (int)(row - 3 * node);
  const int ka = __ldg(rp + node), kb = __ldg(rp + node + 1);
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  for (int k = ka; k < kb; k++) {
    const int64_t cc = 3 * (int64_t)__ldg(ci + k);
    const double* a = vals + 9 * (int64_t)k + 3 * d;
    acc0 += __ldg(a + 0) * x[cc + 0];
    acc1 += __ldg(a + 1) * x[cc + 1];
    acc2 += __ldg(a + 2) * x[cc + 2];
  }
  y[row] = (acc0 + acc1) + acc2;
}

cudaError_t launch_spmv(int nbr, const int* rp, const int* ci, const double* vals, const double* x,
                        double* y, cudaStream_t st) {
  const int64_t n = 3 * (int64_t)nbr;
  if (n == 0) return cudaSuccess;
  k_spmv<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nbr, rp, ci, vals, x, y);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Preconditioner set-up: 1/A_ii (Jacobi) or the inverse of each diagonal 3x3 block
// (cofactors over the determinant).  A block is accepted when its (1,1) entry and its
// determinant are positive (for a Jacobi entry: when it is positive).
// ------------------------------------------------------------------------------------
__global__ void k_precond_setup(int kind, int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ vals, double* __restrict__ minv, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr || kind == 2) return;
  const double* D = nullptr;
  for (int k = rp[i]; k < rp[i + 1]; k++)
    if (ci[k] == i) D = vals + 9 * (int64_t)k;
  if (D == nullptr) {
    if (status) atomicCAS(status, 0, 1 /* KRS_ERR_INVALID_ARG */);
    return;
  }
  if (kind == 0) {
    for (int d = 0; d < 3; d++) {
      const double a = D[4 * d];
      if (!(a > 0.0) && status) atomicCAS(status, 0, 2);
      minv[3 * (int64_t)i + d] = 1.0 / a;
    }
    return;
  }
  const double a = D[0], b = D[1], c = D[2], d = D[3], e = D[4], f = D[5], g = D[6], h = D[7], k = D[8];
  const double c00 = e * k - f * h, c01 = f * g - d * k, c02 = d * h - e * g;
  const double det = a * c00 + b * c01 + c * c02;
  if ((!(det > 0.0) || !(a > 0.0)) && status) atomicCAS(status, 0, 2);
  const double id = 1.0 / det;
  double* o = minv + 9 * (int64_t)i;
  o[0] = c00 * id;
  o[1] = (c * h - b * k) * id;
  o[2] = (b * f - c * e) * id;
  o[3] = c01 * id;
  o[4] = (a * k - c * g) * id;
  o[5] = (c * d - a * f) * id;
  o[6] = c02 * id;
  o[7] = (b * g - a * h) * id;
  o[8] = (a * e - b * d) * id;
}

cudaError_t launch_precond_setup(int kind, int nbr, const int* rp, const int* ci, const double* vals,
                                 double* minv, int* status, cudaStream_t st) {
  if (nbr == 0) return cudaSuccess;
  k_precond_setup<<<(nbr + 127) / 128, 128, 0, st>>>(kind, nbr, rp, ci, vals, minv, status);
  return cudaGetLastError();
}

__global__ void k_precond_apply(int kind, int64_t n, const double* minv, const double* r, double* u) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < n) u[row] = precond_row(kind, minv, r, row);
}

cudaError_t launch_precond_apply(int kind, int nbr, const double* minv, const double* r, double* u,
                                 cudaStream_t st) {
  const int64_t n = 3 * (int64_t)nbr;
  if (n == 0) return cudaSuccess;
  k_precond_apply<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kind, n, minv, r, u);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// AC = A C for columns [c0, c1): thread per scalar row and 8 columns; A's block row is
// read once for the 8 columns.  Per column the summation order equals k_spmv's.  (Columns
// recycled from a solve's directions keep the iteration's own products A w instead.)
// ------------------------------------------------------------------------------------
constexpr int SPMM_COLS = 8;

__global__ void k_spmm(int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ vals, const double* __restrict__ C, double* __restrict__ AC,
                       int64_t ld, int c0, int c1) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= 3 * (int64_t)nbr) return;
  const int cb = c0 + blockIdx.y * SPMM_COLS;
  const int nk = min(SPMM_COLS, c1 - cb);
  const int64_t node = row / 3;
  const int d = (int)(row - 3 * node);
  double acc[SPMM_COLS][3];
#pragma unroll
  for (int q = 0; q < SPMM_COLS; q++) acc[q][0] = acc[q][1] = acc[q][2] = 0.0;
  const int ka = __ldg(rp + node), kb = __ldg(rp + node + 1);
  for (int k = ka; k < kb; k++) {
    const int64_t cc = 3 * (int64_t)__ldg(ci + k);
    const double* a = vals + 9 * (int64_t)k + 3 * d;
    const double a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2);
#pragma unroll
    for (int q = 0; q < SPMM_COLS; q++) {
      if (q < nk) {
        const double* x = C + (int64_t)(cb + q) * ld + cc;
        acc[q][0] += a0 * __ldg(x);
        acc[q][1] += a1 * __ldg(x + 1);
        acc[q][2] += a2 * __ldg(x + 2);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < SPMM_COLS; q++)
    if (q < nk) AC[(int64_t)(cb + q) * ld + row] = (acc[q][0] + acc[q][1]) + acc[q][2];
}

cudaError_t launch_spmm(int nbr, const int* rp, const int* ci, const double* vals, const double* C,
                        double* AC, int64_t ld, int c0, int c1, cudaStream_t st) {
  const int64_t n = 3 * (int64_t)nbr;
  if (n == 0 || c1 <= c0) return cudaSuccess;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((c1 - c0 + SPMM_COLS - 1) / SPMM_COLS));
  k_spmm<<<grid, 256, 0, st>>>(nbr, rp, ci, vals, C, AC, ld, c0, c1);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Gram matrix G = C^T (AC) (Section 2.3 item (ii)): 32 x 32 output tiles (p-tile <= q-tile,
// q-tile touching [q0, nc)), each split over row chunks; per split the partial tile goes
// to scratch, then a second kernel sums the splits in a fixed order and mirrors.
// 256 threads, each owns a 2 x 2 patch of the tile.
// ------------------------------------------------------------------------------------
constexpr int GT = 32;          // tile edge
constexpr int GROWS = 32;       // rows staged per step
constexpr int GSPLIT_ROWS = 8192;   // most rows per split
constexpr int GSPLIT_MIN = 512;     // fewest rows per split
constexpr int GTARGET_CTAS = 304;   // splits are added until the grid has about this many CTAs

struct GramGeom {
  int ntile, qt0, ntiles_pairs, nsplit;
  int64_t rows;  // rows per split (a multiple of GROWS)
};

__host__ __device__ inline GramGeom gram_geom(int64_t n, int nc, int q0) {
  GramGeom g;
  g.ntile = (nc + GT - 1) / GT;
  g.qt0 = q0 / GT;
  // pairs (pt, qt) with pt <= qt, qt >= qt0
  int cnt = 0;
  for (int qt = g.qt0; qt < g.ntile; qt++) cnt += qt + 1;
  g.ntiles_pairs = cnt;
  // enough splits to fill the device (two CTAs per SM) when there are few tiles, each
  // split a multiple of GROWS rows
  int64_t nsplit = (n + GSPLIT_ROWS - 1) / GSPLIT_ROWS;
  const int64_t want = (GTARGET_CTAS + cnt - 1) / (cnt > 0 ? cnt : 1);
  const int64_t most = (n + GSPLIT_MIN - 1) / GSPLIT_MIN;
  if (nsplit < want) nsplit = want < most ? want : most;
  if (nsplit < 1) nsplit = 1;
  g.nsplit = (int)nsplit;
  g.rows = ((n + nsplit - 1) / nsplit + GROWS - 1) / GROWS * GROWS;
  return g;
}

size_t gram_scratch_doubles(int64_t n, int nc, int q0) {
  GramGeom g = gram_geom(n, nc, q0);
  return (size_t)g.ntiles_pairs * g.nsplit * GT * GT;
}

__device__ __forceinline__ void pair_of(int idx, int qt0, int& pt, int& qt) {
  qt = qt0;
  while (idx >= qt + 1) {
    idx -= qt + 1;
    qt++;
  }
  pt = idx;
}

__global__ void __launch_bounds__(256) k_gram_part(int64_t n, const double* __restrict__ C,
                                                   const double* __restrict__ AC, int64_t ld, int nc,
                                                   int qt0, int64_t rows, double* __restrict__ scratch) {
  __shared__ double sa[GROWS][GT + 1];
  __shared__ double sb[GROWS][GT + 1];
  int pt, qt;
  pair_of(blockIdx.x, qt0, pt, qt);
  const int split = blockIdx.y;
  const int64_t ra = (int64_t)split * rows;
  const int64_t rb = kmin64(n, ra + rows);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 each
  // a thread whose 2 x 2 patch lies past column nc - 1 of either tile does no arithmetic
  // (tiles at the edge of a small n_c are mostly padding)
  const bool live = (pt * GT + 2 * ty < nc) && (qt * GT + 2 * tx < nc);
  double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
  for (int64_t r = ra; r < rb; r += GROWS) {
    // stage C[r:r+32, pt*32 : pt*32+32] and AC[r:r+32, qt*32 : ...]
    for (int e = threadIdx.x; e < GROWS * GT; e += 256) {
      const int col = e / GROWS, rr = e % GROWS;
      const int64_t row = r + rr;
      const int cp = pt * GT + col, cq = qt * GT + col;
      sa[rr][col] = (row < rb && cp < nc) ? C[(int64_t)cp * ld + row] : 0.0;
      sb[rr][col] = (row < rb && cq < nc) ? AC[(int64_t)cq * ld + row] : 0.0;
    }
    __syncthreads();
    if (live) {
#pragma unroll 8
      for (int rr = 0; rr < GROWS; rr++) {
        const double a0 = sa[rr][2 * ty], a1 = sa[rr][2 * ty + 1];
        const double b0 = sb[rr][2 * tx], b1 = sb[rr][2 * tx + 1];
        acc00 += a0 * b0;
        acc01 += a0 * b1;
        acc10 += a1 * b0;
        acc11 += a1 * b1;
      }
    }
    __syncthreads();
  }
  double* out = scratch + ((int64_t)blockIdx.x * gridDim.y + split) * GT * GT;
  out[(2 * ty) * GT + 2 * tx] = acc00;
  out[(2 * ty) * GT + 2 * tx + 1] = acc01;
  out[(2 * ty + 1) * GT + 2 * tx] = acc10;
  out[(2 * ty + 1) * GT + 2 * tx + 1] = acc11;
}

__global__ void k_gram_reduce(int nc, int qt0, int nsplit, const double* __restrict__ scratch,
                              double* __restrict__ G, int ldg) {
  int pt, qt;
  pair_of(blockIdx.x, qt0, pt, qt);
  for (int e = threadIdx.x; e < GT * GT; e += blockDim.x) {
    const int lp = e / GT, lq = e % GT;
    const int p = pt * GT + lp, q = qt * GT + lq;
    if (p >= nc || q >= nc || p > q) continue;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; sp++) s += scratch[((int64_t)blockIdx.x * nsplit + sp) * GT * GT + e];
    G[(int64_t)q * ldg + p] = s;   // column-major: G[p, q]
    G[(int64_t)p * ldg + q] = s;   // mirror
  }
}

cudaError_t launch_gram(int64_t n, const double* C, const double* AC, int64_t ld, int nc, int q0,
                        double* G, int ldg, double* scratch, size_t scratch_doubles, cudaStream_t st) {
  if (nc <= 0 || q0 >= nc) return cudaSuccess;
  GramGeom g = gram_geom(n, nc, q0);
  if ((size_t)g.ntiles_pairs * g.nsplit * GT * GT > scratch_doubles) return cudaErrorInvalidValue;
  k_gram_part<<<dim3(g.ntiles_pairs, g.nsplit), 256, 0, st>>>(n, C, AC, ld, nc, g.qt0, g.rows, scratch);
  k_gram_reduce<<<g.ntiles_pairs, 256, 0, st>>>(nc, g.qt0, g.nsplit, scratch, G, ldg);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Cholesky G = L L^T (one CTA, right-looking, column-major in global memory; the matrix
// stays in L2), then Ginv = L^-T L^-1 column by column (one warp per column of the
// identity: forward then backward substitution).
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_cholesky(int nc, const double* __restrict__ G, int ldg,
                                                   double* __restrict__ L, int* status) {
  __shared__ double s_piv;
  __shared__ int s_bad;
  for (int64_t e = threadIdx.x; e < (int64_t)nc * ldg; e += blockDim.x) L[e] = G[e];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < nc; k++) {
    if (threadIdx.x == 0) {
      const double d = L[(int64_t)k * ldg + k];
      if (!(d > 0.0)) s_bad = 1;
      s_piv = sqrt(d);
      L[(int64_t)k * ldg + k] = s_piv;
    }
    __syncthreads();
    if (s_bad) break;
    const double piv = s_piv;
    for (int i = k + 1 + threadIdx.x; i < nc; i += blockDim.x) L[(int64_t)k * ldg + i] /= piv;
    __syncthreads();
    // trailing update of the lower triangle: L[row][col] -= L[row][k] L[col][k] for
    // k < col <= row < nc; consecutive threads take consecutive rows of one column
    const int m = nc - k - 1;
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      const int a = (int)(e % m), bc = (int)(e / m);
      if (bc > a) continue;
      const int row = k + 1 + a, col = k + 1 + bc;
      L[(int64_t)col * ldg + row] -= L[(int64_t)k * ldg + row] * L[(int64_t)k * ldg + col];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_bad && status) atomicCAS(status, 0, 2 /* KRS_ERR_NOT_SPD */);
}

__global__ void k_chol_inv_cols(int nc, const double* __restrict__ L, int ldg, double* __restrict__ Ginv,
                                double* __restrict__ ywork) {
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (col >= nc) return;
  double* y = ywork + (int64_t)col * nc;
  // forward: L y = e_col  (y_i = 0 for i < col)
  for (int i = 0; i < nc; i++) {
    double s = 0.0;
    if (i >= col) {
      for (int k = col + lane; k < i; k += 32) s += L[(int64_t)k * ldg + i] * y[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) y[i] = (i < col) ? 0.0 : (((i == col) ? 1.0 : 0.0) - s) / L[(int64_t)i * ldg + i];
    __syncwarp();
  }
  // backward: L^T x = y
  double* x = Ginv + (int64_t)col * ldg;
  for (int i = nc - 1; i >= 0; i--) {
    double s = 0.0;
    for (int k = i + 1 + lane; k < nc; k += 32) s += L[(int64_t)i * ldg + k] * x[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = (y[i] - s) / L[(int64_t)i * ldg + i];
    __syncwarp();
  }
}

cudaError_t launch_chol_inverse(int nc, const double* G, int ldg, double* Lwork, double* Ginv,
                                int* status, cudaStream_t st) {
  if (nc <= 0) return cudaSuccess;
  k_cholesky<<<1, 1024, 0, st>>>(nc, G, ldg, Lwork, status);
  // ywork: nc * nc doubles after the ldg*nc factor
  k_chol_inv_cols<<<(nc * 32 + 255) / 256, 256, 0, st>>>(nc, Lwork, ldg, Ginv, Lwork + (int64_t)ldg * nc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// true residual ||b - A x||^2
// ------------------------------------------------------------------------------------
__global__ void k_resid_part(int64_t n, const double* b, const double* ax, double* part) {
  __shared__ double red[2 * TPB + 2];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    const double d = b[i] - ax[i];
    s += d * d;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double* part, int cnt, double* out) {
  if (threadIdx.x < 32) {
    const double v = warp_sum_strided(part, cnt, 1);
    if (threadIdx.x == 0) *out = v;
  }
}

cudaError_t launch_true_residual(int nbr, const int* rp, const int* ci, const double* vals,
                                 const double* x, const double* b, double* tmp, double* part,
                                 double* out, cudaStream_t st) {
  const int64_t n = 3 * (int64_t)nbr;
  cudaError_t e = launch_spmv(nbr, rp, ci, vals, x, tmp, st);
  if (e != cudaSuccess) return e;
  const int blocks = 128;
  k_resid_part<<<blocks, TPB, 0, st>>>(n, b, tmp, part);
  k_sum_parts<<<1, 32, 0, st>>>(part, blocks, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// stand-alone tall-skinny kernels over general rows: CTA b owns rows [b*rpc, (b+1)*rpc)
// (rpc a multiple of 4), the same device routines as the iteration
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB, 1) k_gemv_t_rows2(const double* V, int64_t ld, int k, const double* u,
                                                         int64_t n, int64_t rpc, double* vpart, int64_t vld) {
  extern __shared__ double4_32a smem_k4[];
  double* base = reinterpret_cast<double*>(smem_k4);
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = kmin64(n, r0 + rpc);
  cta_gemv_t<true>(V, ld, k, u, r0, r1, vpart + blockIdx.x * vld, base, base + ROW_CHUNK);
}

__global__ void k_reduce_parts_cols(const double* vpart, int64_t vld, int P, int k, double* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= k) return;
  const double v = warp_sum_strided(vpart + warp, P, vld);
  if ((threadIdx.x & 31) == 0) out[warp] = v;
}

__global__ void __launch_bounds__(TPB, 1) k_gemv_n_rows2(const double* V, int64_t ld, int k, const double* s,
                                                         const double* u, double* z, int64_t n, int64_t rpc) {
  extern __shared__ double4_32a smem_k4[];
  double* base = reinterpret_cast<double*>(smem_k4);
  double* ss = base + 4 * TPB;
  for (int i = threadIdx.x; i < k; i += TPB) ss[i] = s[i];
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = kmin64(n, r0 + rpc);
  cta_gemv_n<true>(V, ld, k, ss, -1.0, u, z, r0, r1, base);
}

size_t gemv_rows_smem(int k) { return sizeof(double) * (size_t)(ROW_CHUNK + 4 * TPB + ((k + 3) & ~3)); }

cudaError_t gemv_rows_partition(int64_t n, int* P, int64_t* rpc) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t r = ((n + sms - 1) / (sms > 0 ? sms : 1) + 3) / 4 * 4;
  if (r < 64) r = 64;
  *rpc = r;
  *P = (int)((n + r - 1) / r);
  return cudaSuccess;
}

cudaError_t launch_gemv_t_rows(int64_t n, int k, const double* V, int64_t ldv, const double* u, double* t,
                               double* vpart, int P, int64_t rpc, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  if (P <= 0) return cudaMemsetAsync(t, 0, sizeof(double) * k, st);
  const size_t sm = gemv_rows_smem(0);
  cudaError_t e = cudaFuncSetAttribute((const void*)k_gemv_t_rows2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_gemv_t_rows2<<<P, TPB, sm, st>>>(V, ldv, k, u, n, rpc, vpart, k);
  k_reduce_parts_cols<<<(k * 32 + 255) / 256, 256, 0, st>>>(vpart, k, P, k, t);
  return cudaGetLastError();
}

cudaError_t launch_gemv_n_rows(int64_t n, int k, const double* V, int64_t ldv, const double* s, const double* u,
                               double* z, int P, int64_t rpc, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const size_t sm = gemv_rows_smem(k);
  cudaError_t e = cudaFuncSetAttribute((const void*)k_gemv_n_rows2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_gemv_n_rows2<<<P, TPB, sm, st>>>(V, ldv, k, s, u, z, n, rpc);
  return cudaGetLastError();
}

// out = ||v||^2 (n entries)
__global__ void k_norm2_part(int64_t n, const double* v, double* part) {
  __shared__ double red[2 * TPB + 2];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) s += v[i] * v[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

cudaError_t launch_norm2(int64_t n, const double* v, double* part, double* out, cudaStream_t st) {
  const int blocks = 128;
  k_norm2_part<<<blocks, TPB, 0, st>>>(n, v, part);
  k_sum_parts<<<1, 32, 0, st>>>(part, blocks, out);
  return cudaGetLastError();
}

// x += alpha w; r -= alpha q; partial (r, r) per CTA, then summed
__global__ void k_axpy2_dot_part(int64_t n, const double* alpha, const double* w, const double* q,
                                 double* x, double* r, double* part) {
  __shared__ double red[2 * TPB + 2];
  const double al = *alpha;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    x[i] += al * w[i];
    const double rn = r[i] - al * q[i];
    r[i] = rn;
    s += rn * rn;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

cudaError_t launch_axpy2_dot(int64_t n, const double* alpha, const double* w, const double* q, double* x,
                             double* r, double* rr, double* part, cudaStream_t st) {
  const int blocks = 152;
  k_axpy2_dot_part<<<blocks, TPB, 0, st>>>(n, alpha, w, q, x, r, part);
  k_sum_parts<<<1, 32, 0, st>>>(part, blocks, rr);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// mixed-precision refinement helpers
// ------------------------------------------------------------------------------------
__global__ void k_d2f(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

cudaError_t launch_d2f(const double* src, float* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_d2f<<<1216, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

// double-float copy of FP64 values (the matrix of the double-float precision)
__global__ void k_d2df(const double* __restrict__ src, dfl* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = dfl(src[i]);
}

cudaError_t launch_d2df(const double* src, dfl* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_d2df<<<1216, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

// x += (double) d
__global__ void k_add_f2d(double* __restrict__ x, const float* __restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

cudaError_t launch_add_f2d(double* x, const float* d, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_add_f2d<<<1216, 256, 0, st>>>(x, d, n);
  return cudaGetLastError();
}

// r = b - Ax, r32 = (float) r, partial ||r||^2 per CTA, then summed into out
__global__ void k_resid_update(int64_t n, const double* b, const double* ax, double* r, float* r32, double* part) {
  __shared__ double red[2 * TPB + 2];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    const double d = b[i] - ax[i];
    r[i] = d;
    if (r32) r32[i] = (float)d;
    s += d * d;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

cudaError_t launch_resid_update(int nbr, const int* rp, const int* ci, const double* vals, const double* x,
                                const double* b, double* ax, double* r, float* r32, double* part, double* out,
                                cudaStream_t st) {
  const int64_t n = 3 * (int64_t)nbr;
  cudaError_t e = launch_spmv(nbr, rp, ci, vals, x, ax, st);
  if (e != cudaSuccess) return e;
  const int blocks = 128;
  k_resid_update<<<blocks, TPB, 0, st>>>(n, b, ax, r, r32, part);
  k_sum_parts<<<1, 32, 0, st>>>(part, blocks, out);
  return cudaGetLastError();
}

__global__ void k_add_d(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

cudaError_t launch_add_d(double* x, const double* d, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_add_d<<<1216, 256, 0, st>>>(x, d, n);
  return cudaGetLastError();
}

__global__ void k_fill_zero(double* p, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

cudaError_t launch_fill_zero(double* p, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_fill_zero<<<256, 256, 0, st>>>(p, count);
  return cudaGetLastError();
}

}  // namespace krs
