// krs_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "krs.h"

namespace krs {

// internal solve status (never returned through the ABI): the residual stopped decreasing
constexpr int KRS_STALLED = 7;

// Records msg as the calling thread's krs_last_error() and returns st.
krs_status set_error(krs_status st, const char* msg);

// Everything the iteration kernels need (device pointers, sizes, partition).  The element
// types of the arrays follow `prec` (matrix values, M^-1, x, r, u: FP32 for prec 1, FP64
// otherwise; C, AC: FP64 for prec 0 and 3, FP32 otherwise; W, AW, Z: FP64 for prec 0,
// double-float pairs for prec 3, FP32 otherwise); scalars, partial sums and G^-1 are
// doubles in all.
struct IterArgs {
  int64_t n, ld;
  int nbr, npc, P;
  int nc, ldg;
  int nc_dense;          // columns of C with the dense coarse inverse Ginv (the rest: dinv)
  const double* dinv;    // 1/(w_i, A w_i) for columns [nc_dense, nc)
  int max_iter, reorth_full, precond;
  int jcap;  // iterations j >= jcap do not start in one launch (0: no limit)
  int kmax;  // largest k a tall-skinny phase sees: max(nc, max_iter)
  int prec;  // 0: FP64; 1: FP32 (mixed-precision inner solves); 2: FP64 recurrences with FP32
             // projection / reorthogonalisation (C, AC, W, AW, Z in FP32, q in FP64);
             // 3: FP64 with double-float W, AW, Z and matrix values for the operator
             //    product (q and wv in FP64)
  double tol2;
  long long spin_limit;
  const int* rp;
  const int* ci;
  const void* vals;
  const void* minv;
  const void* C;
  const void* AC;
  const void* Ci;   // C and AC of the init stage (nullptr: C, AC); FP64 for prec 2
  const void* ACi;
  const double* Ginv;
  void *W, *AW, *Z, *x, *r, *u;
  int64_t zld;      // stride of the z columns: ld (Z holds z_j for every j) or 0 (FP64 and
                    // double-float: one z column reused every iteration; the coefficients
                    // of each w_j go to ucoef instead, so that z_j = w_j + sum_i g_i w_i)
  double* ucoef;    // zld == 0: packed rows of those coefficients (row j at j (j - 1) / 2)
  void* q;          // prec 2, 3: FP64 product A w_j
  void* wv;         // prec 3: FP64 search direction w_j (n + padding doubles)
  const void* vals_df;  // prec 3: matrix values as double-float pairs (9 nnzb)
  bool init32;      // prec 2: the init stage reads the FP32 C and AC (restarted passes)
  int stall_win;    // > 0: end the solve when ||r||^2 fell by less than 4x over this many
                    //      iterations (status KRS_STALLED), once it is below stall_rr
  double stall_rr;
  double* rrh;      // ||r_j||^2 history (stall_win > 0)
  double *alpha, *gamma, *rho;
  double *tfull, *sfull, *gfull;
  double* part;
  double* vpart;
  double* gpart;
  int64_t vld;
  int* ctrl;
  unsigned long long* bar;
};

// One launch of the batched persistent kernel (FP64).  The `ctas` CTAs are cut into groups
// (contiguous CTA ranges); the groups of one size form a class.  A group takes solves from
// its class's queue (indices into the device array of contexts written by apcg_fill_ctx,
// each prepared for that class's group size) and runs each for at most `quantum`
// iterations (<= 0: no limit).  All arrays are device arrays.
struct BatchLaunch {
  const void* ctxs;
  const int* queue;           // concatenated class queues
  const int* qoff;            // [classes + 1]
  int* heads;                 // [classes], zeroed before the launch
  const int* cta_group;       // [ctas]
  const int* grp_cta0;        // [groups + 1]
  const int* grp_class;       // [groups]
  int ctas, quantum, kmax;
  int drain_at;               // suspend every solve once this many groups are idle (0: never)
  int* idle;                  // idle-group counter, zeroed before the launch
  int* gstop;                 // [groups] drain words, zeroed before the launch
  int* mail;                  // [2 * groups]
  unsigned long long* gbar;   // [16 * groups], zeroed before the launch
  double *gpart, *gvpart, *ggpart;  // [ctas * PS_STRIDE], [ctas * vld], [ctas * vld]
  int64_t vld;
  long long spin_limit;
  int* bctrl;                 // [CTRL_WORDS], zeroed before the launch
};

// krs_apcg.cu
size_t apcg_smem_bytes(int kmax);
size_t apcg_ctx_bytes();
void apcg_fill_ctx(const IterArgs& a, void* dst);
cudaError_t apcg_batched_coresident(int kmax, int prec, int* blocks_per_sm);
cudaError_t apcg_launch_batched(const BatchLaunch& L, int prec, cudaStream_t st);
// out[4 p + w], w = CTRL_STATUS, CTRL_DONE, CTRL_M, CTRL_J of the control block of ctxs[p]
cudaError_t apcg_gather_ctrl(const void* ctxs, int count, int* out, cudaStream_t st);
cudaError_t apcg_prepare_attributes(int kmax, int prec);
cudaError_t apcg_max_coresident(int kmax, int prec, int* blocks_per_sm);
cudaError_t apcg_launch_init(const IterArgs& a, const void* b, double* scal, cudaStream_t st, int64_t* launches);
cudaError_t apcg_launch_persistent(const IterArgs& a, cudaStream_t st, int64_t* launches);
cudaError_t apcg_launch_phases(const IterArgs& a, int j0, int j1, cudaStream_t st, int64_t* launches);

// krs_kernels.cu
cudaError_t launch_spmv(int nbr, const int* rp, const int* ci, const double* vals, const double* x,
                        double* y, cudaStream_t st);
cudaError_t launch_precond_setup(int kind, int nbr, const int* rp, const int* ci, const double* vals,
                                 double* minv, int* status, cudaStream_t st);
cudaError_t launch_precond_apply(int kind, int nbr, const double* minv, const double* r, double* u,
                                 cudaStream_t st);
// AC[:, c0:c1] = A C[:, c0:c1]  (column-major, leading dimension ld, same summation order
// as the iteration's operator product)
cudaError_t launch_spmm(int nbr, const int* rp, const int* ci, const double* vals, const double* C,
                        double* AC, int64_t ld, int c0, int c1, cudaStream_t st);
// G[p, q] = C[:, p] . AC[:, q] for q in [q0, nc), p <= q, mirrored (G: nc x nc, ldg)
cudaError_t launch_gram(int64_t n, const double* C, const double* AC, int64_t ld, int nc, int q0,
                        double* G, int ldg, double* scratch, size_t scratch_doubles, cudaStream_t st);
size_t gram_scratch_doubles(int64_t n, int nc, int q0);
// Ginv = G^-1 via Cholesky (L in Lwork); status <- KRS_ERR_NOT_SPD on failure
cudaError_t launch_chol_inverse(int nc, const double* G, int ldg, double* Lwork, double* Ginv,
                                int* status, cudaStream_t st);
// res2 = ||b - A x||^2 (scal[0]); uses tmp (n doubles)
cudaError_t launch_true_residual(int nbr, const int* rp, const int* ci, const double* vals,
                                 const double* x, const double* b, double* tmp, double* part,
                                 double* out, cudaStream_t st);
// tall-skinny products over general rows (CTA b owns rows [b*rpc, (b+1)*rpc), rpc % 4 == 0)
// partition of n rows for them: rpc = n / SMs rounded up to a multiple of 4 (at least 64),
// P = ceil(n / rpc) row blocks (at most one per SM)
cudaError_t gemv_rows_partition(int64_t n, int* P, int64_t* rpc);
cudaError_t launch_gemv_t_rows(int64_t n, int k, const double* V, int64_t ldv, const double* u, double* t,
                               double* vpart, int P, int64_t rpc, cudaStream_t st);
cudaError_t launch_gemv_n_rows(int64_t n, int k, const double* V, int64_t ldv, const double* s, const double* u,
                               double* z, int P, int64_t rpc, cudaStream_t st);
cudaError_t launch_norm2(int64_t n, const double* v, double* part, double* out, cudaStream_t st);
cudaError_t launch_axpy2_dot(int64_t n, const double* alpha, const double* w, const double* q, double* x,
                             double* r, double* rr, double* part, cudaStream_t st);
cudaError_t launch_fill_zero(double* p, int64_t count, cudaStream_t st);
// mixed-precision refinement: dst = (float) src; x += (double) d; r = b - A x (FP64),
// r32 = (float) r (skipped when r32 is NULL), out = ||r||^2 (ax: n-vector scratch, part:
// >= 128 doubles)
cudaError_t launch_d2f(const double* src, float* dst, int64_t count, cudaStream_t st);
struct dfl;
cudaError_t launch_d2df(const double* src, dfl* dst, int64_t count, cudaStream_t st);  // dst = double-float src
cudaError_t launch_add_f2d(double* x, const float* d, int64_t n, cudaStream_t st);
cudaError_t launch_add_d(double* x, const double* d, int64_t n, cudaStream_t st);  // x += d
cudaError_t launch_resid_update(int nbr, const int* rp, const int* ci, const double* vals, const double* x,
                                const double* b, double* ax, double* r, float* r32, double* part, double* out,
                                cudaStream_t st);

// krs_eig.cu
// delta/eta of H_m from alpha, rho (Section 4.1)
cudaError_t launch_lanczos(int m, const double* alpha, const double* rho, double* delta, double* eta,
                           cudaStream_t st);
cudaError_t launch_tridiag_eigvals(int m, const double* delta, const double* eta, double* theta,
                                   cudaStream_t st);
cudaError_t launch_tridiag_eigvecs(int m, const double* delta, const double* eta, int k,
                                   const double* theta_sel, double* Q, double* work, cudaStream_t st);
size_t eigvecs_work_doubles(int m, int k);
// SRKS selection on device: sel[0..cnt) (ascending theta), cnt in *count, theta values in tsel
// reselect: 1 = cluster reselection (Section 4.4, end); tsel: 5m doubles of scratch
cudaError_t launch_srks_select(int m, const double* theta_m, const double* theta_m1, double eps,
                               double theta_frac, int reselect, int room, int* sel, int* count, double* tsel,
                               cudaStream_t st);
// Y[:, c] = sum_j z_j (-1)^j Q[j, c] / sqrt(rho_j) / sqrt|theta_c|  for c < k, with the z_j
// given as W U: z_j = w_j + sum_{i<j} U[i, j] w_i, U packed by rows of j (row j at
// j (j - 1) / 2, entries i < j; full == 0: only i = j - 1 is used).  W: FP64, or
// double-float pairs when w_df.  F: m k doubles, F2: m k doubles (scratch).
cudaError_t launch_ritz_vectors_wu(int64_t n, int64_t ld, int m, int k, const void* W, bool w_df, const double* ucoef,
                                   int full, const double* rho, const double* Q, const double* tsel, double* F,
                                   double* F2, double* Y, cudaStream_t st);
// Z = W U (the z_j of a solve that did not store them), n x m into Y (leading dimension ld);
// Ud: m m doubles of scratch
cudaError_t launch_z_from_wu(int64_t n, int64_t ld, int m, const void* W, bool w_df, const double* ucoef, int full,
                             double* Ud, double* Y, cudaStream_t st);
// Y[:, c] = sum_j Z[:, j] (-1)^j Q[j, c] / sqrt(rho_j) / sqrt|theta_c|  for c < k, from the
// FP32 z_j of an inner solve of the mixed-precision refinement
cudaError_t launch_ritz_vectors_f(int64_t n, int64_t ld, int m, int k, const float* Z, const double* rho,
                                  const double* Q, const double* tsel, double* F, double* Y, cudaStream_t st);

}  // namespace krs
