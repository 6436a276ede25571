/*
 * krs.h -- C ABI of the GB300 (sm_103a) library for sequences of sparse SPD systems
 *          A^(k) x^(k) = b^(k) solved by augmented preconditioned conjugate gradient with
 *          Krylov-subspace recycling.
 *
 * Method (Gosselet, Rey & Pebrel, "Total and selective reuse of Krylov subspaces for the
 * resolution of sequences of nonlinear structural problems"):
 *   - APCG: CG preconditioned by M and augmented by the columns of C, implemented with the
 *     initialisation/projector pair x_0 = C (C^T A C)^-1 C^T b, P = I - C (C^T A C)^-1 C^T A
 *     (Section 2.1, Eq. 5, Algorithm 1), with full reorthogonalisation of the search
 *     directions in the A inner product (Section 2.1 remark; Section 5 preamble).
 *   - TRKS: after each solve, C <- [C, W_m] with W_m the solve's search directions
 *     (Section 3, Algorithm 2).
 *   - SRKS: after each solve, the Lanczos tridiagonal H_m is formed from the CG
 *     coefficients (Section 4.1, Eq. 15/17), its eigenpairs and the eigenvalues of H_{m-1}
 *     are computed, converged Ritz values are detected by stagnation (Section 4.4, Eq. 16),
 *     and C <- [C, y / sqrt(theta)] for the selected Ritz vectors y = V q (Algorithm 3).
 *
 * Conventions (every function):
 *   - Errors are returned as krs_status; nothing throws across the ABI; krs_last_error()
 *     gives a thread-local message for the last failing call of the calling thread.
 *   - Pointers are borrowed for the duration of the call only.  "host or device" pointers
 *     are classified with cudaPointerGetAttributes; pageable host memory is accepted.
 *   - Dense multi-vectors (C, W, ...) are column-major with leading dimension n.
 *   - One sequence must not be used from two threads at the same time.
 *   - A failed krs_solve leaves the sequence's augmentation space C unchanged.
 */
#ifndef KRS_H_
#define KRS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KRS_OK = 0,
  KRS_ERR_INVALID_ARG = 1,     /* bad size, pointer, pattern, policy, or non-finite b */
  KRS_ERR_NOT_SPD = 2,         /* chol(C^T A C) failed, (w, Aw) <= 0, (r, z) <= 0, or a
                                  non-positive (block) diagonal in the preconditioner */
  KRS_ERR_NO_CONVERGENCE = 3,  /* max_iter reached; x holds the last iterate */
  KRS_ERR_OOM = 4,             /* the allocator returned NULL */
  KRS_ERR_CUDA = 5,            /* a CUDA runtime call failed (message in krs_last_error) */
  KRS_ERR_TIMEOUT = 6          /* a device-side wait exceeded its bound (see spin_limit) */
} krs_status;

enum { KRS_RECYCLE_NONE = 0, KRS_RECYCLE_TRKS = 1, KRS_RECYCLE_SRKS = 2 };
enum { KRS_PRECOND_JACOBI = 0, KRS_PRECOND_BLOCK_JACOBI3 = 1, KRS_PRECOND_IDENTITY = 2 };
enum { KRS_REORTH_FULL = 0, KRS_REORTH_NONE = 1 };
enum { KRS_FP64 = 0, KRS_MIXED_IR = 1, KRS_MIXED_PROJ = 2, KRS_DOUBLE_FLOAT = 3 };
enum { KRS_CAP_TRUNCATE = 0, KRS_CAP_RESTART = 1 };
enum { KRS_EXEC_PERSISTENT = 0, KRS_EXEC_KERNELS = 1 };
enum { KRS_RESELECT_NONE = 0, KRS_RESELECT_CLUSTER = 1 };

typedef struct krs_seq* krs_seq_t;

/* 3x3 block-CSR matrix (the systems of Eq. 1 / Eq. 11).
 *   row_ptr: int32[n_block_rows + 1]; col_idx: int32[nnzb], ascending within a row, the
 *   diagonal block present; values: float64[nnzb * 9], each block row-major.
 *   on_device = 1: the three arrays are device pointers, read in place (they must stay
 *   valid and unchanged for the duration of the call) when values is 16-byte and col_idx
 *   8-byte aligned, copied to the sequence's own buffers otherwise; 0: host pointers
 *   (validated with krs_validate_bsr and copied).
 *   version: the sequence re-reads values (and rebuilds the preconditioner and A C) when
 *   version differs from the previous call's; the sparsity pattern must not change within
 *   a sequence unless version changes too. */
typedef struct {
  int32_t n_block_rows;
  int32_t block_dim;           /* must be 3 */
  int64_t nnzb;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* values;
  int32_t on_device;
  uint64_t version;
} krs_bsr;

/* Solver policy (the paper's knobs: Section 4.4 epsilon, Algorithm 3 n_clim, tolerance,
 * preconditioner, reorthogonalisation on/off).
 *   ritz_eps:   stagnation epsilon of Eq. 16 (paper: 1e-6 or 1e-14); <= 0 selects nothing.
 *   theta_frac: keep only theta < theta_frac * theta_max (theta_max of the current H_m);
 *               <= 0 disables the filter.
 *   max_aug:    cap on the number of columns of C (Algorithm 3's n_clim); 0 = no cap.
 *   cap_mode:   KRS_CAP_TRUNCATE appends new columns (ascending theta for SRKS, iteration
 *               order for TRKS) until max_aug; KRS_CAP_RESTART appends, then resets C to
 *               C^(0) once n_c >= max_aug (Algorithm 3, last step).
 *   max_iter:   iteration limit of one solve (also sizes the direction storage).
 *   exec:       KRS_EXEC_PERSISTENT runs a whole solve in one cooperative kernel with
 *               grid-wide barriers; KRS_EXEC_KERNELS launches one kernel per phase.  Both
 *               compute the same arithmetic in the same order.
 *   precision:  KRS_FP64: the whole solve in FP64.  KRS_MIXED_IR: iterative refinement --
 *               an FP64 outer loop (a flexible CG over the inner corrections, r = b - A x in
 *               FP64) around inner APCG solves A d = r whose SpMV, preconditioner,
 *               projections and reorthogonalisation run in FP32 (FP32 copies of A, M^-1,
 *               C, AC; FP32 directions), while C^T A C, its Cholesky factor and inverse,
 *               the Lanczos tridiagonal and its eigensolve stay FP64.  Every inner solve
 *               starts from the recycled space C; the recycling step (TRKS / SRKS) between
 *               systems uses the first inner solve.  An FP32 breakdown ((w, Aw) <= 0 or
 *               (r, z) <= 0) after some progress ends that inner solve only.
 *               KRS_MIXED_PROJ: one APCG solve whose operator product, preconditioner and
 *               x / r recurrences (and so the residual it converges on) are FP64, while the
 *               projection (C, AC) and the reorthogonalisation (W, AW, Z) are stored and
 *               combined in FP32 -- on GB300 those tall-skinny products are most of the FP64
 *               arithmetic of an iteration.  chol(C^T A C), x_0 / r_0 and H_m stay FP64; SRKS
 *               forms Ritz vectors from the FP32 z's; krs_last_vectors returns nothing.
 *               KRS_DOUBLE_FLOAT: the FP64 solve (operator product, preconditioner, x / r
 *               recurrences, projection with the FP64 C and AC, coarse set-up, H_m) with the
 *               search directions W, AW, Z stored as double-float pairs (hi + lo, two FP32
 *               numbers in 8 bytes: a 48-bit significand) and the reorthogonalisation's
 *               tall-skinny products taken on the FP32 pipes with error-free products and
 *               compensated sums (about 2^-46 relative per product against 2^-53 in FP64).
 *               On GB300 the FP64 pipe retires 1/64 of the FP32 rate, so these products
 *               become bound by memory instead of by FP64 arithmetic.  There is no
 *               refinement loop: the iteration converges on its FP64 residual as KRS_FP64
 *               does.  The directions must stay within the FP32 exponent range (about
 *               1e-30 .. 1e38 in magnitude keep the full significand); TRKS appends them to C
 *               in FP64, SRKS forms Ritz vectors from them in FP64, krs_last_vectors returns
 *               them as doubles.
 *   inner_tol:  KRS_MIXED_IR: relative residual the first inner solve aims for (<= 0: 0.1);
 *               later inner solves aim for max(inner_tol, 0.1), and none for less than the
 *               outer tolerance still needs.  An inner solve also ends when its residual
 *               stalls (fell less than 4x over 32 iterations once below 1e-3 of its first
 *               value), and a later one after 2 m_first + 100 iterations.  The first inner
 *               solve's Krylov space feeds the recycling step: a smaller inner_tol gives
 *               SRKS converged Ritz vectors.  The outer step is a flexible CG in FP64 over
 *               the inner solves' corrections (each A-orthogonalised against the earlier
 *               ones, step length from FP64 products).
 *   max_outer:  KRS_MIXED_IR: limit of refinement steps (<= 0: 30).  max_iter bounds the
 *               total of inner iterations.
 *   reselect:   SRKS only.  KRS_RESELECT_NONE (0), or KRS_RESELECT_CLUSTER (1): after the
 *               Eq. 16 test and the theta filter, drop the preselected Ritz values of the
 *               central cluster (Section 4.4, end): the gaps between the sorted preselected
 *               values are fitted in least squares by a three-piece constant function
 *               (pieces: gaps before, inside and after the cluster; the cluster holds at least
 *               max(2, ceil(s/5)) of the s preselected values); the cluster's values are dropped
 *               when its mean gap is smaller than that of every non-empty outer piece. */
typedef struct {
  int32_t recycle;
  int32_t precond;
  int32_t reorth;
  int32_t precision;
  double ritz_eps;
  double theta_frac;
  int32_t max_aug;
  int32_t cap_mode;
  int32_t max_iter;
  int32_t exec;
  double inner_tol;
  int32_t max_outer;
  int32_t reselect;
} krs_policy;

/* Device memory and stream.  alloc/free may be NULL (cudaMalloc/cudaFree are used);
 * otherwise every device allocation of the sequence goes through them (e.g. a framework's
 * caching allocator).  cuda_stream is a cudaStream_t (NULL = legacy default stream); all
 * work of the sequence is ordered on it.  device is the CUDA ordinal. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
  void* cuda_stream;
  int32_t device;
} krs_device;

/* Per-solve statistics (the paper's Table 1 columns: iterations, n_c, time split into
 * augmentation -- coarse preparation, initialisation -- and iterations, Section 5). */
typedef struct {
  int32_t status;
  int32_t m;              /* iterations of the solve (KRS_MIXED_IR: all inner solves) */
  int32_t n_c;            /* columns of C used by the solve */
  int32_t n_selected;     /* columns appended after the solve */
  int32_t n_c_after;      /* columns of C after the recycling step */
  double rel_res;         /* ||r_m|| / ||b|| (recursive residual) */
  double true_rel_res;    /* ||b - A x|| / ||b|| recomputed on the device */
  /* Times from CUDA events on the sequence's stream: */
  double t_setup_ms;      /* upload, preconditioner, A C, C^T A C, Cholesky, x_0, z_0 */
  double t_iter_ms;       /* exactly the iteration kernel launch(es) */
  double t_recycle_ms;    /* x copy-out, true residual, Lanczos, eigensolve, selection,
                             Ritz vectors, concatenation */
  double t_total_ms;
  int64_t kernel_launches;/* kernels this library launched for the solve */
  int32_t outer_iters;    /* refinement steps (KRS_MIXED_IR; 0 for KRS_FP64) */
  int32_t inner_m_first;  /* iterations of the first inner solve (KRS_MIXED_IR) */
  double inner_m2;        /* sum over the solve's passes of their iteration counts squared (one
                             pass: m^2); with m and outer_iters it gives the reorthogonalisation
                             work, which grows with the square of a pass's length */
} krs_solve_stats;

/* --- sequence life cycle -------------------------------------------------------------- */

/* Create a sequence for systems of order n (n = 3 * n_block_rows).  C starts empty
 * (C^(0) = [] ; Algorithms 2 and 3 allow any full-rank C_0, see krs_import_space).
 * dev may be NULL (device 0, default stream, cudaMalloc).  On success *out owns all its
 * device memory until krs_destroy_sequence. */
krs_status krs_create_sequence(int64_t n, const krs_device* dev, krs_seq_t* out);

/* Solve A x = b (zero initial guess, Section 2.1) with APCG(A, M, C, b) to
 * ||r||_2 <= tol ||b||_2 (recursive residual), then update C per the policy (TRKS:
 * Algorithm 2; SRKS: Algorithm 3).  b, x: n doubles, host or device.  On return x holds
 * x_m (also on KRS_ERR_NO_CONVERGENCE).  The call is synchronous with respect to the
 * sequence's stream (it returns after x is written). */
krs_status krs_solve(krs_seq_t s, const krs_bsr* A, const double* b, double* x, double tol,
                     const krs_policy* p);

/* Statistics of the last krs_solve. */
krs_status krs_stats(krs_seq_t s, krs_solve_stats* out);

krs_status krs_destroy_sequence(krs_seq_t s);

/* Thread-local message of the last error of the calling thread ("" if none). */
const char* krs_last_error(void);

/* Default policy: FP64, block-Jacobi, full reorthogonalisation, no recycling,
 * ritz_eps 1e-14, no theta filter, no cap, max_iter 2000, persistent execution,
 * inner_tol 0.1 and max_outer 30 (used by KRS_MIXED_IR only). */
krs_status krs_policy_default(krs_policy* p);

/* --- recycled space (checkpoint, eviction, lock-step comparison) ----------------------- */

/* Number of columns of C. */
krs_status krs_space_size(krs_seq_t s, int32_t* n_c);

/* Copy C (n x n_c, column-major) to C_out (host or device, n * n_c doubles). */
krs_status krs_export_space(krs_seq_t s, double* C_out);

/* Replace C by the n x n_c matrix C_in (host or device).  as_c0 != 0 also makes it the
 * C^(0) that KRS_CAP_RESTART returns to.  n_c = 0 empties C. */
krs_status krs_import_space(krs_seq_t s, int32_t n_c, const double* C_in, int32_t as_c0);

/* Internals of the last solve, for verification (host pointers, any may be NULL):
 * alpha[m], rho[m] = (r_j, z_j), gamma[m] = (w_j, A w_j); theta_m[m] (descending Ritz
 * values of H_m) and theta_m1[m-1] (of H_{m-1}) when the policy was SRKS and m >= 2;
 * sel[n_selected] (0-based indices into theta_m, in append order). */
krs_status krs_last_coeffs(krs_seq_t s, double* alpha, double* rho, double* gamma);
krs_status krs_last_ritz(krs_seq_t s, double* theta_m, double* theta_m1, int32_t* sel);

/* Copy the last solve's stored vectors (n x m, column-major, host or device):
 * which = 0: W (search directions w_j), 1: AW (A w_j), 2: Z (z_j = P M^-1 r_j). */
krs_status krs_last_vectors(krs_seq_t s, int32_t which, double* out);

/* Bound of every device-side wait (grid barrier spins), in spin iterations; after it the
 * kernel records KRS_ERR_TIMEOUT and returns.  0 restores the default (about 2^24). */
krs_status krs_set_spin_limit(krs_seq_t s, int64_t spins);

/* --- device memory of a sequence ------------------------------------------------------
 * The paper keeps every sequence's space in memory; a process serving many sequences
 * needs to know and bound what each holds.  These two calls have no counterpart in the
 * paper.  krs_device_bytes: device bytes the sequence holds now (its own allocations,
 * rounded to 256 bytes each).  krs_release frees parts of it between solves (never while
 * a batched solve of the sequence is in flight: KRS_ERR_INVALID_ARG):
 *   KRS_RELEASE_SCRATCH  direction storage W, AW, Z, partial sums, eigen / Gram scratch and
 *                        FP32 copies (reallocated by the next solve; krs_last_* then
 *                        return nothing);
 *   KRS_RELEASE_SPACE    C, AC, C^T A C and its factor / inverse; n_c becomes 0 (export
 *                        the space first with krs_export_space to restore it later with
 *                        krs_import_space; C^(0) of the restart mode is kept);
 *   KRS_RELEASE_MATRIX   the sequence's copy of A (re-uploaded by the next solve). */
enum { KRS_RELEASE_SCRATCH = 1, KRS_RELEASE_SPACE = 2, KRS_RELEASE_MATRIX = 4 };
krs_status krs_device_bytes(krs_seq_t s, int64_t* bytes);
krs_status krs_release(krs_seq_t s, int32_t what);

/* --- batched solves --------------------------------------------------------------------
 * An engine that runs the iteration loops of many solves -- of different sequences,
 * sizes and spaces -- in one cooperative persistent launch (the paper solves one system
 * at a time; this is the same Algorithm 1 per solve).  The grid is cut into groups of
 * group_ctas CTAs; each group takes the next solve from a queue ordered by estimated
 * remaining work (largest first) and runs it with its own barrier and partial sums.
 * Per solve, everything around the loop (set-up, init, recycling step, result, stats in
 * krs_stats of its sequence) is the same as krs_solve's, on the engine's stream.
 * Results: a solve's arithmetic depends only on group_ctas (its partition), so it is
 * bitwise the same whichever other solves share the engine; against krs_solve (another
 * partition) it differs by rounding only.
 * Direction storage starts at 1.25x the sequence's previous iteration count (12 n^(1/3)
 * for its first solve) and grows between launches when a solve fills it.
 * KRS_FP64, KRS_DOUBLE_FLOAT and KRS_MIXED_IR policies are accepted (one launch per precision
 * present); `exec` is ignored (the batched persistent kernel
 * runs every solve).  The engine must not be used from two threads at once, and a
 * sequence with a solve in flight must not be used elsewhere until it is returned. */
typedef struct krs_batch* krs_batch_t;

typedef struct {
  int32_t group_ctas;   /* CTAs per solve in every launch; 0 = chosen per launch from its
                           queue (at least SMs / solves and the largest solve's work share
                           of the SMs, times group_scale / 100), with draining */
  int32_t group_scale;  /* with group_ctas = 0: percent scale of that size; 0 = chosen by
                           the autotuner on the first launch */
  int32_t quantum;      /* iterations a solve runs per launch before the engine returns
                           control (finished solves are returned, new ones admitted);
                           0 = a launch runs until its queue is empty (or it drains) */
  int32_t reserved[5];
} krs_batch_config;

typedef struct {
  int32_t group_ctas;          /* CTAs per group of the last launch */
  int32_t groups, classes;     /* groups and group sizes of the last launch */
  int32_t in_flight;           /* submitted solves not yet returned */
  int32_t last_launch_solves;  /* solves queued in the last launch */
  int32_t tuned_group_scale;   /* autotuner's choice (0 if it did not run) */
  int64_t launches;            /* batched persistent launches so far */
  int64_t kernel_launches;     /* all kernels the engine itself launched */
  double last_kernel_ms;       /* event time of the last batched launch */
  double total_kernel_ms;
  int32_t tune_candidates;     /* entries of tune_scale / tune_ms / tune_rate */
  int32_t tune_scale[8];       /* candidate group_scale */
  double tune_ms[8];           /* probe launch time of each candidate */
  double tune_rate[8];         /* rows x iterations per second of each candidate */
} krs_batch_stats;

/* Create an engine on dev (allocator, stream, device as for krs_create_sequence); cfg may
 * be NULL (autotuned group size, quantum 0).  group_ctas larger than the SM count:
 * KRS_ERR_INVALID_ARG. */
krs_status krs_batch_create(const krs_device* dev, const krs_batch_config* cfg, krs_batch_t* out);
/* Destroy the engine; solves still in flight are dropped (their sequences stay usable). */
krs_status krs_batch_destroy(krs_batch_t b);
/* Submit one solve of sequence s (arguments as for krs_solve; x receives the result when
 * the solve is returned by krs_batch_step and must stay valid until then).  Set-up and
 * init run now; errors there (bad argument, NOT_SPD preconditioner or coarse factor) are
 * returned here and nothing is queued.  tag is returned with the result. */
krs_status krs_batch_submit(krs_batch_t b, krs_seq_t s, const krs_bsr* A, const double* rhs, double* x,
                            double tol, const krs_policy* p, int64_t tag);
/* One launch over every queued solve (at most `quantum` iterations each), then the
 * recycling step and result of every solve that ended.  Up to max_done (tag, status)
 * pairs of returned solves are written; further ones are kept for the next call.
 * A device wait that timed out ends the launch: unfinished solves return KRS_ERR_TIMEOUT. */
krs_status krs_batch_step(krs_batch_t b, int32_t max_done, int64_t* done_tags, int32_t* done_status,
                          int32_t* n_done);
/* One solve of each of `count` distinct sequences: seqs[i] with A[i], rhs[i], x[i], all
 * with tol and p; status[i] receives each solve's outcome.  Returns KRS_OK when all
 * succeeded, else the first failure.  The engine must have no solve in flight. */
krs_status krs_solve_batch(krs_batch_t b, int32_t count, const krs_seq_t* seqs, const krs_bsr* A,
                           const double* const* rhs, double* const* x, double tol, const krs_policy* p,
                           int32_t* status);
krs_status krs_batch_get_stats(krs_batch_t b, krs_batch_stats* out);

/* --- single kernels (device pointers, ordered on `stream`; asynchronous) ----------------
 * These are the building blocks of the solve, exposed for verification and measurement.
 * Scratch memory they need is allocated with cudaMallocAsync on the stream.              */

/* y = A x for a 3x3 block-CSR A (Algorithm 1's operator product).  x, y: n doubles. */
krs_status krs_spmv_bsr3(int32_t n_block_rows, const int32_t* row_ptr, const int32_t* col_idx,
                         const double* values, const double* x, double* y, void* stream);

/* Preconditioner set-up (Algorithm 1's M^-1): kind KRS_PRECOND_JACOBI writes 1/A_ii into
 * minv[n]; KRS_PRECOND_BLOCK_JACOBI3 writes the inverse of each diagonal 3x3 block into
 * minv[9 * n_block_rows] (row-major).  status (device int32, may be NULL) receives
 * KRS_ERR_NOT_SPD if a diagonal entry / block is not positive definite. */
krs_status krs_precond_setup(int32_t kind, int32_t n_block_rows, const int32_t* row_ptr,
                             const int32_t* col_idx, const double* values, double* minv,
                             int32_t* status, void* stream);

/* u = M^-1 r for a set-up preconditioner (Algorithm 1, z = P M^-1 r before projection). */
krs_status krs_precond_apply(int32_t kind, int32_t n_block_rows, const double* minv,
                             const double* r, double* u, void* stream);

/* Tall-skinny products with V (n x k, column-major, leading dimension ldv >= n):
 * t = V^T u (k doubles) -- the block dot product (AC)^T x of Section 2.3 and the
 * reorthogonalisation coefficients; z = u - V s -- the product C alpha of Section 2.3. */
krs_status krs_gemv_t(int64_t n, int32_t k, const double* V, int64_t ldv, const double* u,
                      double* t, void* stream);
krs_status krs_gemv_n_sub(int64_t n, int32_t k, const double* V, int64_t ldv,
                          const double* s, const double* u, double* z, void* stream);

/* Fused x += alpha w, r -= alpha q, rr = (r, r) (Algorithm 1's vector updates);
 * alpha and rr are device scalars. */
krs_status krs_axpy2_dot(int64_t n, const double* alpha, const double* w, const double* q,
                         double* x, double* r, double* rr, void* stream);

/* Eigenvalues (descending) of the symmetric tridiagonal matrix with diagonal delta[m] and
 * off-diagonal eta[m-1] (device pointers; theta: m doubles) by bisection on Sturm counts
 * -- the eigensolve of H_m (Section 4.1, Algorithm 3).  m <= 16001 (KRS_ERR_INVALID_ARG
 * beyond); orders whose matrix does not fit in shared memory read it from global memory. */
krs_status krs_tridiag_eigvals(int32_t m, const double* delta, const double* eta,
                               double* theta, void* stream);

/* Eigenvectors of the same matrix for the k given eigenvalues theta_sel[k] (device), by
 * inverse iteration with orthogonalisation inside clusters; Q_out: m x k column-major,
 * unit 2-norm, sign fixed so that the largest-magnitude component is positive. */
krs_status krs_tridiag_eigvecs(int32_t m, const double* delta, const double* eta, int32_t k,
                               const double* theta_sel, double* Q_out, void* stream);

/* t = V^T u exactly as krs_gemv_t computes it (same partition, same summation order), but
 * allocating no device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate -- a framework that has reserved the device memory for its
 * own pool, a latency-bound loop that cannot pay for an allocation or its implicit
 * synchronisation, code where another component owns every allocation.  Its per-block
 * partial sums live in a fixed 2 MiB array in device global memory that every GPU loading
 * the library holds until the process exits.  Limits: k <= 1024 (larger k returns
 * KRS_ERR_INVALID_ARG with a message); the row blocks follow krs_gemv_t's partition (at
 * most one per SM).  The first call on each device looks up the array's device address on
 * that device (and a call made under a new context of that device, after cudaDeviceReset
 * for instance, looks it up again); make that first call before any stream capture.  It
 * launches krs_gemv_t's own kernels on krs_gemv_t's partition.  All calls share the array
 * and it keeps the previous call's contents (nothing needs clearing: every value read is
 * written first by the same call); calls whose kernels overlap on the GPU race.
 * Arguments, layout and alignment as for krs_gemv_t; asynchronous on `stream`. */
krs_status krs_gemv_t_noalloc(int64_t n, int32_t k, const double* V, int64_t ldv, const double* u,
                              double* t, void* stream);

/* Host-only validation of a BSR pattern (no GPU needed): sizes, monotone row_ptr, column
 * indices in range and strictly ascending per row, diagonal block present.  Host arrays. */
krs_status krs_validate_bsr(int32_t n_block_rows, int64_t nnzb, const int32_t* row_ptr,
                            const int32_t* col_idx);

/* Library version string. */
const char* krs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KRS_H_ */
