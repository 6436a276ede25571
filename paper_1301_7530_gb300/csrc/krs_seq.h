// krs_seq.h -- the state of one sequence of solves (krs_seq_t) and the host-side stages
// of a solve, shared by the single-solve entry point and the batched engine.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "krs.h"
#include "krs_internal.h"

namespace krs {
// printf-style krs_last_error() message; returns st
krs_status failf(krs_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
}  // namespace krs

#define KRS_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      return krs::failf(KRS_ERR_CUDA, "%s failed: %s (line %d)", #call, cudaGetErrorString(e_), \
                        __LINE__);                                                           \
    }                                                                                        \
  } while (0)

#define KRS_TRY(expr)            \
  do {                           \
    krs_status s_ = (expr);      \
    if (s_ != KRS_OK) return s_; \
  } while (0)

constexpr long long kDefaultSpin = 1ll << 24;
constexpr int kMinNodesPerCta = 16;

struct krs_seq {
  int64_t n = 0, ld = 0;
  int nbr = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* uctx = nullptr;
  int sms = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;  // size of each entry of allocs
  int64_t bytes_held = 0;           // device bytes this sequence holds
  bool busy = false;                // a batched solve of this sequence is in flight

  // matrix
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* vals = nullptr;
  int64_t nnzb_cap = 0;
  const int32_t* rp_use = nullptr;
  const int32_t* ci_use = nullptr;
  const double* vals_use = nullptr;
  bool A_valid = false;
  uint64_t A_version = 0;
  int precond_built = -1;
  double* minv = nullptr;

  // augmentation space
  int nc = 0, cap_c = 0;
  double* C = nullptr;
  double* AC = nullptr;
  int ac_valid = 0;   // columns of AC valid for the current A
  int g_valid = 0;    // leading columns of G valid
  bool ginv_valid = false;
  double* G = nullptr;
  double* Lw = nullptr;
  double* Ginv = nullptr;
  int nc0 = 0;
  double* C0 = nullptr;

  // Krylov storage and vectors
  int cap_w = 0;   // columns of the FP64 W, AW (and rows of ucoef)
  int cap_sc = 0;  // iterations the scalar arrays alpha, gamma, rho, gfull hold
  // FP64 / double-float solves keep no z_j: Z is one column, reused every iteration, and
  // ucoef the packed reorthogonalisation coefficients (row j at j (j - 1) / 2: the g_i of
  // w_j = z_j - sum_{i<j} g_i w_i), from which z_j = w_j + sum_i g_i w_i when needed
  double *W = nullptr, *AW = nullptr, *Z = nullptr, *ucoef = nullptr;
  int last_reorth_full = 1;  // reorthogonalisation of the last solve (which U entries exist)
  double *x = nullptr, *r = nullptr, *u = nullptr, *b = nullptr, *tmp = nullptr;

  // scalars, partials, control
  double *alpha = nullptr, *gamma = nullptr, *rho = nullptr;
  double *tfull = nullptr, *sfull = nullptr, *gfull = nullptr;
  double* part = nullptr;
  double* vpart = nullptr;
  double* gpart = nullptr;
  int64_t vld = 0;
  int vpart_P = 0;
  int* ctrl = nullptr;
  unsigned long long* bar = nullptr;
  double* scal = nullptr;  // [0] bb, [1] rr0, [2] true residual^2

  // eigen / Ritz scratch (sized by cap_w)
  double *delta = nullptr, *eta = nullptr, *theta_m = nullptr, *theta_m1 = nullptr, *tsel = nullptr;
  int* sel = nullptr;
  int* selcount = nullptr;
  double *Qsel = nullptr, *F = nullptr, *eigwork = nullptr;
  int eig_cap = 0;

  // Gram scratch
  double* gram_scratch = nullptr;
  size_t gram_cap = 0;

  // FP32 copies for the inner solves of the mixed-precision refinement
  float *vals32 = nullptr, *minv32 = nullptr, *C32 = nullptr, *AC32 = nullptr;
  float *W32 = nullptr, *AW32 = nullptr, *Z32 = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *u32 = nullptr, *b32 = nullptr;
  double* q64 = nullptr;   // FP32-projection and double-float precisions: the FP64 product A w_j
  double* wv = nullptr;    // double-float precision: the FP64 search direction w_j
  krs::dfl* vals_df = nullptr;  // double-float precision: the matrix values as double-float pairs
  int64_t vals_df_cap = 0;
  bool vals_df_valid = false;
  // KRS_MIXED_IR: the FP64 outer directions of the flexible CG over the refinement passes
  // (p_k from pass k's FP32 correction, A-orthogonalised against the earlier p_i), their
  // products A p_k, scalars (gamma_k, coefficients, step) and partial sums
  double *Pout = nullptr, *APout = nullptr, *oscal = nullptr, *ovpart = nullptr;
  int cap_out = 0;
  double* xacc = nullptr;  //   sum of the passes' corrections
  double* rres = nullptr;  //   FP64 residual b - A xacc (the next pass's right-hand side)
  double* rrh = nullptr;   //   ||r_j||^2 history of the stall test
  int rrh_cap = 0;
  int last_prec = 0;       // precision of the last solve (what its stored directions are)
  double* dinv = nullptr;  // 1/(w, Aw) of the inner directions appended within one system
  int64_t vals32_cap = 0;
  int cap_c32 = 0, cap_w32 = 0;
  bool vals32_valid = false;
  int minv32_kind = -1;

  // pinned host mirrors
  double* h_scal = nullptr;
  int* h_ctrl = nullptr;

  // last solve
  krs_solve_stats st{};
  int last_m = 0;
  int last_ritz_m = 0;
  int last_srks = 0;
  int last_nsel = 0;
  long long spin_limit = kDefaultSpin;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace krs {

krs_status dev_alloc(krs_seq* s, size_t bytes, void** out);
void dev_free(krs_seq* s, void* p);
template <typename T>
krs_status alloc_n(krs_seq* s, T** p, size_t count) {
  void* v = nullptr;
  KRS_TRY(dev_alloc(s, count * sizeof(T), &v));
  *p = static_cast<T*>(v);
  return KRS_OK;
}
bool is_device_ptr(const void* p);
// KRS_OK when every policy field is in range (message in krs_last_error otherwise)
krs_status validate_policy(const krs_policy* p);
inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// One FP64 solve split into the stages around its iteration loop.
struct SolveState {
  int nc = 0;        // columns of C used by this solve
  int room = 0;      // columns the recycling step may append
  int kmax = 0;      // largest column count a tall-skinny phase sees
  int bps = 0;       // co-resident CTAs per SM of the persistent kernel
  IterArgs a{};      // iteration arguments (own partition)
  double tol = 0.0;
  double bb = 0.0;   // ||b||^2
  double rr0 = 0.0;  // ||r_0||^2
  bool need_iter = false;
  int add = 0;        // columns the recycling step appended (committed by seq_end)
  int outer = 0;      // mixed precision: refinement steps
  int m_first = 0;    // mixed precision: iterations of the first inner solve
  int64_t launches = 0;
  float t_iter = 0.f;
  // refinement state (KRS_MIXED_IR, KRS_MIXED_PROJ) between passes
  double rr = 0.0;     // ||b - A x||^2 of the current iterate
  double rr_best = 0.0;  // KRS_MIXED_IR: smallest ||b - A x||^2 so far, and outer steps since
  int stall = 0;         //   it last fell by 10 % (three such steps end the refinement)
  bool first = true;   // the next pass is the first one
  int status = 0;      // outcome so far
  int m = 0;           // inner iterations so far
  double m2 = 0.0;     // sum of the passes' iteration counts squared
};

// Stage 1: matrix, preconditioner, right-hand side, storage (direction capacity `cap_iter`
// columns), coarse set-up, and the init kernels (x_0, r_0, z_0, w_0, rho_0), followed by
// one read of ||b||^2 and ||r_0||^2.  On return ss->need_iter says whether iterations run.
krs_status seq_begin(krs_seq* s, const krs_bsr* A, const double* b, double tol, const krs_policy* p, int cap_iter,
                     SolveState* ss);
// Grow the direction storage of precision `prec` (FP64 W, AW and the coefficient rows, or
// FP32 W32, AW32, Z32 for KRS_MIXED_PROJ) to at least cap_iter + 1 columns keeping the
// first `keep` columns, coefficient rows and the scalars of the first `keep` iterations
// (between launches).
krs_status seq_grow_directions(krs_seq* s, int cap_iter, int keep, int prec);
// columns of the direction storage a solve of precision `prec` uses (KRS_DOUBLE_FLOAT keeps
// its double-float directions in the 8-byte W, AW of the FP64 path)
inline int dir_cap(const krs_seq* s, int prec) {
  return (prec == KRS_FP64 || prec == KRS_DOUBLE_FLOAT) ? s->cap_w : s->cap_w32;
}
// internal precision id of the iteration kernels (IterArgs::prec)
inline int prec_id(int precision) {
  return precision == KRS_MIXED_IR ? 1 : precision == KRS_MIXED_PROJ ? 2 : precision == KRS_DOUBLE_FLOAT ? 3 : 0;
}
// one APCG solve per system with an FP64 residual (no refinement loop)
inline bool single_pass(int precision) { return precision == KRS_FP64 || precision == KRS_DOUBLE_FLOAT; }
// Stage 3: recycling step (TRKS / SRKS), result copy to x (host or device), true residual,
// statistics and the commit of the new augmentation space.  `status` and `m` are the
// iteration loop's outcome.
krs_status seq_end(krs_seq* s, SolveState* ss, int status, int m, double* x, const krs_policy* p);
// Refinement (KRS_MIXED_IR, KRS_MIXED_PROJ) as resumable steps, after seq_setup-like set-up
// (refine_setup): refine_start forms the first FP64 residual; refine_pass_begin checks
// convergence and limits (*finished) and otherwise runs the next pass's init stage
// (*need_loop: the pass has iterations to run); the caller runs the pass's iteration loop
// and gives its outcome to refine_pass_end, which updates x, the residual and the
// augmentation; refine_finish ends the loop.
krs_status refine_setup(krs_seq* s, const krs_bsr* A, const double* b, const krs_policy* p, SolveState* ss);
krs_status refine_start(krs_seq* s, const krs_policy* p, double tol, SolveState* ss);
krs_status refine_pass_begin(krs_seq* s, const krs_policy* p, double tol, SolveState* ss, bool* need_loop,
                             bool* finished);
krs_status refine_pass_end(krs_seq* s, const krs_policy* p, double tol, SolveState* ss, int st_in, int m_in,
                           bool* finished);
krs_status refine_finish(krs_seq* s, const krs_policy* p, SolveState* ss);
// seq_end in three stages, for callers that finish many solves at once: stage 1 enqueues the
// first half of the recycling step (SRKS eigenvalues and selection), stage 2 -- after the
// stream was synchronised -- the rest of it, the result copy and the true residual, stage 3
// -- after another synchronisation -- the statistics and the commit.
krs_status seq_end_stage(krs_seq* s, SolveState* ss, int status, int m, double* x, const krs_policy* p, int stage);

}  // namespace krs
