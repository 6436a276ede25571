// krs_api.cu -- the C ABI (include/krs.h): sequence state, device memory, and the
// orchestration of one solve of the sequence:
//   set-up  : upload A if its version changed, preconditioner, A C (new columns only
//             while A is unchanged), C^T A C (new tiles only while A is unchanged), its
//             Cholesky factor and inverse (Algorithm 1 step 1; Section 2.3);
//   init    : x_0, r_0, z_0, w_0 (Algorithm 1 steps 2-3);
//   iterate : the persistent kernel or the per-phase kernels (krs_apcg.cu);
//   recycle : TRKS (Algorithm 2) or SRKS (Algorithm 3) on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "krs.h"
#include "krs_device.cuh"
#include "krs_internal.h"
#include "krs_seq.h"

using namespace krs;

namespace krs {
// eigenvalues of H_m and of its leading block of order m1 (Sturm multisection); e2_scratch:
// m doubles, used when the order is too large to stage the matrix in shared memory
cudaError_t launch_tridiag_eigvals2(int m, int m1, const double* delta, const double* eta, double* theta_m,
                                    double* theta_m1, cudaStream_t st, double* e2_scratch);
}
static cudaError_t launch_df2d(const dfl* src, double* dst, int64_t count, cudaStream_t st);

static thread_local std::string g_last_error;

krs_status krs::failf(krs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}
#define fail krs::failf

krs_status krs::set_error(krs_status st, const char* msg) {
  g_last_error = msg;
  return st;
}

// ------------------------------------------------------------------------------------
// memory helpers
// ------------------------------------------------------------------------------------
krs_status krs::dev_alloc(krs_seq* s, size_t bytes, void** out) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  if (s->ualloc) {
    p = s->ualloc(bytes, s->uctx);
    if (!p) return fail(KRS_ERR_OOM, "allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? KRS_ERR_OOM : KRS_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                  cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaMemsetAsync(p, 0, bytes, s->stream);
  if (e != cudaSuccess) return fail(KRS_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  s->allocs.push_back(p);
  s->alloc_bytes.push_back(bytes);
  s->bytes_held += (int64_t)bytes;
  *out = p;
  return KRS_OK;
}

void krs::dev_free(krs_seq* s, void* p) {
  if (!p) return;
  for (size_t i = 0; i < s->allocs.size(); i++) {
    if (s->allocs[i] == p) {
      s->bytes_held -= (int64_t)s->alloc_bytes[i];
      s->allocs[i] = s->allocs.back();
      s->alloc_bytes[i] = s->alloc_bytes.back();
      s->allocs.pop_back();
      s->alloc_bytes.pop_back();
      break;
    }
  }
  if (s->ufree) {
    cudaStreamSynchronize(s->stream);
    s->ufree(p, s->uctx);
  } else {
    cudaFree(p);
  }
}

bool krs::is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// grow C / AC (and C^T A C work) to hold `need` columns, keeping the first nc columns
static krs_status ensure_cap_c(krs_seq* s, int need) {
  if (need <= s->cap_c) return KRS_OK;
  int cap = s->cap_c ? s->cap_c : 16;
  while (cap < need) cap *= 2;
  double *C = nullptr, *AC = nullptr, *G = nullptr, *Lw = nullptr, *Gi = nullptr;
  KRS_TRY(alloc_n(s, &C, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &AC, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &G, (size_t)cap * cap));
  KRS_TRY(alloc_n(s, &Lw, (size_t)2 * cap * cap));
  KRS_TRY(alloc_n(s, &Gi, (size_t)cap * cap));
  if (s->nc > 0) {
    KRS_CUDA(cudaMemcpyAsync(C, s->C, sizeof(double) * (size_t)s->nc * s->ld, cudaMemcpyDeviceToDevice, s->stream));
    if (s->ac_valid > 0)
      KRS_CUDA(cudaMemcpyAsync(AC, s->AC, sizeof(double) * (size_t)s->ac_valid * s->ld, cudaMemcpyDeviceToDevice,
                               s->stream));
  }
  if (s->g_valid > 0 && s->G)  // keep the valid leading block of C^T A C (new leading dimension)
    KRS_CUDA(cudaMemcpy2DAsync(G, sizeof(double) * cap, s->G, sizeof(double) * s->cap_c, sizeof(double) * s->g_valid,
                               s->g_valid, cudaMemcpyDeviceToDevice, s->stream));
  dev_free(s, s->C);  // cudaFree / the stream sync in dev_free orders it after the copies
  dev_free(s, s->AC);
  dev_free(s, s->G);
  dev_free(s, s->Lw);
  dev_free(s, s->Ginv);
  s->C = C;
  s->AC = AC;
  s->G = G;
  s->Lw = Lw;
  s->Ginv = Gi;
  s->cap_c = cap;
  s->ginv_valid = false;
  return KRS_OK;
}

// scalar arrays of the iteration (alpha, gamma, rho, g) for `need` iterations; the first
// `keep` iterations' values are kept
static krs_status ensure_scalars(krs_seq* s, int need, int keep) {
  if (need <= s->cap_sc) return KRS_OK;
  const int cap = (int)round_up(need, 32);
  double *al = nullptr, *ga = nullptr, *rh = nullptr, *gf = nullptr;
  KRS_TRY(alloc_n(s, &al, cap));
  KRS_TRY(alloc_n(s, &ga, cap));
  KRS_TRY(alloc_n(s, &rh, cap + 1));
  KRS_TRY(alloc_n(s, &gf, cap));
  if (keep > s->cap_sc) keep = s->cap_sc;
  if (keep > 0) {
    KRS_CUDA(cudaMemcpyAsync(al, s->alpha, sizeof(double) * keep, cudaMemcpyDeviceToDevice, s->stream));
    KRS_CUDA(cudaMemcpyAsync(ga, s->gamma, sizeof(double) * keep, cudaMemcpyDeviceToDevice, s->stream));
    KRS_CUDA(cudaMemcpyAsync(rh, s->rho, sizeof(double) * (keep + 1), cudaMemcpyDeviceToDevice, s->stream));
  }
  dev_free(s, s->alpha);
  dev_free(s, s->gamma);
  dev_free(s, s->rho);
  dev_free(s, s->gfull);
  s->alpha = al;
  s->gamma = ga;
  s->rho = rh;
  s->gfull = gf;
  s->cap_sc = cap;
  return KRS_OK;
}

// packed reorthogonalisation coefficient rows of `cap` columns (rows 1 .. cap - 1)
static size_t ucoef_entries(int cap) { return cap > 1 ? (size_t)cap * (size_t)(cap - 1) / 2 : 1; }

// FP64 direction storage (W, AW, one z column, the coefficient rows U) and the scalars for
// max_iter iterations
static krs_status ensure_cap_w(krs_seq* s, int max_iter) {
  const int need = max_iter + 1;
  KRS_TRY(ensure_scalars(s, need, 0));
  if (!s->Z) KRS_TRY(alloc_n(s, &s->Z, (size_t)s->ld));
  if (need <= s->cap_w) return KRS_OK;
  int cap = (int)round_up(need, 32);
  dev_free(s, s->W);
  dev_free(s, s->AW);
  dev_free(s, s->ucoef);
  s->W = s->AW = s->ucoef = nullptr;
  KRS_TRY(alloc_n(s, &s->W, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &s->AW, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &s->ucoef, ucoef_entries(cap)));
  s->cap_w = cap;
  return KRS_OK;
}

// FP32 direction storage (W32, AW32, Z32) for `need` columns and the scalars; the first
// `keep` columns / iterations are kept
static krs_status ensure_w32(krs_seq* s, int need, int keep) {
  KRS_TRY(ensure_scalars(s, need, keep));
  if (need <= s->cap_w32) return KRS_OK;
  const int cap = (int)round_up(need, 32);
  float *W = nullptr, *AW = nullptr, *Z = nullptr;
  KRS_TRY(alloc_n(s, &W, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &AW, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &Z, (size_t)cap * s->ld));
  if (keep > s->cap_w32) keep = s->cap_w32;
  if (keep > 0) {
    const size_t vb = sizeof(float) * (size_t)keep * s->ld;
    KRS_CUDA(cudaMemcpyAsync(W, s->W32, vb, cudaMemcpyDeviceToDevice, s->stream));
    KRS_CUDA(cudaMemcpyAsync(AW, s->AW32, vb, cudaMemcpyDeviceToDevice, s->stream));
    KRS_CUDA(cudaMemcpyAsync(Z, s->Z32, vb, cudaMemcpyDeviceToDevice, s->stream));
  }
  dev_free(s, s->W32);
  dev_free(s, s->AW32);
  dev_free(s, s->Z32);
  s->W32 = W;
  s->AW32 = AW;
  s->Z32 = Z;
  s->cap_w32 = cap;
  return KRS_OK;
}

static krs_status ensure_vpart(krs_seq* s, int P, int kmax) {
  const int64_t vld = round_up(kmax + 1, 32);
  if (P <= s->vpart_P && vld <= s->vld) return KRS_OK;
  const int Pn = P > s->vpart_P ? P : s->vpart_P;
  const int64_t vn = vld > s->vld ? vld : s->vld;
  dev_free(s, s->vpart);
  dev_free(s, s->gpart);
  dev_free(s, s->part);
  dev_free(s, s->tfull);
  dev_free(s, s->sfull);
  KRS_TRY(alloc_n(s, &s->vpart, (size_t)Pn * vn));
  KRS_TRY(alloc_n(s, &s->gpart, (size_t)Pn * vn));
  KRS_TRY(alloc_n(s, &s->part, (size_t)Pn * PS_STRIDE + 256));
  KRS_TRY(alloc_n(s, &s->tfull, vn));
  KRS_TRY(alloc_n(s, &s->sfull, vn));
  s->vpart_P = Pn;
  s->vld = vn;
  return KRS_OK;
}

static krs_status ensure_eig(krs_seq* s, int m) {
  if (m <= s->eig_cap) return KRS_OK;
  const int cap = (int)round_up(m, 64);
  dev_free(s, s->delta);
  dev_free(s, s->eta);
  dev_free(s, s->theta_m);
  dev_free(s, s->theta_m1);
  dev_free(s, s->tsel);
  dev_free(s, s->sel);
  KRS_TRY(alloc_n(s, &s->delta, cap));
  KRS_TRY(alloc_n(s, &s->eta, cap));
  KRS_TRY(alloc_n(s, &s->theta_m, cap));
  KRS_TRY(alloc_n(s, &s->theta_m1, cap));
  KRS_TRY(alloc_n(s, &s->tsel, 5 * (size_t)cap));
  KRS_TRY(alloc_n(s, &s->sel, cap));
  s->eig_cap = cap;
  return KRS_OK;
}

// partition of the block rows over P CTAs (npc nodes each, a multiple of 4)
static void partition(const krs_seq* s, int blocks_per_sm, int* P, int* npc) {
  const int pmax = (blocks_per_sm > 0 ? blocks_per_sm : 1) * s->sms;
  int64_t per = (s->nbr + pmax - 1) / pmax;
  if (per < kMinNodesPerCta) per = kMinNodesPerCta;
  per = round_up(per, 4);
  *npc = (int)per;
  *P = (int)((s->nbr + per - 1) / per);
  if (*P < 1) *P = 1;
}

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" {

const char* krs_last_error(void) { return g_last_error.c_str(); }

const char* krs_version(void) { return "krs 0.1 (sm_103a)"; }

krs_status krs_policy_default(krs_policy* p) {
  if (!p) return fail(KRS_ERR_INVALID_ARG, "policy is NULL");
  memset(p, 0, sizeof(*p));
  p->recycle = KRS_RECYCLE_NONE;
  p->precond = KRS_PRECOND_BLOCK_JACOBI3;
  p->reorth = KRS_REORTH_FULL;
  p->precision = KRS_FP64;
  p->ritz_eps = 1e-14;
  p->theta_frac = 0.0;
  p->max_aug = 0;
  p->cap_mode = KRS_CAP_TRUNCATE;
  p->max_iter = 2000;
  p->exec = KRS_EXEC_PERSISTENT;
  p->inner_tol = 0.1;
  p->max_outer = 30;
  return KRS_OK;
}

krs_status krs_validate_bsr(int32_t nbr, int64_t nnzb, const int32_t* rp, const int32_t* ci) {
  if (nbr < 0 || nnzb < 0) return fail(KRS_ERR_INVALID_ARG, "negative size");
  if (nbr > 0 && (!rp || !ci)) return fail(KRS_ERR_INVALID_ARG, "NULL pattern array");
  if (nbr == 0) return KRS_OK;
  if (rp[0] != 0) return fail(KRS_ERR_INVALID_ARG, "row_ptr[0] = %d, expected 0", rp[0]);
  if ((int64_t)rp[nbr] != nnzb) return fail(KRS_ERR_INVALID_ARG, "row_ptr[n] = %d != nnzb %lld", rp[nbr], (long long)nnzb);
  for (int i = 0; i < nbr; i++) {
    if (rp[i + 1] < rp[i]) return fail(KRS_ERR_INVALID_ARG, "row_ptr decreases at row %d", i);
    int has_diag = 0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
      if (ci[k] < 0 || ci[k] >= nbr) return fail(KRS_ERR_INVALID_ARG, "col_idx[%d] = %d out of range", k, ci[k]);
      if (k > rp[i] && ci[k] <= ci[k - 1]) return fail(KRS_ERR_INVALID_ARG, "row %d columns not strictly ascending", i);
      if (ci[k] == i) has_diag = 1;
    }
    if (!has_diag) return fail(KRS_ERR_INVALID_ARG, "row %d has no diagonal block", i);
  }
  return KRS_OK;
}

krs_status krs_create_sequence(int64_t n, const krs_device* dev, krs_seq_t* out) {
  if (!out) return fail(KRS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || n % 3 != 0 || n / 3 > 0x7fffffff) return fail(KRS_ERR_INVALID_ARG, "n = %lld must be a positive multiple of 3", (long long)n);
  if (dev && ((dev->alloc == nullptr) != (dev->free == nullptr)))
    return fail(KRS_ERR_INVALID_ARG, "alloc and free must both be set or both be NULL");
  krs_seq* s = new (std::nothrow) krs_seq();
  if (!s) return fail(KRS_ERR_OOM, "host allocation failed");
  s->n = n;
  s->nbr = (int)(n / 3);
  s->ld = round_up(n, 32);
  if (dev) {
    s->device = dev->device;
    s->stream = (cudaStream_t)dev->cuda_stream;
    s->ualloc = dev->alloc;
    s->ufree = dev->free;
    s->uctx = dev->ctx;
  }
  auto bail = [&](krs_status st) {
    krs_destroy_sequence(s);
    return st;
  };
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) {
    delete s;
    return fail(KRS_ERR_CUDA, "cudaSetDevice(%d): %s", dev ? dev->device : 0, cudaGetErrorString(e));
  }
  e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  if (e != cudaSuccess) {
    delete s;
    return fail(KRS_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
  }
  krs_status st;
  if ((st = alloc_n(s, &s->x, s->ld)) || (st = alloc_n(s, &s->r, s->ld)) || (st = alloc_n(s, &s->u, s->ld)) ||
      (st = alloc_n(s, &s->b, s->ld)) || (st = alloc_n(s, &s->tmp, s->ld)) ||
      (st = alloc_n(s, &s->minv, 3 * s->ld + 64)) || (st = alloc_n(s, &s->ctrl, 64)) ||
      (st = alloc_n(s, &s->bar, 8)) || (st = alloc_n(s, &s->scal, 16)) || (st = alloc_n(s, &s->selcount, 8)))
    return bail(st);
  if (cudaMallocHost(&s->h_scal, 16 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&s->h_ctrl, 64 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(KRS_ERR_OOM, "pinned host allocation failed"));
  }
  for (int i = 0; i < 6; i++) {
    if (cudaEventCreate(&s->ev[i]) != cudaSuccess) return bail(fail(KRS_ERR_CUDA, "cudaEventCreate failed"));
  }
  *out = s;
  return KRS_OK;
}

krs_status krs_destroy_sequence(krs_seq_t s) {
  if (!s) return KRS_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  std::vector<void*> all = s->allocs;
  for (void* p : all) dev_free(s, p);
  if (s->h_scal) cudaFreeHost(s->h_scal);
  if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
  for (int i = 0; i < 6; i++)
    if (s->ev[i]) cudaEventDestroy(s->ev[i]);
  delete s;
  return KRS_OK;
}

krs_status krs_stats(krs_seq_t s, krs_solve_stats* out) {
  if (!s || !out) return fail(KRS_ERR_INVALID_ARG, "NULL argument");
  *out = s->st;
  return KRS_OK;
}

krs_status krs_set_spin_limit(krs_seq_t s, int64_t spins) {
  if (!s || spins < 0) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  s->spin_limit = spins ? spins : kDefaultSpin;
  return KRS_OK;
}

krs_status krs_space_size(krs_seq_t s, int32_t* n_c) {
  if (!s || !n_c) return fail(KRS_ERR_INVALID_ARG, "NULL argument");
  *n_c = s->nc;
  return KRS_OK;
}

krs_status krs_export_space(krs_seq_t s, double* C_out) {
  if (!s || (!C_out && s->nc > 0)) return fail(KRS_ERR_INVALID_ARG, "NULL argument");
  if (s->nc == 0) return KRS_OK;
  KRS_CUDA(cudaSetDevice(s->device));
  const bool dv = is_device_ptr(C_out);
  KRS_CUDA(cudaMemcpy2DAsync(C_out, sizeof(double) * s->n, s->C, sizeof(double) * s->ld, sizeof(double) * s->n,
                             s->nc, dv ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  return KRS_OK;
}

krs_status krs_import_space(krs_seq_t s, int32_t n_c, const double* C_in, int32_t as_c0) {
  if (!s || n_c < 0 || (n_c > 0 && !C_in)) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  KRS_CUDA(cudaSetDevice(s->device));
  KRS_TRY(ensure_cap_c(s, n_c));
  const bool dv = n_c > 0 && is_device_ptr(C_in);
  if (n_c > 0)
    KRS_CUDA(cudaMemcpy2DAsync(s->C, sizeof(double) * s->ld, C_in, sizeof(double) * s->n, sizeof(double) * s->n,
                               n_c, dv ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  s->nc = n_c;
  s->ac_valid = 0;
  s->g_valid = 0;
  s->ginv_valid = false;
  if (as_c0) {
    dev_free(s, s->C0);
    s->C0 = nullptr;
    s->nc0 = n_c;
    if (n_c > 0) {
      KRS_TRY(alloc_n(s, &s->C0, (size_t)n_c * s->ld));
      KRS_CUDA(cudaMemcpyAsync(s->C0, s->C, sizeof(double) * (size_t)n_c * s->ld, cudaMemcpyDeviceToDevice,
                               s->stream));
    }
  }
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  return KRS_OK;
}

krs_status krs_device_bytes(krs_seq_t s, int64_t* bytes) {
  if (!s || !bytes) return fail(KRS_ERR_INVALID_ARG, "NULL argument");
  *bytes = s->bytes_held;
  return KRS_OK;
}

krs_status krs_release(krs_seq_t s, int32_t what) {
  if (!s || (what & ~(KRS_RELEASE_SCRATCH | KRS_RELEASE_SPACE | KRS_RELEASE_MATRIX)))
    return fail(KRS_ERR_INVALID_ARG, "bad argument");
  if (s->busy) return fail(KRS_ERR_INVALID_ARG, "the sequence has a solve in flight");
  KRS_CUDA(cudaSetDevice(s->device));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  auto drop = [&](auto*& p) {
    dev_free(s, p);
    p = nullptr;
  };
  if (what & KRS_RELEASE_SCRATCH) {
    drop(s->W); drop(s->AW); drop(s->Z); drop(s->ucoef);
    drop(s->alpha); drop(s->gamma); drop(s->rho); drop(s->gfull);
    s->cap_w = 0;
    s->cap_sc = 0;
    drop(s->q64); drop(s->wv); drop(s->xacc); drop(s->rres); drop(s->rrh);
    drop(s->vals_df);
    s->vals_df_cap = 0;
    s->vals_df_valid = false;
    s->rrh_cap = 0;
    drop(s->vpart); drop(s->gpart); drop(s->part); drop(s->tfull); drop(s->sfull);
    s->vpart_P = 0;
    s->vld = 0;
    drop(s->delta); drop(s->eta); drop(s->theta_m); drop(s->theta_m1); drop(s->tsel); drop(s->sel);
    s->eig_cap = 0;
    drop(s->eigwork);
    drop(s->gram_scratch);
    s->gram_cap = 0;
    drop(s->W32); drop(s->AW32); drop(s->Z32);
    s->cap_w32 = 0;
    drop(s->C32); drop(s->AC32); drop(s->dinv);
    s->cap_c32 = 0;
    drop(s->x32); drop(s->r32); drop(s->u32); drop(s->b32); drop(s->minv32);
    drop(s->Pout); drop(s->APout); drop(s->oscal); drop(s->ovpart);
    s->cap_out = 0;
    s->minv32_kind = -1;
    drop(s->vals32);
    s->vals32_cap = 0;
    s->vals32_valid = false;
    s->last_m = 0;
    s->last_ritz_m = 0;
    s->last_srks = 0;
    s->last_nsel = 0;
  }
  if (what & KRS_RELEASE_SPACE) {
    drop(s->C); drop(s->AC); drop(s->G); drop(s->Lw); drop(s->Ginv);
    s->cap_c = 0;
    s->nc = 0;
    s->ac_valid = 0;
    s->g_valid = 0;
    s->ginv_valid = false;
  }
  if (what & KRS_RELEASE_MATRIX) {
    drop(s->rp); drop(s->ci); drop(s->vals);
    s->nnzb_cap = 0;
    s->rp_use = nullptr;
    s->ci_use = nullptr;
    s->vals_use = nullptr;
    s->A_valid = false;
    s->precond_built = -1;
    s->ac_valid = 0;
    s->g_valid = 0;
    s->ginv_valid = false;
    drop(s->vals32);
    s->vals32_cap = 0;
    s->vals32_valid = false;
    drop(s->vals_df);
    s->vals_df_cap = 0;
    s->vals_df_valid = false;
  }
  return KRS_OK;
}

krs_status krs_last_coeffs(krs_seq_t s, double* alpha, double* rho, double* gamma) {
  if (!s) return fail(KRS_ERR_INVALID_ARG, "NULL sequence");
  const int m = s->last_m;
  KRS_CUDA(cudaSetDevice(s->device));
  if (m > 0) {
    if (alpha) KRS_CUDA(cudaMemcpyAsync(alpha, s->alpha, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream));
    if (rho) KRS_CUDA(cudaMemcpyAsync(rho, s->rho, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream));
    if (gamma) KRS_CUDA(cudaMemcpyAsync(gamma, s->gamma, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream));
  }
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  return KRS_OK;
}

krs_status krs_last_ritz(krs_seq_t s, double* theta_m, double* theta_m1, int32_t* sel) {
  if (!s) return fail(KRS_ERR_INVALID_ARG, "NULL sequence");
  const int m = s->last_ritz_m;
  if (!s->last_srks || m < 2) return KRS_OK;
  KRS_CUDA(cudaSetDevice(s->device));
  if (theta_m) KRS_CUDA(cudaMemcpyAsync(theta_m, s->theta_m, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream));
  if (theta_m1)
    KRS_CUDA(cudaMemcpyAsync(theta_m1, s->theta_m1, sizeof(double) * (m - 1), cudaMemcpyDeviceToHost, s->stream));
  if (sel && s->last_nsel > 0)
    KRS_CUDA(cudaMemcpyAsync(sel, s->sel, sizeof(int32_t) * s->last_nsel, cudaMemcpyDeviceToHost, s->stream));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  return KRS_OK;
}

krs_status krs_last_vectors(krs_seq_t s, int32_t which, double* out) {
  if (!s || which < 0 || which > 2) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  const int m = s->last_m;
  if (m == 0) return KRS_OK;
  if (!out) return fail(KRS_ERR_INVALID_ARG, "NULL output");
  KRS_CUDA(cudaSetDevice(s->device));
  const double* src = which == 0 ? s->W : (which == 1 ? s->AW : s->W);
  if (!src || !single_pass(s->last_prec))
    return fail(KRS_ERR_INVALID_ARG, "the last solve stored no FP64 vectors (mixed precision)");
  double* tmp = nullptr;
  double* ud = nullptr;
  const bool df = s->last_prec == KRS_DOUBLE_FLOAT;
  if (which == 2) {  // z_j = w_j + sum_i U[i, j] w_i from the stored coefficients
    KRS_TRY(alloc_n(s, &tmp, (size_t)m * s->ld));
    KRS_TRY(alloc_n(s, &ud, (size_t)m * m));
    KRS_CUDA(launch_z_from_wu(s->n, s->ld, m, s->W, df, s->ucoef, s->last_reorth_full, ud, tmp, s->stream));
    src = tmp;
  } else if (df) {  // double-float pairs -> doubles
    KRS_TRY(alloc_n(s, &tmp, (size_t)m * s->ld));
    KRS_CUDA(launch_df2d(reinterpret_cast<const dfl*>(src), tmp, (int64_t)m * s->ld, s->stream));
    src = tmp;
  }
  const bool dv = is_device_ptr(out);
  cudaError_t e = cudaMemcpy2DAsync(out, sizeof(double) * s->n, src, sizeof(double) * s->ld, sizeof(double) * s->n, m,
                                    dv ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dev_free(s, tmp);
  dev_free(s, ud);
  KRS_CUDA(e);
  return KRS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// the solve
// ------------------------------------------------------------------------------------
krs_status krs::validate_policy(const krs_policy* p) {
  if (!p) return fail(KRS_ERR_INVALID_ARG, "policy is NULL");
  if (p->recycle < 0 || p->recycle > 2) return fail(KRS_ERR_INVALID_ARG, "bad recycle %d", p->recycle);
  if (p->precond < 0 || p->precond > 2) return fail(KRS_ERR_INVALID_ARG, "bad precond %d", p->precond);
  if (p->reorth < 0 || p->reorth > 1) return fail(KRS_ERR_INVALID_ARG, "bad reorth %d", p->reorth);
  if (p->precision != KRS_FP64 && p->precision != KRS_MIXED_IR && p->precision != KRS_MIXED_PROJ &&
      p->precision != KRS_DOUBLE_FLOAT)
    return fail(KRS_ERR_INVALID_ARG, "bad precision %d", p->precision);
  if (!(p->inner_tol == p->inner_tol) || p->inner_tol >= 1.0) return fail(KRS_ERR_INVALID_ARG, "inner_tol must be < 1");
  if (p->cap_mode < 0 || p->cap_mode > 1) return fail(KRS_ERR_INVALID_ARG, "bad cap_mode %d", p->cap_mode);
  if (p->max_aug < 0) return fail(KRS_ERR_INVALID_ARG, "bad max_aug %d", p->max_aug);
  if (p->max_iter < 1 || p->max_iter > 16000) return fail(KRS_ERR_INVALID_ARG, "max_iter %d outside [1, 16000]", p->max_iter);
  if (p->exec < 0 || p->exec > 1) return fail(KRS_ERR_INVALID_ARG, "bad exec %d", p->exec);
  if (!(p->ritz_eps == p->ritz_eps) || !(p->theta_frac == p->theta_frac)) return fail(KRS_ERR_INVALID_ARG, "NaN policy field");
  if (p->reselect < 0 || p->reselect > 1) return fail(KRS_ERR_INVALID_ARG, "bad reselect %d", p->reselect);
  return KRS_OK;
}

static krs_status upload_matrix(krs_seq* s, const krs_bsr* A, bool* changed) {
  *changed = false;
  if (A->block_dim != 3) return fail(KRS_ERR_INVALID_ARG, "block_dim %d != 3", A->block_dim);
  if ((int64_t)A->n_block_rows * 3 != s->n) return fail(KRS_ERR_INVALID_ARG, "matrix order %lld != sequence order %lld",
                                                        (long long)A->n_block_rows * 3, (long long)s->n);
  if (A->nnzb <= 0 || !A->row_ptr || !A->col_idx || !A->values) return fail(KRS_ERR_INVALID_ARG, "empty matrix");
  const bool same = s->A_valid && A->version == s->A_version &&
                    (A->on_device ? (A->values == s->vals_use && A->row_ptr == s->rp_use && A->col_idx == s->ci_use)
                                  : true);
  if (same) return KRS_OK;
  *changed = true;
  // the iteration's product reads block pairs with 16-byte loads: a caller's device matrix
  // is used in place when values are 16-byte and col_idx 8-byte aligned, copied otherwise
  const bool aligned = ((uintptr_t)A->values % 16 == 0) && ((uintptr_t)A->col_idx % 8 == 0);
  if (A->on_device && aligned) {
    s->rp_use = A->row_ptr;
    s->ci_use = A->col_idx;
    s->vals_use = A->values;
  } else {
    if (!A->on_device) KRS_TRY(krs_validate_bsr(A->n_block_rows, A->nnzb, A->row_ptr, A->col_idx));
    if (A->nnzb > s->nnzb_cap) {
      dev_free(s, s->rp);
      dev_free(s, s->ci);
      dev_free(s, s->vals);
      s->rp = nullptr;
      s->ci = nullptr;
      s->vals = nullptr;
      KRS_TRY(alloc_n(s, &s->rp, (size_t)s->nbr + 1));
      KRS_TRY(alloc_n(s, &s->ci, (size_t)A->nnzb));
      KRS_TRY(alloc_n(s, &s->vals, (size_t)A->nnzb * 9));
      s->nnzb_cap = A->nnzb;
    }
    const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    KRS_CUDA(cudaMemcpyAsync(s->rp, A->row_ptr, sizeof(int32_t) * ((size_t)s->nbr + 1), kind, s->stream));
    KRS_CUDA(cudaMemcpyAsync(s->ci, A->col_idx, sizeof(int32_t) * (size_t)A->nnzb, kind, s->stream));
    KRS_CUDA(cudaMemcpyAsync(s->vals, A->values, sizeof(double) * 9 * (size_t)A->nnzb, kind, s->stream));
    s->rp_use = s->rp;
    s->ci_use = s->ci;
    s->vals_use = s->vals;
  }
  s->A_valid = true;
  s->A_version = A->version;
  s->precond_built = -1;
  s->ac_valid = 0;
  s->g_valid = 0;
  s->ginv_valid = false;
  return KRS_OK;
}

static krs_status read_status(krs_seq* s, int* st) {
  KRS_CUDA(cudaMemcpyAsync(s->h_ctrl, s->ctrl, sizeof(int) * CTRL_WORDS, cudaMemcpyDeviceToHost, s->stream));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  *st = s->h_ctrl[CTRL_STATUS];
  return KRS_OK;
}

// FP32 storage of the mixed-precision inner solves (sized like the FP64 state)
static krs_status ensure_mixed(krs_seq* s, int max_iter, int64_t nnzb) {
  if (!s->x32) {
    KRS_TRY(alloc_n(s, &s->x32, s->ld));
    KRS_TRY(alloc_n(s, &s->r32, s->ld));
    KRS_TRY(alloc_n(s, &s->u32, s->ld));
    KRS_TRY(alloc_n(s, &s->b32, s->ld));
    KRS_TRY(alloc_n(s, &s->minv32, 3 * s->ld + 64));
  }
  if (nnzb > s->vals32_cap) {
    dev_free(s, s->vals32);
    s->vals32 = nullptr;
    KRS_TRY(alloc_n(s, &s->vals32, (size_t)nnzb * 9 + 4));
    s->vals32_cap = nnzb;
    s->vals32_valid = false;
  }
  KRS_TRY(ensure_w32(s, max_iter + 1, 0));
  if (s->rrh_cap < s->cap_w32) {
    dev_free(s, s->rrh);
    s->rrh = nullptr;
    KRS_TRY(alloc_n(s, &s->rrh, (size_t)s->cap_w32));
    s->rrh_cap = s->cap_w32;
  }
  // C32 / AC32 hold the FP32 copy of C (every inner solve starts from the recycled space
  // alone, so no room for earlier passes' directions)
  if (s->cap_c > s->cap_c32 || !s->C32) {
    const int cap = s->cap_c > 0 ? s->cap_c : 1;
    dev_free(s, s->C32);
    dev_free(s, s->AC32);
    dev_free(s, s->dinv);
    s->C32 = s->AC32 = nullptr;
    s->dinv = nullptr;
    KRS_TRY(alloc_n(s, &s->C32, (size_t)cap * s->ld));
    KRS_TRY(alloc_n(s, &s->AC32, (size_t)cap * s->ld));
    KRS_TRY(alloc_n(s, &s->dinv, 1));
    s->cap_c32 = cap;
  }
  return KRS_OK;
}

// Storage of the FP32-projection precision: FP32 directions for max_iter iterations (all
// passes of one system), FP32 copies of C and AC followed by room for the earlier passes'
// directions and their diagonal coarse block, the FP64 product q, the residual history of
// the stall test, the pass right-hand side and the accumulated solution.
static krs_status ensure_proj(krs_seq* s, int max_iter) {
  KRS_TRY(ensure_w32(s, max_iter + 1, 0));
  if (s->cap_c + s->cap_w32 > s->cap_c32) {
    const int cap = s->cap_c + s->cap_w32;
    dev_free(s, s->C32);
    dev_free(s, s->AC32);
    dev_free(s, s->dinv);
    s->C32 = s->AC32 = nullptr;
    s->dinv = nullptr;
    KRS_TRY(alloc_n(s, &s->C32, (size_t)cap * s->ld));
    KRS_TRY(alloc_n(s, &s->AC32, (size_t)cap * s->ld));
    KRS_TRY(alloc_n(s, &s->dinv, (size_t)s->cap_w32));
    s->cap_c32 = cap;
  }
  if (s->rrh_cap < s->cap_w32) {
    dev_free(s, s->rrh);
    s->rrh = nullptr;
    KRS_TRY(alloc_n(s, &s->rrh, (size_t)s->cap_w32));
    s->rrh_cap = s->cap_w32;
  }
  if (!s->q64) KRS_TRY(alloc_n(s, &s->q64, s->ld));
  if (!s->xacc) KRS_TRY(alloc_n(s, &s->xacc, s->ld));
  if (!s->rres) KRS_TRY(alloc_n(s, &s->rres, s->ld));
  return KRS_OK;
}

// Init kernels of an APCG solve for the IterArgs `a` with right-hand side b_in (device, a's
// value type), then one read of ||b_in||^2 (*bb) and ||r_0||^2 (*rr0); sets a.tol2.
static krs_status run_init(krs_seq* s, IterArgs& a, const void* b_in, double tol, double* bb, double* rr0,
                           int64_t* launches) {
  KRS_CUDA(apcg_launch_init(a, b_in, s->scal, s->stream, launches));
  KRS_CUDA(cudaMemcpyAsync(s->h_scal, s->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  *bb = s->h_scal[0];
  *rr0 = s->h_scal[1];
  if (!isfinite(*bb)) return fail(KRS_ERR_INVALID_ARG, "right-hand side is not finite");
  a.tol2 = tol * tol * (*bb);
  return KRS_OK;
}

// The iteration loop of an initialised solve (persistent kernel, or per-phase kernels).
// Adds the iteration kernels' event time to *t_iter_ms; the solve's outcome is in *status
// and its iteration count in *m.
static krs_status run_loop(krs_seq* s, IterArgs& a, int exec, int* status, int* m, float* t_iter_ms,
                           int64_t* launches) {
  KRS_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(int) * CTRL_WORDS, s->stream));
  KRS_CUDA(cudaMemsetAsync(s->bar, 0, sizeof(unsigned long long), s->stream));
  KRS_CUDA(cudaEventRecord(s->ev[4], s->stream));
  if (exec == KRS_EXEC_PERSISTENT) {
    KRS_CUDA(apcg_launch_persistent(a, s->stream, launches));
    KRS_CUDA(cudaEventRecord(s->ev[5], s->stream));
    KRS_CUDA(cudaMemcpyAsync(s->h_ctrl, s->ctrl, sizeof(int) * CTRL_WORDS, cudaMemcpyDeviceToHost, s->stream));
    KRS_CUDA(cudaStreamSynchronize(s->stream));
  } else {
    int j = 0;
    const int batch = 16;
    for (;;) {
      const int j1 = (j + batch < a.max_iter) ? j + batch : a.max_iter;
      KRS_CUDA(apcg_launch_phases(a, j, j1, s->stream, launches));
      KRS_CUDA(cudaMemcpyAsync(s->h_ctrl, s->ctrl, sizeof(int) * CTRL_WORDS, cudaMemcpyDeviceToHost, s->stream));
      KRS_CUDA(cudaStreamSynchronize(s->stream));
      j = j1;
      if (s->h_ctrl[CTRL_DONE] || j >= a.max_iter) break;
    }
    KRS_CUDA(cudaEventRecord(s->ev[5], s->stream));
    KRS_CUDA(cudaEventSynchronize(s->ev[5]));
  }
  float dt = 0.f;
  cudaEventElapsedTime(&dt, s->ev[4], s->ev[5]);
  *t_iter_ms += dt;
  *status = s->h_ctrl[CTRL_STATUS];
  *m = s->h_ctrl[CTRL_M];
  if (!s->h_ctrl[CTRL_DONE] && *status == KRS_OK) *status = KRS_ERR_CUDA;
  return KRS_OK;
}

// SRKS, first half: H_m from the coefficients, the eigenvalues of H_m and H_{m-1}, the
// selection; the selected count goes to pinned host memory (h_ctrl[16]), valid once the
// stream has been synchronised.
static krs_status srks_begin(krs_seq* s, int m, int room, const krs_policy* p, int64_t* launches) {
  s->last_srks = 1;
  s->last_ritz_m = m;
  KRS_TRY(ensure_eig(s, m));
  KRS_CUDA(launch_lanczos(m, s->alpha, s->rho, s->delta, s->eta, s->stream));
  // tsel (5m doubles) is free until the selection: scratch of the long-order bisection
  KRS_CUDA(launch_tridiag_eigvals2(m, m - 1, s->delta, s->eta, s->theta_m, s->theta_m1, s->stream, s->tsel));
  KRS_CUDA(launch_srks_select(m, s->theta_m, s->theta_m1, p->ritz_eps, p->theta_frac, p->reselect, room, s->sel,
                              s->selcount, s->tsel, s->stream));
  *launches += 3;
  KRS_CUDA(cudaMemcpyAsync(&s->h_ctrl[16], s->selcount, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  return KRS_OK;
}

// SRKS, second half (after the stream was synchronised): eigenvectors of the selected
// values and the Ritz vectors, written to C[:, nc .. nc + *cnt) (not yet counted in s->nc).
// The z's: Z32 (FP32) when given, else W and the coefficient rows U (z_j = w_j + sum_i
// U[i, j] w_i) -- FP64 W, or double-float pairs when w_df.
static krs_status srks_finish(krs_seq* s, int m, int nc, const float* Z32, int* cnt, int64_t* launches,
                              bool can_grow, bool w_df = false) {
  *cnt = 0;
  const int k = s->h_ctrl[16];
  s->last_nsel = k;
  if (k <= 0) return KRS_OK;
  if (nc + k > s->cap_c) {
    if (!can_grow) return fail(KRS_ERR_INVALID_ARG, "internal: augmentation capacity not reserved");
    KRS_TRY(ensure_cap_c(s, nc + k));  // one APCG solve: nothing else uses C, AC, G^-1 now
  }
  const size_t wneed = eigvecs_work_doubles(m, k) + (size_t)m * k * 3;
  dev_free(s, s->eigwork);
  s->eigwork = nullptr;
  KRS_TRY(alloc_n(s, &s->eigwork, wneed));
  double* Q = s->eigwork;
  double* Fm = s->eigwork + (size_t)m * k;
  double* F2 = s->eigwork + 2 * (size_t)m * k;
  double* wk = s->eigwork + 3 * (size_t)m * k;
  KRS_CUDA(launch_tridiag_eigvecs(m, s->delta, s->eta, k, s->tsel, Q, wk, s->stream));
  if (Z32) {
    KRS_CUDA(launch_ritz_vectors_f(s->n, s->ld, m, k, Z32, s->rho, Q, s->tsel, Fm, s->C + (size_t)nc * s->ld,
                                   s->stream));
    *launches += 3;
  } else {
    KRS_CUDA(launch_ritz_vectors_wu(s->n, s->ld, m, k, s->W, w_df, s->ucoef, s->last_reorth_full, s->rho, Q, s->tsel,
                                    Fm, F2, s->C + (size_t)nc * s->ld, s->stream));
    *launches += 4;
  }
  *cnt = k;
  return KRS_OK;
}

// SRKS extraction (Algorithm 3) from the coefficients of an m-iteration solve and its z's
// (FP64 or FP32): selected Ritz vectors written to C[:, nc .. nc + *cnt) (not yet counted in
// s->nc).  room: how many may be appended.
static krs_status srks_extract(krs_seq* s, int m, int nc, int room, const krs_policy* p, const float* Z32, int* cnt,
                               int64_t* launches, bool can_grow) {
  *cnt = 0;
  KRS_TRY(srks_begin(s, m, room, p, launches));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  return srks_finish(s, m, nc, Z32, cnt, launches, can_grow);
}

__global__ void k_recip(const double* __restrict__ src, double* __restrict__ dst, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = 1.0 / src[i];
}

// t[i] /= gamma[i], i < k (the A-orthogonalisation coefficients of a new outer direction)
__global__ void k_div_elem(double* __restrict__ t, const double* __restrict__ gamma, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) t[i] /= gamma[i];
}

// out = num / den (one thread): the flexible CG step length
__global__ void k_ratio(const double* __restrict__ num, const double* __restrict__ den, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = num[0] / den[0];
}

__global__ void k_f2d_cols(const float* __restrict__ src, double* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

__global__ void k_df2d(const dfl* __restrict__ src, double* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// dst = src as doubles (count double-float pairs; dst may not overlap src)
static cudaError_t launch_df2d(const dfl* src, double* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = (count + 255) / 256;
  k_df2d<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

// Set-up shared by both precisions: matrix, preconditioner, right-hand side, storage,
// partition, coarse set-up (FP64), the FP32 copies (mixed), and the iteration arguments.
// cap_iter: direction columns reserved (FP64 path).
static krs_status seq_setup(krs_seq* s, const krs_bsr* A, const double* b, const krs_policy* p, int cap_iter,
                            SolveState* ss) {
  krs_solve_stats st{};
  st.n_c = s->nc;
  s->st = st;
  s->last_m = 0;
  s->last_ritz_m = 0;
  s->last_srks = 0;
  s->last_nsel = 0;
  int64_t& launches = ss->launches;
  const bool mixed = p->precision == KRS_MIXED_IR;
  const bool proj = p->precision == KRS_MIXED_PROJ;
  const bool dfk = p->precision == KRS_DOUBLE_FLOAT;
  const int prec = prec_id(p->precision);
  s->last_prec = p->precision;
  KRS_CUDA(cudaSetDevice(s->device));
  KRS_CUDA(cudaEventRecord(s->ev[0], s->stream));

  // ---- matrix, preconditioner
  bool changed = false;
  KRS_TRY(upload_matrix(s, A, &changed));
  if (changed) {
    s->vals32_valid = false;
    s->vals_df_valid = false;
  }
  if (s->precond_built != p->precond) {
    KRS_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(int) * CTRL_WORDS, s->stream));
    KRS_CUDA(launch_precond_setup(p->precond, s->nbr, s->rp_use, s->ci_use, s->vals_use, s->minv, s->ctrl + CTRL_STATUS,
                                  s->stream));
    launches++;
    int code = 0;
    KRS_TRY(read_status(s, &code));
    if (code) return fail((krs_status)code, code == KRS_ERR_NOT_SPD ? "preconditioner: a diagonal block is not positive definite"
                                                                    : "preconditioner: missing diagonal block");
    s->precond_built = p->precond;
    s->minv32_kind = -1;
  }

  // ---- right-hand side into the padded device vector
  const bool b_dev = is_device_ptr(b);
  KRS_CUDA(cudaMemcpyAsync(s->b, b, sizeof(double) * s->n, b_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s->stream));

  // ---- storage, augmentation capacity for this solve's recycling step, partition
  const int nc = s->nc;
  ss->nc = nc;
  const int cap = p->max_aug > 0 ? p->max_aug : 0x7fffffff;
  int room = 0;
  if (p->recycle != KRS_RECYCLE_NONE) {
    room = (p->cap_mode == KRS_CAP_TRUNCATE) ? (cap - nc > 0 ? cap - nc : 0) : p->max_iter + 1;
    if (room > p->max_iter + 1) room = p->max_iter + 1;
  }
  ss->room = room;
  // The mixed path appends after its first inner solve while later inner solves still use
  // C, AC and G^-1, so the room is reserved now; the FP64 path grows after its solve.
  if (mixed) {
    KRS_TRY(ensure_cap_c(s, nc + room));
    KRS_TRY(ensure_mixed(s, p->max_iter, A->nnzb));
  } else if (proj) {
    KRS_TRY(ensure_cap_c(s, nc + room));
    KRS_TRY(ensure_proj(s, p->max_iter));
  } else {
    KRS_TRY(ensure_cap_c(s, nc));
    KRS_TRY(ensure_cap_w(s, cap_iter));
    if (dfk) {  // the FP64 copies of w_j and A w_j beside the double-float directions
      if (!s->q64) KRS_TRY(alloc_n(s, &s->q64, s->ld));
      if (!s->wv) KRS_TRY(alloc_n(s, &s->wv, s->ld));
      if (A->nnzb > s->vals_df_cap) {  // double-float matrix values for the operator product
        dev_free(s, s->vals_df);
        s->vals_df = nullptr;
        KRS_TRY(alloc_n(s, &s->vals_df, (size_t)A->nnzb * 9));
        s->vals_df_cap = A->nnzb;
        s->vals_df_valid = false;
      }
      if (!s->vals_df_valid) {
        KRS_CUDA(launch_d2df(s->vals_use, s->vals_df, 9 * A->nnzb, s->stream));
        s->vals_df_valid = true;
        launches++;
      }
    }
  }
  // largest column count a tall-skinny phase sees (mixed: C plus earlier inner directions)
  const int kmax = (mixed || proj) ? nc + p->max_iter + 1 : ((nc > cap_iter + 1) ? nc : cap_iter + 1);
  ss->kmax = kmax;
  KRS_CUDA(apcg_prepare_attributes(kmax, prec));
  int bps = 0;
  KRS_CUDA(apcg_max_coresident(kmax, prec, &bps));
  if (bps < 1) return fail(KRS_ERR_CUDA, "persistent kernel cannot be resident (kmax %d)", kmax);
  ss->bps = bps;
  int P = 0, npc = 0;
  partition(s, bps, &P, &npc);
  KRS_TRY(ensure_vpart(s, P, kmax));

  // ---- coarse set-up (FP64): A C (new columns), C^T A C (new tiles), Cholesky and inverse
  if (nc > 0) {
    if (s->ac_valid < nc) {
      KRS_CUDA(launch_spmm(s->nbr, s->rp_use, s->ci_use, s->vals_use, s->C, s->AC, s->ld, s->ac_valid, nc, s->stream));
      launches++;
      if (s->g_valid > s->ac_valid) s->g_valid = s->ac_valid;
      s->ac_valid = nc;
    }
    if (s->g_valid < nc) {
      const size_t need = gram_scratch_doubles(s->n, nc, s->g_valid);
      if (need > s->gram_cap) {
        dev_free(s, s->gram_scratch);
        s->gram_scratch = nullptr;
        KRS_TRY(alloc_n(s, &s->gram_scratch, need));
        s->gram_cap = need;
      }
      KRS_CUDA(launch_gram(s->n, s->C, s->AC, s->ld, nc, s->g_valid, s->G, s->cap_c, s->gram_scratch, s->gram_cap,
                           s->stream));
      launches += 2;
      s->g_valid = nc;
      s->ginv_valid = false;
    }
    if (!s->ginv_valid) {
      KRS_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(int) * CTRL_WORDS, s->stream));
      KRS_CUDA(launch_chol_inverse(nc, s->G, s->cap_c, s->Lw, s->Ginv, s->ctrl + CTRL_STATUS, s->stream));
      launches += 2;
      int code = 0;
      KRS_TRY(read_status(s, &code));
      if (code) {
        s->st.status = code;
        return fail((krs_status)code, "Cholesky of C^T A C failed (C rank deficient or A not SPD)");
      }
      s->ginv_valid = true;
    }
  }

  // ---- FP32 copies of C and AC for the projection
  if (proj && nc > 0) {
    KRS_CUDA(launch_d2f(s->C, s->C32, (int64_t)nc * s->ld, s->stream));
    KRS_CUDA(launch_d2f(s->AC, s->AC32, (int64_t)nc * s->ld, s->stream));
    launches += 2;
  }

  // ---- FP32 copies for the inner solves
  if (mixed) {
    if (!s->vals32_valid) {
      KRS_CUDA(launch_d2f(s->vals_use, s->vals32, 9 * A->nnzb, s->stream));
      s->vals32_valid = true;
      launches++;
    }
    if (s->minv32_kind != p->precond) {
      KRS_CUDA(launch_d2f(s->minv, s->minv32, (p->precond == KRS_PRECOND_BLOCK_JACOBI3) ? 9 * (int64_t)s->nbr : s->n,
                          s->stream));
      s->minv32_kind = p->precond;
      launches++;
    }
    if (nc > 0) {
      KRS_CUDA(launch_d2f(s->C, s->C32, (int64_t)nc * s->ld, s->stream));
      KRS_CUDA(launch_d2f(s->AC, s->AC32, (int64_t)nc * s->ld, s->stream));
      launches += 2;
    }
  }

  IterArgs& a = ss->a;
  a = IterArgs{};
  a.n = s->n; a.ld = s->ld; a.nbr = s->nbr; a.npc = npc; a.P = P;
  a.nc = nc; a.nc_dense = nc; a.dinv = s->dinv;
  a.ldg = s->cap_c; a.max_iter = p->max_iter; a.reorth_full = (p->reorth == KRS_REORTH_FULL);
  a.precond = p->precond; a.kmax = kmax; a.spin_limit = s->spin_limit; a.prec = prec;
  a.rp = s->rp_use; a.ci = s->ci_use; a.Ginv = s->Ginv;
  a.alpha = s->alpha; a.gamma = s->gamma; a.rho = s->rho;
  a.tfull = s->tfull; a.sfull = s->sfull; a.gfull = s->gfull;
  a.part = s->part; a.vpart = s->vpart; a.gpart = s->gpart; a.vld = s->vld; a.ctrl = s->ctrl; a.bar = s->bar;
  if (mixed) {
    a.vals = s->vals32; a.minv = s->minv32; a.C = s->C32; a.AC = s->AC32;
    a.W = s->W32; a.AW = s->AW32; a.Z = s->Z32; a.zld = s->ld; a.x = s->x32; a.r = s->r32; a.u = s->u32;
    a.stall_win = 32; a.rrh = s->rrh;
  } else if (proj) {
    a.vals = s->vals_use; a.minv = s->minv; a.C = s->C32; a.AC = s->AC32; a.Ci = s->C; a.ACi = s->AC;
    a.W = s->W32; a.AW = s->AW32; a.Z = s->Z32; a.zld = s->ld; a.x = s->x; a.r = s->r; a.u = s->u; a.q = s->q64;
    a.stall_win = 32; a.rrh = s->rrh;
  } else {
    // KRS_DOUBLE_FLOAT: W, AW, z hold double-float pairs (8 bytes, like the FP64 directions);
    // one z column, the coefficient rows U instead of the stored z_j
    a.vals = s->vals_use; a.minv = s->minv; a.C = s->C; a.AC = s->AC;
    a.W = s->W; a.AW = s->AW; a.Z = s->Z; a.zld = 0; a.ucoef = s->ucoef; a.x = s->x; a.r = s->r; a.u = s->u;
    s->last_reorth_full = (p->reorth == KRS_REORTH_FULL);
    if (dfk) {
      a.q = s->q64;
      a.wv = s->wv;
      a.vals_df = s->vals_df;
    }
  }
  KRS_CUDA(cudaEventRecord(s->ev[1], s->stream));
  return KRS_OK;
}

krs_status krs::seq_begin(krs_seq* s, const krs_bsr* A, const double* b, double tol, const krs_policy* p,
                          int cap_iter, SolveState* ss) {
  if (!single_pass(p->precision)) return fail(KRS_ERR_INVALID_ARG, "internal: seq_begin is the single-pass path");
  ss->tol = tol;
  KRS_TRY(seq_setup(s, A, b, p, cap_iter, ss));
  KRS_TRY(run_init(s, ss->a, s->b, tol, &ss->bb, &ss->rr0, &ss->launches));
  ss->need_iter = ss->rr0 > ss->a.tol2;
  return KRS_OK;
}

krs_status krs::seq_grow_directions(krs_seq* s, int cap_iter, int keep, int prec) {
  const int need = cap_iter + 1;
  if (prec == KRS_MIXED_PROJ) return ensure_w32(s, need, keep);
  KRS_TRY(ensure_scalars(s, need, keep));
  if (!s->Z) KRS_TRY(alloc_n(s, &s->Z, (size_t)s->ld));
  if (need <= s->cap_w) return KRS_OK;
  const int cap = (int)round_up(need, 32);
  double *W = nullptr, *AW = nullptr, *U = nullptr;
  KRS_TRY(alloc_n(s, &W, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &AW, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &U, ucoef_entries(cap)));
  if (keep > s->cap_w) keep = s->cap_w;
  if (keep > 0) {
    const size_t vb = sizeof(double) * (size_t)keep * s->ld;
    KRS_CUDA(cudaMemcpyAsync(W, s->W, vb, cudaMemcpyDeviceToDevice, s->stream));
    KRS_CUDA(cudaMemcpyAsync(AW, s->AW, vb, cudaMemcpyDeviceToDevice, s->stream));
    if (keep > 1)  // coefficient rows 1 .. keep - 1
      KRS_CUDA(cudaMemcpyAsync(U, s->ucoef, sizeof(double) * ucoef_entries(keep), cudaMemcpyDeviceToDevice,
                               s->stream));
  }
  dev_free(s, s->W);
  dev_free(s, s->AW);
  dev_free(s, s->ucoef);
  s->W = W; s->AW = AW; s->ucoef = U;
  s->cap_w = cap;
  return KRS_OK;
}

krs_status krs::seq_end_stage(krs_seq* s, SolveState* ss, int status, int m, double* x, const krs_policy* p,
                              int stage) {
  // both refinement precisions did their recycling step inside the refinement loop
  const bool mixed = p->precision == KRS_MIXED_IR || p->precision == KRS_MIXED_PROJ;
  const int nc = ss->nc;
  int64_t& launches = ss->launches;
  const bool srks = !mixed && status == KRS_OK && p->recycle == KRS_RECYCLE_SRKS && m >= 2;
  if (stage == 1) {
    if (!mixed) {
      s->last_m = m;
      KRS_CUDA(cudaEventRecord(s->ev[2], s->stream));
      ss->add = 0;
      if (srks) KRS_TRY(srks_begin(s, m, ss->room, p, &launches));
    }
    return KRS_OK;
  }
  if (stage == 2) {
    if (!mixed && status == KRS_OK) {
      // ---- FP64: the recycling step on this solve's W (and its coefficient rows U)
      const bool dfk = p->precision == KRS_DOUBLE_FLOAT;  // W, AW hold double-float pairs
      if (p->recycle == KRS_RECYCLE_TRKS && m > 0) {
        const int add = m < ss->room ? m : ss->room;
        if (add > 0) {
          KRS_TRY(ensure_cap_c(s, nc + add));
          if (dfk) {
            KRS_CUDA(launch_df2d(reinterpret_cast<const dfl*>(s->W), s->C + (size_t)nc * s->ld, (int64_t)add * s->ld,
                                 s->stream));
            launches++;
          } else {
            KRS_CUDA(cudaMemcpyAsync(s->C + (size_t)nc * s->ld, s->W, sizeof(double) * (size_t)add * s->ld,
                                     cudaMemcpyDeviceToDevice, s->stream));
          }
          if (s->ac_valid == nc) {
            // A is unchanged since the directions' products were formed: A W is A C's new block
            if (dfk) {
              KRS_CUDA(launch_df2d(reinterpret_cast<const dfl*>(s->AW), s->AC + (size_t)nc * s->ld,
                                   (int64_t)add * s->ld, s->stream));
              launches++;
            } else {
              KRS_CUDA(cudaMemcpyAsync(s->AC + (size_t)nc * s->ld, s->AW, sizeof(double) * (size_t)add * s->ld,
                                       cudaMemcpyDeviceToDevice, s->stream));
            }
            s->ac_valid = nc + add;
          }
        }
        ss->add = add;
      } else if (srks) {
        KRS_TRY(srks_finish(s, m, nc, nullptr, &ss->add, &launches, true, dfk));
      }
    }
    // ---- result and true residual
    const bool x_dev = is_device_ptr(x);
    KRS_CUDA(cudaMemcpyAsync(x, s->x, sizeof(double) * s->n, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             s->stream));
    KRS_CUDA(launch_true_residual(s->nbr, s->rp_use, s->ci_use, s->vals_use, s->x, s->b, s->tmp, s->part, s->scal + 2,
                                  s->stream));
    launches += 3;
    if (!mixed) {
      KRS_CUDA(launch_norm2(s->n, s->r, s->part, s->scal + 3, s->stream));
      launches += 2;
    }
    KRS_CUDA(cudaMemcpyAsync(s->h_scal, s->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    return KRS_OK;
  }
  // stage 3 (the stream has been synchronised): statistics and the commit
  krs_solve_stats st{};
  const int add = ss->add;
  const double bb = ss->bb;
  st.status = status;
  st.m = m;
  st.n_c = nc;
  st.outer_iters = ss->outer;
  st.inner_m_first = ss->m_first;
  st.inner_m2 = single_pass(p->precision) ? (double)st.m * (double)st.m : ss->m2;
  st.true_rel_res = bb > 0.0 ? sqrt(s->h_scal[2] / bb) : 0.0;
  st.rel_res = mixed ? st.true_rel_res : (bb > 0.0 ? sqrt(s->h_scal[3] / bb) : 0.0);
  if (status != KRS_OK) {
    st.n_c_after = nc;
    float t1 = 0.f, t3 = 0.f;
    cudaEventElapsedTime(&t1, s->ev[0], s->ev[1]);
    cudaEventElapsedTime(&t3, s->ev[0], s->ev[2]);
    st.t_setup_ms = t1;
    st.t_iter_ms = ss->t_iter;
    st.t_total_ms = t3;
    st.kernel_launches = launches;
    s->st = st;
    const char* what = status == KRS_ERR_NOT_SPD ? "operator not SPD ((w, Aw) <= 0 or (r, z) <= 0)"
                       : status == KRS_ERR_NO_CONVERGENCE ? "max_iter / max_outer reached or refinement stagnated"
                       : status == KRS_ERR_TIMEOUT ? "device wait timed out"
                                                  : "solve did not complete";
    return fail((krs_status)status, "%s (m = %d)", what, m);
  }
  // ---- commit the recycled columns
  s->nc = nc + add;
  if (p->cap_mode == KRS_CAP_RESTART && p->max_aug > 0 && s->nc >= p->max_aug) {
    // Algorithm 3, last step: back to C^(0)
    if (s->nc0 > 0)
      KRS_CUDA(cudaMemcpyAsync(s->C, s->C0, sizeof(double) * (size_t)s->nc0 * s->ld, cudaMemcpyDeviceToDevice, s->stream));
    s->nc = s->nc0;
    s->ac_valid = 0;
    s->g_valid = 0;
    s->ginv_valid = false;
  }
  KRS_CUDA(cudaEventRecord(s->ev[3], s->stream));
  KRS_CUDA(cudaEventSynchronize(s->ev[3]));
  float t1 = 0.f, t3 = 0.f, tt = 0.f;
  cudaEventElapsedTime(&t1, s->ev[0], s->ev[1]);
  cudaEventElapsedTime(&t3, s->ev[2], s->ev[3]);
  cudaEventElapsedTime(&tt, s->ev[0], s->ev[3]);
  st.n_selected = add;
  st.n_c_after = s->nc;
  st.t_setup_ms = t1;
  st.t_iter_ms = ss->t_iter;
  st.t_recycle_ms = t3;
  st.t_total_ms = tt;
  st.kernel_launches = launches;
  s->st = st;
  return KRS_OK;
}

krs_status krs::seq_end(krs_seq* s, SolveState* ss, int status, int m, double* x, const krs_policy* p) {
  KRS_TRY(seq_end_stage(s, ss, status, m, x, p, 1));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  KRS_TRY(seq_end_stage(s, ss, status, m, x, p, 2));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  return seq_end_stage(s, ss, status, m, x, p, 3);
}

// ------------------------------------------------------------------------------------
// refinement: FP64 outer residual around inner APCG passes (KRS_MIXED_IR: FP32 passes on
// r32 with x accumulated in s->x; KRS_MIXED_PROJ: FP32-projection passes on the FP64
// residual rres, each pass's correction in s->x and their sum in s->xacc)
// ------------------------------------------------------------------------------------
krs_status krs::refine_setup(krs_seq* s, const krs_bsr* A, const double* b, const krs_policy* p, SolveState* ss) {
  return seq_setup(s, A, b, p, p->max_iter, ss);
}

// storage of the flexible CG over the refinement passes (KRS_MIXED_IR): cap outer directions
static krs_status ensure_outer(krs_seq* s, int cap) {
  if (cap <= s->cap_out) return KRS_OK;
  dev_free(s, s->Pout);
  dev_free(s, s->APout);
  dev_free(s, s->oscal);
  dev_free(s, s->ovpart);
  s->Pout = s->APout = s->oscal = s->ovpart = nullptr;
  s->cap_out = 0;
  KRS_TRY(alloc_n(s, &s->Pout, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &s->APout, (size_t)cap * s->ld));
  KRS_TRY(alloc_n(s, &s->oscal, (size_t)2 * cap + 8));
  KRS_TRY(alloc_n(s, &s->ovpart, (size_t)256 * (cap + 2)));
  // rows n .. ld - 1 of the directions stay zero (the tall-skinny kernels read them)
  KRS_CUDA(cudaMemsetAsync(s->Pout, 0, sizeof(double) * (size_t)cap * s->ld, s->stream));
  KRS_CUDA(cudaMemsetAsync(s->APout, 0, sizeof(double) * (size_t)cap * s->ld, s->stream));
  s->cap_out = cap;
  return KRS_OK;
}

// One outer step of the flexible CG over the refinement passes (KRS_MIXED_IR), all FP64:
// p_k = d - sum_{i<k} ((A p_i, d) / (p_i, A p_i)) p_i with d the pass's FP32 correction,
// gamma_k = (p_k, A p_k), alpha = (p_k, r) / gamma_k, x += alpha p_k.  Iterative refinement
// takes x += d; choosing the step and removing the components along the earlier
// corrections makes every step minimise the A-norm of the error over all corrections so
// far, so an inexact FP32 correction cannot make the refinement stall or diverge.
static krs_status fcg_step(krs_seq* s, int k, double* x, double* r, int64_t* launches) {
  const int64_t ld = s->ld, n = s->n;
  double* pk = s->Pout + (size_t)k * ld;
  double* apk = s->APout + (size_t)k * ld;
  double* gam = s->oscal;
  double* t = s->oscal + s->cap_out;
  double* sc = s->oscal + 2 * s->cap_out;  // [0] (p, r), [1] alpha, [2] scratch
  k_f2d_cols<<<1216, 256, 0, s->stream>>>(s->x32, pk, n);
  KRS_CUDA(cudaGetLastError());
  int P = 0;
  int64_t rpc = 0;
  KRS_CUDA(gemv_rows_partition(n, &P, &rpc));
  if (k > 0) {
    KRS_CUDA(launch_gemv_t_rows(n, k, s->APout, ld, pk, t, s->ovpart, P, rpc, s->stream));
    k_div_elem<<<(k + 255) / 256, 256, 0, s->stream>>>(t, gam, k);
    KRS_CUDA(cudaGetLastError());
    KRS_CUDA(launch_gemv_n_rows(n, k, s->Pout, ld, t, pk, pk, P, rpc, s->stream));
    *launches += 4;
  }
  KRS_CUDA(launch_spmv(s->nbr, s->rp_use, s->ci_use, s->vals_use, pk, apk, s->stream));
  KRS_CUDA(launch_gemv_t_rows(n, 1, apk, ld, pk, gam + k, s->ovpart, P, rpc, s->stream));
  KRS_CUDA(launch_gemv_t_rows(n, 1, r, ld, pk, sc, s->ovpart, P, rpc, s->stream));
  k_ratio<<<1, 32, 0, s->stream>>>(sc, gam + k, sc + 1);
  KRS_CUDA(cudaGetLastError());
  // x += alpha p_k (the r update of this kernel is overwritten by the FP64 residual after)
  KRS_CUDA(launch_axpy2_dot(n, sc + 1, pk, apk, x, r, sc + 2, s->ovpart, s->stream));
  *launches += 10;
  return KRS_OK;
}

krs_status krs::refine_start(krs_seq* s, const krs_policy* p, double tol, SolveState* ss) {
  const bool pp = p->precision == KRS_MIXED_PROJ;
  double* xtot = pp ? s->xacc : s->x;
  double* rout = pp ? s->rres : s->r;
  float* r32out = pp ? nullptr : s->b32;
  ss->tol = tol;
  ss->first = true;
  ss->status = KRS_OK;
  ss->m = 0;
  ss->outer = 0;
  ss->m_first = 0;
  ss->add = 0;
  ss->stall = 0;
  ss->m2 = 0.0;
  if (!pp) KRS_TRY(ensure_outer(s, p->max_outer > 0 ? p->max_outer : 30));
  KRS_CUDA(cudaMemsetAsync(xtot, 0, sizeof(double) * s->ld, s->stream));
  // r = b - A*0 = b (FP64), r32 = (float) b, rr = ||b||^2
  KRS_CUDA(launch_resid_update(s->nbr, s->rp_use, s->ci_use, s->vals_use, xtot, s->b, s->tmp, rout, r32out,
                               s->part, s->scal + 4, s->stream));
  ss->launches += 3;
  KRS_CUDA(cudaMemcpyAsync(s->h_scal + 4, s->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  ss->bb = s->h_scal[4];
  ss->rr = ss->bb;
  ss->rr_best = ss->bb;
  if (!isfinite(ss->bb)) return fail(KRS_ERR_INVALID_ARG, "right-hand side is not finite");
  return KRS_OK;
}

krs_status krs::refine_pass_begin(krs_seq* s, const krs_policy* p, double tol, SolveState* ss, bool* need_loop,
                                  bool* finished) {
  const bool pp = p->precision == KRS_MIXED_PROJ;
  const void* rhs_in = pp ? (const void*)s->rres : (const void*)s->b32;
  const double inner_tol = pp ? 0.0 : (p->inner_tol > 0.0 ? p->inner_tol : 0.1);
  const int max_outer = p->max_outer > 0 ? p->max_outer : 30;
  IterArgs& a = ss->a;
  *need_loop = false;
  *finished = false;
  const double bb = ss->bb;
  if (ss->rr <= tol * tol * bb) {
    *finished = true;
    return KRS_OK;
  }
  if (ss->outer >= max_outer || ss->m >= p->max_iter) {
    ss->status = KRS_ERR_NO_CONVERGENCE;
    *finished = true;
    return KRS_OK;
  }
  // the first pass aims at inner_tol (its Krylov space feeds the recycling step: a longer
  // first pass gives SRKS converged Ritz vectors), later passes at max(inner_tol, 0.1); none
  // aims lower than the outer tolerance still needs
  const double pass_tol = (pp || ss->first) ? inner_tol : (inner_tol > 0.1 ? inner_tol : 0.1);
  double tin = 0.5 * tol * sqrt(bb / ss->rr);
  if (tin < pass_tol) tin = pass_tol;
  if (tin > 0.5) tin = 0.5;
  a.max_iter = p->max_iter - ss->m;
  // KRS_MIXED_IR: a later pass (same operator, new right-hand side) gets at most twice the
  // first pass's iterations; one that stagnates above its target ends there and the flexible
  // CG uses its partial correction
  if (!pp && !ss->first && a.max_iter > 2 * ss->m_first + 100) a.max_iter = 2 * ss->m_first + 100;
  double bb_in = 0.0, rr0 = 0.0;
  KRS_TRY(run_init(s, a, rhs_in, tin, &bb_in, &rr0, &ss->launches));
  // the stall test watches only the last stretch: below 1e-3 of the pass's first residual
  a.stall_rr = 1e-6 * rr0;
  *need_loop = rr0 > a.tol2;
  return KRS_OK;
}

krs_status krs::refine_pass_end(krs_seq* s, const krs_policy* p, double tol, SolveState* ss, int st_in, int m_in,
                                bool* finished) {
  const bool pp = p->precision == KRS_MIXED_PROJ;
  double* xtot = pp ? s->xacc : s->x;
  double* rout = pp ? s->rres : s->r;
  float* r32out = pp ? nullptr : s->b32;
  IterArgs& a = ss->a;
  const int nc = ss->nc;
  const int room = ss->room;
  int64_t& launches = ss->launches;
  *finished = false;
  // An FP32 breakdown ((w, Aw) <= 0 or (r, z) <= 0) after some progress, or a stalled
  // residual, only ends this pass: its iterate and directions up to there are valid, and
  // the FP64 outer residual decides whether refinement still advances.
  if (st_in == KRS_STALLED) st_in = KRS_OK;
  if (st_in != KRS_OK && st_in != KRS_ERR_NO_CONVERGENCE && !(st_in == KRS_ERR_NOT_SPD && m_in > 0)) {
    ss->status = st_in;
    *finished = true;
    return KRS_OK;
  }
  ss->m += m_in;
  ss->m2 += (double)m_in * (double)m_in;
  s->last_m = m_in;
  if (ss->first) {
    ss->m_first = m_in;
    // recycling from the first inner solve (staged beyond nc until the system converges)
    if (p->recycle == KRS_RECYCLE_TRKS && m_in > 0) {
      const int add = m_in < room ? m_in : room;
      if (add > 0) {
        k_f2d_cols<<<1216, 256, 0, s->stream>>>(s->W32, s->C + (size_t)nc * s->ld, (int64_t)add * s->ld);
        KRS_CUDA(cudaGetLastError());
        launches++;
      }
      ss->add = add;
    } else if (p->recycle == KRS_RECYCLE_SRKS && m_in >= 2) {
      KRS_TRY(srks_extract(s, m_in, nc, room, p, s->Z32, &ss->add, &launches, false));
    }
    ss->first = false;
  }
  // KRS_MIXED_PROJ: the next inner solve (same operator) is augmented by this one's
  // directions: they are A-conjugate to C and to each other, so their coarse block is
  // diag(1/(w, Aw)).  KRS_MIXED_IR does not: FP32 directions are A-conjugate only to about
  // u_32 kappa, and with hundreds of them the assumed-diagonal coarse block stops being a
  // projector (later passes stagnated on the stiff-inclusion cubes); its passes start from
  // the recycled space alone and the FP64 flexible CG combines their corrections.
  if (m_in > 0 && pp) {
    const int nct = a.nc;
    KRS_CUDA(cudaMemcpyAsync(s->C32 + (size_t)nct * s->ld, s->W32, sizeof(float) * (size_t)m_in * s->ld,
                             cudaMemcpyDeviceToDevice, s->stream));
    KRS_CUDA(cudaMemcpyAsync(s->AC32 + (size_t)nct * s->ld, s->AW32, sizeof(float) * (size_t)m_in * s->ld,
                             cudaMemcpyDeviceToDevice, s->stream));
    k_recip<<<(m_in + 255) / 256, 256, 0, s->stream>>>(s->gamma, s->dinv + (nct - nc), m_in);
    KRS_CUDA(cudaGetLastError());
    launches++;
    a.nc = nct + m_in;
    if (pp) {  // the earlier passes' directions exist in FP32 only: later inits read C32, AC32
      a.init32 = true;
      a.Ci = nullptr;
      a.ACi = nullptr;
    }
  }
  // KRS_MIXED_PROJ: x += d; KRS_MIXED_IR: the flexible CG step over the FP32 corrections
  // (FP64); then r = b - A x (FP64) and the next pass's right-hand side (r32 = (float) r)
  if (pp) KRS_CUDA(launch_add_d(xtot, s->x, s->n, s->stream));
  else KRS_TRY(fcg_step(s, ss->outer, xtot, rout, &launches));
  KRS_CUDA(launch_resid_update(s->nbr, s->rp_use, s->ci_use, s->vals_use, xtot, s->b, s->tmp, rout, r32out,
                               s->part, s->scal + 4, s->stream));
  launches += 4;
  KRS_CUDA(cudaMemcpyAsync(s->h_scal + 4, s->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  KRS_CUDA(cudaStreamSynchronize(s->stream));
  const double rr_new = s->h_scal[4];
  ss->outer++;
  const double bb = ss->bb;
  if (!(rr_new <= tol * tol * bb)) {
    bool stalled;
    if (pp) {
      stalled = !(rr_new < 0.81 * ss->rr);  // one step without a 10 % fall
    } else {
      // the flexible CG minimises the A-norm of the error, not ||r||: three steps in a row
      // without a new 10 % low of ||r|| end it
      if (rr_new < 0.81 * ss->rr_best) {
        ss->rr_best = rr_new;
        ss->stall = 0;
      } else {
        ss->stall++;
      }
      stalled = ss->stall >= 3 || !isfinite(rr_new);
    }
    if (stalled) {  // stagnation: refinement no longer pays
      ss->rr = rr_new;
      ss->status = KRS_ERR_NO_CONVERGENCE;
      *finished = true;
      return KRS_OK;
    }
  }
  ss->rr = rr_new;
  return KRS_OK;
}

krs_status krs::refine_finish(krs_seq* s, const krs_policy* p, SolveState* ss) {
  if (p->precision == KRS_MIXED_PROJ)  // the result and the true residual are taken from s->x
    KRS_CUDA(cudaMemcpyAsync(s->x, s->xacc, sizeof(double) * s->ld, cudaMemcpyDeviceToDevice, s->stream));
  KRS_CUDA(cudaEventRecord(s->ev[2], s->stream));
  return KRS_OK;
}

// the whole refinement loop of one system (krs_solve)
static krs_status mixed_refine(krs_seq* s, const krs_policy* p, double tol, SolveState* ss, int* status_out,
                               int* m_out) {
  KRS_TRY(refine_start(s, p, tol, ss));
  for (;;) {
    bool need_loop = false, finished = false;
    KRS_TRY(refine_pass_begin(s, p, tol, ss, &need_loop, &finished));
    if (finished) break;
    int st_in = KRS_OK, m_in = 0;
    if (need_loop) KRS_TRY(run_loop(s, ss->a, p->exec, &st_in, &m_in, &ss->t_iter, &ss->launches));
    KRS_TRY(refine_pass_end(s, p, tol, ss, st_in, m_in, &finished));
    if (finished) break;
  }
  KRS_TRY(refine_finish(s, p, ss));
  *status_out = ss->status;
  *m_out = ss->m;
  return KRS_OK;
}

static krs_status solve_impl(krs_seq* s, const krs_bsr* A, const double* b, double* x, double tol,
                             const krs_policy* p) {
  SolveState ss;
  ss.tol = tol;
  int status = KRS_OK, m = 0;
  if (p->precision == KRS_MIXED_IR || p->precision == KRS_MIXED_PROJ) {
    KRS_TRY(seq_setup(s, A, b, p, p->max_iter, &ss));
    KRS_TRY(mixed_refine(s, p, tol, &ss, &status, &m));
  } else {
    KRS_TRY(seq_begin(s, A, b, tol, p, p->max_iter, &ss));
    if (ss.need_iter) KRS_TRY(run_loop(s, ss.a, p->exec, &status, &m, &ss.t_iter, &ss.launches));
  }
  return seq_end(s, &ss, status, m, x, p);
}

extern "C" krs_status krs_solve(krs_seq_t s, const krs_bsr* A, const double* b, double* x, double tol,
                                const krs_policy* p) {
  if (!s || !A || !b || !x) return fail(KRS_ERR_INVALID_ARG, "NULL argument");
  if (s->busy) return fail(KRS_ERR_INVALID_ARG, "the sequence has a batched solve in flight");
  if (!(tol >= 0.0) || !isfinite(tol)) return fail(KRS_ERR_INVALID_ARG, "tol must be finite and >= 0");
  KRS_TRY(validate_policy(p));
  krs_status st = solve_impl(s, A, b, x, tol, p);
  if (st != KRS_OK && s->st.status == 0) s->st.status = st;
  return st;
}

// ------------------------------------------------------------------------------------
// single-kernel entry points
// ------------------------------------------------------------------------------------
extern "C" {

krs_status krs_spmv_bsr3(int32_t nbr, const int32_t* rp, const int32_t* ci, const double* vals, const double* x,
                         double* y, void* stream) {
  if (nbr < 0 || (nbr > 0 && (!rp || !ci || !vals || !x || !y))) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  KRS_CUDA(launch_spmv(nbr, rp, ci, vals, x, y, (cudaStream_t)stream));
  return KRS_OK;
}

krs_status krs_precond_setup(int32_t kind, int32_t nbr, const int32_t* rp, const int32_t* ci, const double* vals,
                             double* minv, int32_t* status, void* stream) {
  if (kind < 0 || kind > 2 || nbr < 0 || (nbr > 0 && (!rp || !ci || !vals || (kind != 2 && !minv))))
    return fail(KRS_ERR_INVALID_ARG, "bad argument");
  KRS_CUDA(launch_precond_setup(kind, nbr, rp, ci, vals, minv, status, (cudaStream_t)stream));
  return KRS_OK;
}

krs_status krs_precond_apply(int32_t kind, int32_t nbr, const double* minv, const double* r, double* u, void* stream) {
  if (kind < 0 || kind > 2 || nbr < 0 || (nbr > 0 && (!r || !u || (kind != 2 && !minv))))
    return fail(KRS_ERR_INVALID_ARG, "bad argument");
  KRS_CUDA(launch_precond_apply(kind, nbr, minv, r, u, (cudaStream_t)stream));
  return KRS_OK;
}

static krs_status check_tall(int64_t n, int32_t k, const double* V, int64_t ldv, const void* u) {
  if (n < 0 || k < 0 || (k > 0 && n > 0 && (!V || !u))) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  if (ldv % 4 != 0 || ldv < round_up(n, 4)) return fail(KRS_ERR_INVALID_ARG, "ldv must be a multiple of 4 and >= n rounded up to 4");
  if (((uintptr_t)V & 31) || ((uintptr_t)u & 31)) return fail(KRS_ERR_INVALID_ARG, "V and u must be 32-byte aligned");
  if (k > 16384) return fail(KRS_ERR_INVALID_ARG, "k > 16384");
  return KRS_OK;
}

// rows per CTA of the stand-alone tall-skinny launches
static krs_status tall_partition(int64_t n, int* P, int64_t* rpc) {
  KRS_CUDA(gemv_rows_partition(n, P, rpc));
  return KRS_OK;
}

krs_status krs_gemv_t(int64_t n, int32_t k, const double* V, int64_t ldv, const double* u, double* t, void* stream) {
  KRS_TRY(check_tall(n, k, V, ldv, u));
  if (k == 0) return KRS_OK;
  if (!t) return fail(KRS_ERR_INVALID_ARG, "t is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int P = 0;
  int64_t rpc = 0;
  KRS_TRY(tall_partition(n, &P, &rpc));
  double* vpart = nullptr;
  KRS_CUDA(cudaMallocAsync((void**)&vpart, sizeof(double) * (size_t)(P > 0 ? P : 1) * k, st));
  KRS_CUDA(launch_gemv_t_rows(n, k, V, ldv, u, t, vpart, P, rpc, st));
  KRS_CUDA(cudaFreeAsync(vpart, st));
  return KRS_OK;
}

krs_status krs_gemv_n_sub(int64_t n, int32_t k, const double* V, int64_t ldv, const double* s, const double* u,
                          double* z, void* stream) {
  KRS_TRY(check_tall(n, k, V, ldv, u));
  if (n == 0) return KRS_OK;
  if (!z || (k > 0 && !s)) return fail(KRS_ERR_INVALID_ARG, "NULL argument");
  int P = 0;
  int64_t rpc = 0;
  KRS_TRY(tall_partition(n, &P, &rpc));
  KRS_CUDA(launch_gemv_n_rows(n, k, V, ldv, s, u, z, P, rpc, (cudaStream_t)stream));
  return KRS_OK;
}

krs_status krs_axpy2_dot(int64_t n, const double* alpha, const double* w, const double* q, double* x, double* r,
                         double* rr, void* stream) {
  if (n < 0 || !alpha || !rr || (n > 0 && (!w || !q || !x || !r))) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* part = nullptr;
  KRS_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * 256, st));
  KRS_CUDA(launch_axpy2_dot(n, alpha, w, q, x, r, rr, part, st));
  KRS_CUDA(cudaFreeAsync(part, st));
  return KRS_OK;
}

krs_status krs_tridiag_eigvals(int32_t m, const double* delta, const double* eta, double* theta, void* stream) {
  if (m < 0 || (m > 0 && (!delta || !theta || (m > 1 && !eta)))) return fail(KRS_ERR_INVALID_ARG, "bad argument");
  if (m > 16001) return fail(KRS_ERR_INVALID_ARG, "m > 16001");
  cudaStream_t st = (cudaStream_t)stream;
  double* e2 = nullptr;  // scratch of the long-order path (squared off-diagonal)
  if (m > 1) KRS_CUDA(cudaMallocAsync((void**)&e2, sizeof(double) * (size_t)m, st));
  const cudaError_t e = launch_tridiag_eigvals2(m, 0, delta, eta, theta, nullptr, st, e2);
  if (e2) cudaFreeAsync(e2, st);
  KRS_CUDA(e);
  return KRS_OK;
}

krs_status krs_tridiag_eigvecs(int32_t m, const double* delta, const double* eta, int32_t k, const double* theta_sel,
                               double* Q_out, void* stream) {
  if (m < 0 || k < 0 || (m > 0 && k > 0 && (!delta || !theta_sel || !Q_out || (m > 1 && !eta))))
    return fail(KRS_ERR_INVALID_ARG, "bad argument");
  if (m == 0 || k == 0) return KRS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  double* work = nullptr;
  KRS_CUDA(cudaMallocAsync((void**)&work, sizeof(double) * eigvecs_work_doubles(m, k), st));
  KRS_CUDA(launch_tridiag_eigvecs(m, delta, eta, k, theta_sel, Q_out, work, st));
  KRS_CUDA(cudaFreeAsync(work, st));
  return KRS_OK;
}

}  // extern "C"
