// krs_batch.cu -- many independent solves in one persistent launch (krs_batch_t).
//
// A batch engine holds solves of different sequences (each with its own matrix, size and
// augmentation space) and runs their iteration loops together in the batched persistent
// kernel: the grid is cut into groups of g CTAs; each group takes the next solve from a
// work queue, iterates it with its own barrier counter, and takes the next one.  Per
// solve, the host stages around the loop are the ones of a single solve (set-up and init
// before, recycling step and result after), run on the engine's stream.
//
// Work order.  The queue is sorted by estimated remaining work, largest first (longest
// processing time first), so that the solves left at the end of a launch are short ones.
// The estimate is n * remaining iterations * (n_c + j + 30): per iteration a solve streams
// its operator (about 30 vector-equivalents for a 3x3 block row of 27 blocks) plus the
// n_c + j columns of the projection and reorthogonalisation; the iteration count is the
// sequence's previous one, or 12 n^(1/3) for its first solve.
//
// Launch quantum.  Each launch runs a solve for at most `quantum` iterations; a solve
// that has not ended is suspended (every value its loop carries lives in global memory)
// and resumed by a later launch, possibly in another group.  Between launches the engine
// finishes ended solves (their results are returned), admits newly submitted ones, and
// grows direction storage that a long solve has filled: the kernel never starts an
// iteration whose direction column is not allocated, so storage starts at the expected
// size instead of max_iter.
//
// Group size.  g (CTAs per solve) is the engine's tile shape: small g gives many solves
// in flight with little barrier cost per row, large g finishes each solve sooner.  With
// group_ctas > 0 every launch uses that size.  Otherwise each launch picks g from its
// queue: at least SMs / solves (so few solves still fill the device; a lone solve gets
// all of it) and at least the largest solve's share of the SMs by estimated work (so that
// solve is not the launch's critical path), times group_scale / 100, then the size near
// it that leaves the fewest SMs idle.  Such a launch also drains: once half of its groups
// have found the queue empty, every group suspends its solve at the end of the current
// iteration and the launch ends, so the host relaunches the remaining solves with a larger
// g (and admits new ones) instead of leaving half the device idle.  With group_scale = 0
// the autotuner picks the scale at the first launch: it runs each candidate on the queued
// solves for a few iterations, times the launch with events, keeps the one with the most
// rows x iterations per second, and re-initialises the solves (the init stage recomputes
// every value the probe iterations changed, so results do not depend on the probe).
//
// Reproducibility.  A launch prepares every solve's context for a partition over g CTAs,
// and a solve's bits depend on the partitions of its launches only: with group_ctas
// fixed, a solve gives the same bits whichever group runs it, however its iterations are
// split across launches and whatever other solves share the engine; with an adaptive g
// the results of a solve in different mixes agree to rounding.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "krs.h"
#include "krs_device.cuh"
#include "krs_internal.h"
#include "krs_seq.h"

using namespace krs;

namespace {

struct Entry {
  krs_seq* s = nullptr;
  krs_policy p{};
  double tol = 0.0;
  double* x_out = nullptr;
  int64_t tag = 0;
  SolveState ss;
  cudaStream_t saved_stream = nullptr;
  bool ended = false;  // the iteration loop has terminated (or never had to run)
  int status = KRS_OK;
  int m = 0;
  int j = 0;           // next iteration
  double m_est = 0.0;  // expected iteration count
  int g = 0;           // CTAs per group in the current launch
};

constexpr int kTuneIters = 8;
const int kTuneScale[] = {50, 100, 200};

}  // namespace

struct krs_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* uctx = nullptr;
  int sms = 0;
  krs_batch_config cfg{};
  int scale = 0;  // group_scale in use (0 until chosen)

  std::vector<Entry*> entries;  // submitted, not yet returned
  std::vector<int64_t> done_tags;
  std::vector<int32_t> done_status;

  // device buffers
  void* d_ctxs = nullptr;
  int ctx_cap = 0;
  int* d_tab = nullptr;               // queue | qoff | heads | cta_group | grp_cta0 | grp_class
  int* d_gather = nullptr;
  int* d_misc = nullptr;              // idle [1], bctrl [8 .. 8 + CTRL_WORDS), drain words [64 .. 64 + SMs)
  int* d_mail = nullptr;
  unsigned long long* d_gbar = nullptr;
  double *d_gpart = nullptr, *d_gvpart = nullptr, *d_ggpart = nullptr;
  int grp_cta_cap = 0;                // CTAs the group buffers hold
  int64_t vld_cap = 0;

  // pinned host staging
  char* h_ctxs = nullptr;
  int* h_tab = nullptr;
  int* h_gather = nullptr;
  int h_cap = 0;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t post[4] = {nullptr, nullptr, nullptr, nullptr};  // finishing streams
  krs_batch_stats st{};
};

constexpr int kPostStreams = 4;

// ------------------------------------------------------------------------------------
// engine memory
// ------------------------------------------------------------------------------------
static krs_status b_alloc(krs_batch* b, size_t bytes, void** out) {
  void* p = nullptr;
  bytes = (bytes + 255) & ~size_t(255);
  if (b->ualloc) {
    p = b->ualloc(bytes, b->uctx);
    if (!p) return failf(KRS_ERR_OOM, "batch: allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return failf(e == cudaErrorMemoryAllocation ? KRS_ERR_OOM : KRS_ERR_CUDA, "batch: cudaMalloc(%zu): %s", bytes,
                   cudaGetErrorString(e));
    }
  }
  KRS_CUDA(cudaMemsetAsync(p, 0, bytes, b->stream));
  *out = p;
  return KRS_OK;
}

static void b_free(krs_batch* b, void* p) {
  if (!p) return;
  if (b->ufree) {
    cudaStreamSynchronize(b->stream);
    b->ufree(p, b->uctx);
  } else {
    cudaFree(p);
  }
}

template <typename T>
static krs_status b_alloc_n(krs_batch* b, T** p, size_t count) {
  void* v = nullptr;
  KRS_TRY(b_alloc(b, count * sizeof(T), &v));
  *p = static_cast<T*>(v);
  return KRS_OK;
}

// ints of the launch table for `count` solves: queue, class offsets and heads, CTA ->
// group map, group offsets and classes (classes and groups <= SMs)
static size_t tab_ints(const krs_batch* b, int count) { return (size_t)count + 6 * (size_t)b->sms + 16; }

// table of `count` solves (contexts, launch table, gathered control words)
static krs_status ensure_table(krs_batch* b, int count) {
  if (count <= b->ctx_cap) return KRS_OK;
  int cap = b->ctx_cap ? b->ctx_cap : 64;
  while (cap < count) cap *= 2;
  b_free(b, b->d_ctxs);
  b_free(b, b->d_tab);
  b_free(b, b->d_gather);
  b->d_ctxs = nullptr;
  b->d_tab = b->d_gather = nullptr;
  KRS_TRY(b_alloc(b, apcg_ctx_bytes() * cap, &b->d_ctxs));
  KRS_TRY(b_alloc_n(b, &b->d_tab, tab_ints(b, cap)));
  KRS_TRY(b_alloc_n(b, &b->d_gather, 4 * (size_t)cap + CTRL_WORDS));
  if (b->h_ctxs) cudaFreeHost(b->h_ctxs);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  if (b->h_gather) cudaFreeHost(b->h_gather);
  b->h_ctxs = nullptr;
  b->h_tab = b->h_gather = nullptr;
  if (cudaMallocHost(&b->h_ctxs, apcg_ctx_bytes() * cap) != cudaSuccess ||
      cudaMallocHost(&b->h_tab, sizeof(int) * tab_ints(b, cap)) != cudaSuccess ||
      cudaMallocHost(&b->h_gather, sizeof(int) * (4 * (size_t)cap + CTRL_WORDS)) != cudaSuccess) {
    cudaGetLastError();
    return failf(KRS_ERR_OOM, "batch: pinned host allocation failed");
  }
  b->ctx_cap = cap;
  b->h_cap = cap;
  return KRS_OK;
}

// per-group barrier counters, mailboxes and partial sums for `ctas` CTAs, vld columns
static krs_status ensure_groups(krs_batch* b, int ctas, int64_t vld) {
  if (ctas <= b->grp_cta_cap && vld <= b->vld_cap) return KRS_OK;
  const int c = std::max(ctas, b->grp_cta_cap);
  const int64_t v = std::max(vld, b->vld_cap);
  b_free(b, b->d_mail);
  b_free(b, b->d_gbar);
  b_free(b, b->d_gpart);
  b_free(b, b->d_gvpart);
  b_free(b, b->d_ggpart);
  b->d_mail = nullptr;
  b->d_gbar = nullptr;
  b->d_gpart = b->d_gvpart = b->d_ggpart = nullptr;
  // groups <= ctas
  KRS_TRY(b_alloc_n(b, &b->d_mail, 2 * (size_t)c));
  KRS_TRY(b_alloc_n(b, &b->d_gbar, 16 * (size_t)c));
  KRS_TRY(b_alloc_n(b, &b->d_gpart, (size_t)c * PS_STRIDE));
  KRS_TRY(b_alloc_n(b, &b->d_gvpart, (size_t)c * v));
  KRS_TRY(b_alloc_n(b, &b->d_ggpart, (size_t)c * v));
  b->grp_cta_cap = c;
  b->vld_cap = v;
  return KRS_OK;
}

// ------------------------------------------------------------------------------------
// solves in the engine
// ------------------------------------------------------------------------------------
static double remaining_work(const Entry* e) {
  const double n = (double)e->s->n;
  double left = e->m_est - e->j;
  if (left < 16.0) left = 16.0;
  return n * left * (e->ss.nc + e->j + 0.5 * left + 30.0);
}

static int first_cap(const Entry* e) {
  int cap = (int)ceil(1.25 * e->m_est) + 16;
  cap = (int)round_up(cap, 32) - 1;  // columns cap + 1 fill whole 32-column steps
  if (cap > e->p.max_iter) cap = e->p.max_iter;
  if (cap < 31 && e->p.max_iter >= 31) cap = 31;
  return cap;
}

// iteration arguments of entry e for a partition over its g CTAs
static IterArgs group_args(const Entry* e, int64_t vld) {
  const int g = e->g;
  krs_seq* s = e->s;
  IterArgs a = e->ss.a;
  if (single_pass(e->p.precision)) {  // FP64 / double-float storage may have grown since the set-up
    a.W = s->W; a.AW = s->AW; a.Z = s->Z; a.ucoef = s->ucoef;
    a.alpha = s->alpha; a.gamma = s->gamma; a.rho = s->rho; a.gfull = s->gfull;
  }
  a.tfull = s->tfull; a.sfull = s->sfull;
  a.P = g;
  int64_t per = (s->nbr + g - 1) / g;
  a.npc = (int)round_up(per, 4);
  a.jcap = dir_cap(s, e->p.precision) - 1;  // iteration j writes direction column j + 1
  a.vld = vld;
  a.ctrl = s->ctrl;
  return a;
}

static krs_status restore_stream(Entry* e) {
  e->s->stream = e->saved_stream;
  e->s->busy = false;
  return KRS_OK;
}

// Refinement solves (KRS_MIXED_IR): after a pass's iterations (have_pass: their outcome
// st_in, m_in), update the FP64 iterate and residual, then start the next pass: the entry
// is queued again with iteration 0 when the pass has iterations to run, or it ends.
static krs_status advance_refinement(krs_batch* b, Entry* e, int st_in, int m_in, bool have_pass) {
  krs_seq* s = e->s;
  bool finished = false;
  for (;;) {
    if (have_pass) {
      KRS_TRY(refine_pass_end(s, &e->p, e->tol, &e->ss, st_in, m_in, &finished));
      if (finished) break;
    }
    bool need_loop = false;
    KRS_TRY(refine_pass_begin(s, &e->p, e->tol, &e->ss, &need_loop, &finished));
    if (finished) break;
    if (need_loop) {
      KRS_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(int) * CTRL_WORDS, b->stream));
      e->j = 0;
      e->ended = false;
      e->m_est = e->ss.m_first > 0 ? (double)e->ss.m_first : e->m_est;
      return KRS_OK;
    }
    have_pass = true;  // a pass already within its tolerance: no iterations
    st_in = KRS_OK;
    m_in = 0;
  }
  e->ended = true;
  e->status = e->ss.status;
  e->m = e->ss.m;
  return KRS_OK;
}

// Group size of a launch over `run` (see the file comment).
static int choose_group(const krs_batch* b, const std::vector<Entry*>& run) {
  const int T = b->sms;
  if (b->cfg.group_ctas > 0) return b->cfg.group_ctas;
  double W = 0.0, wmax = 0.0;
  for (Entry* e : run) {
    const double w = remaining_work(e);
    W += w;
    wmax = std::max(wmax, w);
  }
  double g = std::max((double)T / (double)run.size(), W > 0.0 ? wmax / W * T : 1.0);
  g *= (b->scale > 0 ? b->scale : 100) / 100.0;
  if (g < 1.0) g = 1.0;
  if (g > T) g = T;
  // among sizes within 15% of g, the one that leaves the fewest SMs idle
  int best = std::max(1, (int)(g + 0.5));
  int best_used = (T / best) * best;
  for (int c = std::max(1, (int)(0.85 * g)); c <= std::min(T, (int)(1.15 * g) + 1); c++) {
    const int used = (T / c) * c;
    if (used > best_used) {
      best = c;
      best_used = used;
    }
  }
  return best;
}

// Run the not-ended entries of `run` for at most `quantum` iterations in one launch (or
// until the launch drains).
// *ms: the launch's event time; *rows_iters: sum over the solves that ran of n x the
// iterations they did (the autotuner's work measure).
static krs_status launch_once(krs_batch* b, std::vector<Entry*>& run, int quantum, float* ms,
                              double* rows_iters = nullptr) {
  *ms = 0.f;
  if (rows_iters) *rows_iters = 0.0;
  if (run.empty()) return KRS_OK;
  const int T = b->sms;  // one CTA per SM (the kernel's register budget)
  const int g = choose_group(b, run);
  if (g > T) return failf(KRS_ERR_INVALID_ARG, "batch: group of %d CTAs exceeds the %d SMs", g, T);
  const int ngroups_all = T / g;
  // one class: every solve, largest remaining work first
  std::vector<Entry*> queued = run;
  std::stable_sort(queued.begin(), queued.end(), [](Entry* x, Entry* y) { return remaining_work(x) > remaining_work(y); });
  for (Entry* e : queued) e->g = g;
  std::vector<int> qoff = {0, (int)queued.size()}, act = {0};
  std::vector<int> gs = {g}, groups = {std::min(ngroups_all, (int)queued.size())};
  const int drain_at = (b->cfg.group_ctas > 0 || groups[0] < 2) ? 0 : (groups[0] + 1) / 2;
  const int count = (int)queued.size();
  const int nact = (int)act.size();
  int kmax = 1;
  for (Entry* e : queued)  // refinement passes project against C and the earlier passes' directions
    kmax = std::max(kmax, std::max(std::max(e->ss.nc, e->ss.a.nc), dir_cap(e->s, e->p.precision)));
  const int64_t vld = round_up(kmax + 1, 32);
  int bps = 0;
  const int prec = prec_id(queued[0]->p.precision);  // one precision per launch
  KRS_CUDA(apcg_batched_coresident(kmax, prec, &bps));
  if (bps < 1) return failf(KRS_ERR_CUDA, "batch: persistent kernel cannot be resident (kmax %d)", kmax);
  KRS_TRY(ensure_table(b, count));
  KRS_TRY(ensure_groups(b, T, vld));

  // launch table: queue | qoff | heads | cta_group | grp_cta0 | grp_class
  int* tq = b->h_tab;
  int* tqoff = tq + count;
  int* theads = tqoff + (nact + 1);
  int* tcg = theads + nact;
  std::vector<int> cta0(1, 0), gcls;
  for (int a = 0; a < nact; a++) {
    const int c = act[a];
    for (int k = 0; k < groups[c]; k++) {
      cta0.push_back(cta0.back() + gs[c]);
      gcls.push_back(a);
    }
  }
  const int ngroups = (int)gcls.size();
  const int ctas = cta0.back();
  int* tg0 = tcg + ctas;
  int* tgc = tg0 + (ngroups + 1);
  const size_t cb = apcg_ctx_bytes();
  for (int i = 0; i < count; i++) {
    IterArgs a = group_args(queued[i], vld);
    apcg_fill_ctx(a, b->h_ctxs + cb * i);
    tq[i] = i;
  }
  for (int a = 0; a <= nact; a++) tqoff[a] = qoff[a];
  for (int a = 0; a < nact; a++) theads[a] = 0;
  for (int gi = 0; gi < ngroups; gi++)
    for (int t = cta0[gi]; t < cta0[gi + 1]; t++) tcg[t] = gi;
  for (int gi = 0; gi <= ngroups; gi++) tg0[gi] = cta0[gi];
  for (int gi = 0; gi < ngroups; gi++) tgc[gi] = gcls[gi];
  const size_t tab_n = (size_t)(tgc + ngroups - tq);
  KRS_CUDA(cudaMemcpyAsync(b->d_ctxs, b->h_ctxs, cb * count, cudaMemcpyHostToDevice, b->stream));
  KRS_CUDA(cudaMemcpyAsync(b->d_tab, b->h_tab, sizeof(int) * tab_n, cudaMemcpyHostToDevice, b->stream));
  KRS_CUDA(cudaMemsetAsync(b->d_misc, 0, sizeof(int) * (64 + (size_t)T), b->stream));
  KRS_CUDA(cudaMemsetAsync(b->d_gbar, 0, sizeof(unsigned long long) * 16 * ngroups, b->stream));
  int* d = b->d_tab;
  BatchLaunch L{};
  L.ctxs = b->d_ctxs;
  L.queue = d;
  L.qoff = d + (tqoff - tq);
  L.heads = d + (theads - tq);
  L.cta_group = d + (tcg - tq);
  L.grp_cta0 = d + (tg0 - tq);
  L.grp_class = d + (tgc - tq);
  L.ctas = ctas;
  L.quantum = quantum;
  L.kmax = kmax;
  L.drain_at = drain_at;
  L.idle = b->d_misc + 1;
  L.gstop = b->d_misc + 64;
  L.mail = b->d_mail;
  L.gbar = b->d_gbar;
  L.gpart = b->d_gpart;
  L.gvpart = b->d_gvpart;
  L.ggpart = b->d_ggpart;
  L.vld = vld;
  L.spin_limit = queued[0]->s->spin_limit;
  L.bctrl = b->d_misc + 8;
  KRS_CUDA(cudaEventRecord(b->e0, b->stream));
  KRS_CUDA(apcg_launch_batched(L, prec, b->stream));
  KRS_CUDA(cudaEventRecord(b->e1, b->stream));
  KRS_CUDA(apcg_gather_ctrl(b->d_ctxs, count, b->d_gather, b->stream));
  KRS_CUDA(cudaMemcpyAsync(b->h_gather, b->d_gather, sizeof(int) * 4 * count, cudaMemcpyDeviceToHost, b->stream));
  int bctrl[CTRL_WORDS];
  KRS_CUDA(cudaMemcpyAsync(b->h_gather + 4 * count, b->d_misc + 8, sizeof(int) * CTRL_WORDS, cudaMemcpyDeviceToHost,
                           b->stream));
  KRS_CUDA(cudaStreamSynchronize(b->stream));
  memcpy(bctrl, b->h_gather + 4 * count, sizeof(bctrl));
  cudaEventElapsedTime(ms, b->e0, b->e1);
  b->st.launches++;
  b->st.kernel_launches += 3;
  b->st.last_kernel_ms = *ms;
  b->st.total_kernel_ms += *ms;
  b->st.group_ctas = ngroups > 0 ? ctas / ngroups : 0;
  b->st.groups = ngroups;
  b->st.classes = nact;
  b->st.last_launch_solves = count;
  for (int i = 0; i < count; i++) {
    Entry* e = queued[i];
    const int* cw = b->h_gather + 4 * i;
    const int j_before = e->j;
    e->ss.t_iter += *ms;
    if (cw[CTRL_DONE] && e->p.precision == KRS_MIXED_IR) {
      // one refinement pass ended: the next pass starts (or the refinement ends)
      if (rows_iters) *rows_iters += (double)e->s->n * (cw[CTRL_M] - j_before);
      KRS_TRY(advance_refinement(b, e, cw[CTRL_STATUS], cw[CTRL_M], true));
    } else if (cw[CTRL_DONE]) {
      e->ended = true;
      e->status = cw[CTRL_STATUS];
      e->m = cw[CTRL_M];
      if (rows_iters) *rows_iters += (double)e->s->n * (e->m - j_before);
    } else if (bctrl[CTRL_STATUS] || bctrl[CTRL_ABORT]) {
      e->ended = true;  // a group gave up waiting: the launch was abandoned
      e->status = bctrl[CTRL_STATUS] ? bctrl[CTRL_STATUS] : KRS_ERR_TIMEOUT;
      e->m = cw[CTRL_J];
    } else {
      e->j = cw[CTRL_J];
      if (rows_iters) *rows_iters += (double)e->s->n * (e->j - j_before);
    }
  }
  return KRS_OK;
}

// Re-run the init stage of entries (after the autotuner's probe iterations).
static krs_status reinit(krs_batch* b, std::vector<Entry*>& run) {
  for (Entry* e : run) {
    krs_seq* s = e->s;
    KRS_CUDA(apcg_launch_init(e->ss.a, s->b, s->scal, b->stream, &e->ss.launches));
    KRS_CUDA(cudaMemsetAsync(s->ctrl, 0, sizeof(int) * CTRL_WORDS, b->stream));
    e->j = 0;
    e->g = 0;
    e->ended = false;
    e->status = KRS_OK;
    e->m = 0;
  }
  KRS_CUDA(cudaStreamSynchronize(b->stream));
  return KRS_OK;
}

static krs_status autotune(krs_batch* b, std::vector<Entry*>& run) {
  // every candidate runs the same solves for their first iterations; compare rows x
  // iterations per second
  int nc = 0;
  double best = -1.0;
  int best_r = 0;
  for (int r : kTuneScale) {
    if (nc > 0) KRS_TRY(reinit(b, run));
    b->scale = r;
    float ms = 0.f;
    double ri = 0.0;
    std::vector<Entry*> part[4];
    for (Entry* e : run) part[prec_id(e->p.precision)].push_back(e);
    for (auto& pr : part) {
      if (pr.empty()) continue;
      float ms1 = 0.f;
      double ri1 = 0.0;
      KRS_TRY(launch_once(b, pr, kTuneIters, &ms1, &ri1));
      ms += ms1;
      ri += ri1;
    }
    for (Entry* e : run) e->ss.t_iter = 0.f;
    const double rate = ms > 0.f ? ri / ms : 0.0;
    if (nc < 8) {
      b->st.tune_scale[nc] = r;
      b->st.tune_ms[nc] = ms;
      b->st.tune_rate[nc] = rate * 1e3;
    }
    nc++;
    if (rate > best) {
      best = rate;
      best_r = r;
    }
  }
  b->st.tune_candidates = nc;
  KRS_TRY(reinit(b, run));
  b->st.tuned_group_scale = best_r;
  b->scale = best_r;
  return KRS_OK;
}

// Finish ended entries: recycling, result, statistics; they leave the engine.  The stages
// of every ended solve are enqueued together, round-robin over a few streams, with one
// synchronisation per stage instead of two per solve, so the small between-solve kernels
// of different solves run concurrently.
static krs_status finish_ended(krs_batch* b) {
  std::vector<Entry*> keep, done;
  for (Entry* e : b->entries) (e->ended ? done : keep).push_back(e);
  if (done.empty()) return KRS_OK;
  // the solves' last kernels ran on the engine's stream
  KRS_CUDA(cudaStreamSynchronize(b->stream));
  std::vector<krs_status> res(done.size(), KRS_OK);
  for (size_t i = 0; i < done.size(); i++) done[i]->s->stream = b->post[i % kPostStreams];
  for (size_t i = 0; i < done.size(); i++)
    if (done[i]->p.precision == KRS_MIXED_IR) res[i] = refine_finish(done[i]->s, &done[i]->p, &done[i]->ss);
  for (int stage = 1; stage <= 3; stage++) {
    for (size_t i = 0; i < done.size(); i++) {
      Entry* e = done[i];
      if (res[i] != KRS_OK) continue;
      res[i] = seq_end_stage(e->s, &e->ss, e->status, e->m, e->x_out, &e->p, stage);
    }
    if (stage < 3)
      for (int k = 0; k < kPostStreams; k++) KRS_CUDA(cudaStreamSynchronize(b->post[k]));
  }
  for (size_t i = 0; i < done.size(); i++) {
    Entry* e = done[i];
    if (res[i] != KRS_OK && e->s->st.status == 0) e->s->st.status = res[i];
    restore_stream(e);
    b->done_tags.push_back(e->tag);
    b->done_status.push_back((int32_t)res[i]);
    delete e;
  }
  b->entries.swap(keep);
  return KRS_OK;
}

// Grow the direction storage of suspended entries that reached it.
static krs_status grow_full(krs_batch* b) {
  for (Entry* e : b->entries) {
    if (e->ended) continue;
    krs_seq* s = e->s;
    const int dc = dir_cap(s, e->p.precision);
    if (e->j < dc - 1) continue;
    int cap = (int)round_up((int64_t)(1.5 * (dc - 1)) + 1, 32) - 1;
    if (cap > e->p.max_iter) cap = e->p.max_iter;
    KRS_TRY(seq_grow_directions(s, cap, e->j + 1, e->p.precision));
  }
  return KRS_OK;
}

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" {

krs_status krs_batch_create(const krs_device* dev, const krs_batch_config* cfg, krs_batch_t* out) {
  if (!out) return failf(KRS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (dev && ((dev->alloc == nullptr) != (dev->free == nullptr)))
    return failf(KRS_ERR_INVALID_ARG, "alloc and free must both be set or both be NULL");
  krs_batch_config c{};
  if (cfg) c = *cfg;
  if (c.group_ctas < 0 || c.quantum < 0 || c.group_scale < 0)
    return failf(KRS_ERR_INVALID_ARG, "group_ctas, group_scale and quantum must be >= 0");
  krs_batch* b = new (std::nothrow) krs_batch();
  if (!b) return failf(KRS_ERR_OOM, "host allocation failed");
  b->cfg = c;
  if (dev) {
    b->device = dev->device;
    b->stream = (cudaStream_t)dev->cuda_stream;
    b->ualloc = dev->alloc;
    b->ufree = dev->free;
    b->uctx = dev->ctx;
  }
  auto bail = [&](krs_status st) {
    krs_batch_destroy(b);
    return st;
  };
  if (cudaSetDevice(b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return failf(KRS_ERR_CUDA, "batch: no CUDA device %d", dev ? dev->device : 0);
  }
  if (c.group_ctas > b->sms) {
    delete b;
    return failf(KRS_ERR_INVALID_ARG, "group_ctas %d exceeds the %d SMs", c.group_ctas, b->sms);
  }
  b->scale = c.group_scale;
  krs_status st = b_alloc_n(b, &b->d_misc, 64 + (size_t)b->sms);
  if (st) return bail(st);
  if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess)
    return bail(failf(KRS_ERR_CUDA, "cudaEventCreate failed"));
  for (int k = 0; k < kPostStreams; k++)
    if (cudaStreamCreateWithFlags(&b->post[k], cudaStreamNonBlocking) != cudaSuccess)
      return bail(failf(KRS_ERR_CUDA, "cudaStreamCreate failed"));
  *out = b;
  return KRS_OK;
}

krs_status krs_batch_destroy(krs_batch_t b) {
  if (!b) return KRS_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  for (Entry* e : b->entries) {
    restore_stream(e);
    delete e;
  }
  b->entries.clear();
  void* bufs[] = {b->d_ctxs, b->d_tab, b->d_gather, b->d_misc, b->d_mail, b->d_gbar, b->d_gpart, b->d_gvpart, b->d_ggpart};
  for (void* p : bufs) b_free(b, p);
  if (b->h_ctxs) cudaFreeHost(b->h_ctxs);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  if (b->h_gather) cudaFreeHost(b->h_gather);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  for (int k = 0; k < kPostStreams; k++)
    if (b->post[k]) {
      cudaStreamSynchronize(b->post[k]);
      cudaStreamDestroy(b->post[k]);
    }
  delete b;
  return KRS_OK;
}

krs_status krs_batch_submit(krs_batch_t b, krs_seq_t s, const krs_bsr* A, const double* rhs, double* x, double tol,
                            const krs_policy* p, int64_t tag) {
  if (!b || !s || !A || !rhs || !x || !p) return failf(KRS_ERR_INVALID_ARG, "NULL argument");
  if (!(tol >= 0.0) || !isfinite(tol)) return failf(KRS_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (s->busy) return failf(KRS_ERR_INVALID_ARG, "the sequence already has a solve in flight");
  if (s->device != b->device) return failf(KRS_ERR_INVALID_ARG, "sequence and batch are on different devices");
  KRS_TRY(validate_policy(p));
  if (p->precision == KRS_MIXED_PROJ)
    return failf(KRS_ERR_INVALID_ARG, "batched solves run in KRS_FP64, KRS_DOUBLE_FLOAT or KRS_MIXED_IR");
  if (p->max_iter < 1 || p->max_iter > 16000) return failf(KRS_ERR_INVALID_ARG, "max_iter %d outside [1, 16000]", p->max_iter);
  Entry* e = new (std::nothrow) Entry();
  if (!e) return failf(KRS_ERR_OOM, "host allocation failed");
  e->s = s;
  e->p = *p;
  e->tol = tol;
  e->x_out = x;
  e->tag = tag;
  e->m_est = s->st.m > 0 ? (double)s->st.m : 12.0 * cbrt((double)s->n);
  e->saved_stream = s->stream;
  s->stream = b->stream;
  s->busy = true;
  krs_status st = KRS_OK;
  if (p->precision == KRS_MIXED_IR) {
    // FP64 refinement around FP32 passes: set-up, the first FP64 residual, the first pass's
    // init (the pass's iterations run in the batched launches)
    st = refine_setup(s, A, rhs, p, &e->ss);
    if (st == KRS_OK) st = refine_start(s, p, tol, &e->ss);
    if (st == KRS_OK) st = advance_refinement(b, e, KRS_OK, 0, false);
  } else {
    st = seq_begin(s, A, rhs, tol, p, first_cap(e), &e->ss);
    if (st == KRS_OK) {
      cudaError_t ce = cudaMemsetAsync(s->ctrl, 0, sizeof(int) * CTRL_WORDS, b->stream);
      if (ce != cudaSuccess) st = failf(KRS_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(ce));
    }
  }
  if (st != KRS_OK) {
    if (s->st.status == 0) s->st.status = st;
    restore_stream(e);
    delete e;
    return st;
  }
  if (single_pass(p->precision) && !e->ss.need_iter) e->ended = true;  // ||r_0|| within tolerance: m = 0
  b->entries.push_back(e);
  return KRS_OK;
}

krs_status krs_batch_step(krs_batch_t b, int32_t max_done, int64_t* done_tags, int32_t* done_status,
                          int32_t* n_done) {
  if (!b || !n_done || max_done < 0 || (max_done > 0 && (!done_tags || !done_status)))
    return failf(KRS_ERR_INVALID_ARG, "bad argument");
  *n_done = 0;
  KRS_CUDA(cudaSetDevice(b->device));
  std::vector<Entry*> run;
  for (Entry* e : b->entries)
    if (!e->ended) run.push_back(e);
  if (!run.empty()) {
    if (b->cfg.group_ctas == 0 && b->scale == 0) {
      bool fresh = true;  // (refinement passes change state the probe could not restore)
      for (Entry* e : run) fresh = fresh && e->j == 0 && e->g == 0 && single_pass(e->p.precision);
      if (fresh) KRS_TRY(autotune(b, run));
      if (b->scale == 0) b->scale = 100;
    }
    // one launch per precision present (each launch runs one kernel instantiation)
    std::vector<Entry*> part[4];
    for (Entry* e : run) part[prec_id(e->p.precision)].push_back(e);
    for (auto& pr : part) {
      if (pr.empty()) continue;
      float ms = 0.f;
      KRS_TRY(launch_once(b, pr, b->cfg.quantum, &ms));
    }
    KRS_TRY(grow_full(b));
  }
  KRS_TRY(finish_ended(b));
  b->st.in_flight = (int32_t)b->entries.size();
  const int k = std::min<int>((int)b->done_tags.size(), max_done);
  for (int i = 0; i < k; i++) {
    done_tags[i] = b->done_tags[i];
    done_status[i] = b->done_status[i];
  }
  b->done_tags.erase(b->done_tags.begin(), b->done_tags.begin() + k);
  b->done_status.erase(b->done_status.begin(), b->done_status.begin() + k);
  *n_done = k;
  return KRS_OK;
}

krs_status krs_solve_batch(krs_batch_t b, int32_t count, const krs_seq_t* seqs, const krs_bsr* A,
                           const double* const* rhs, double* const* x, double tol, const krs_policy* p,
                           int32_t* status) {
  if (!b || count < 0 || (count > 0 && (!seqs || !A || !rhs || !x || !status)) || !p)
    return failf(KRS_ERR_INVALID_ARG, "bad argument");
  if (!b->entries.empty() || !b->done_tags.empty())
    return failf(KRS_ERR_INVALID_ARG, "krs_solve_batch needs an engine with no solve in flight");
  for (int i = 0; i < count; i++)
    for (int k = 0; k < i; k++)
      if (seqs[k] == seqs[i]) return failf(KRS_ERR_INVALID_ARG, "sequence %d appears twice", i);
  krs_status first_err = KRS_OK;
  for (int i = 0; i < count; i++) {
    krs_status st = krs_batch_submit(b, seqs[i], &A[i], rhs[i], x[i], tol, p, i);
    status[i] = st;
    if (st != KRS_OK && first_err == KRS_OK) first_err = st;
  }
  std::vector<int64_t> tags(count > 0 ? count : 1);
  std::vector<int32_t> sts(count > 0 ? count : 1);
  while (!b->entries.empty()) {
    int32_t nd = 0;
    krs_status st = krs_batch_step(b, count, tags.data(), sts.data(), &nd);
    if (st != KRS_OK) return st;
    for (int i = 0; i < nd; i++) {
      status[tags[i]] = sts[i];
      if (sts[i] != KRS_OK && first_err == KRS_OK) first_err = (krs_status)sts[i];
    }
  }
  return first_err == KRS_OK ? KRS_OK : failf(first_err, "at least one solve of the batch failed (see status[])");
}

krs_status krs_batch_get_stats(krs_batch_t b, krs_batch_stats* out) {
  if (!b || !out) return failf(KRS_ERR_INVALID_ARG, "NULL argument");
  b->st.in_flight = (int32_t)b->entries.size();
  *out = b->st;
  return KRS_OK;
}

}  // extern "C"
