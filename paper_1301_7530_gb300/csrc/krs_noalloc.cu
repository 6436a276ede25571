// krs_noalloc.cu -- krs_gemv_t_noalloc: the tall-skinny product t = V^T u without any
// device allocation.
//
// Who needs it: callers that must not touch the CUDA allocator at all -- a framework that
// has reserved the whole device for its own pool (any cudaMalloc / cudaMallocAsync outside
// it fails or fragments that pool), a latency-bound loop that cannot afford an
// allocation's cost or its implicit synchronisation, or code running where another
// component owns every allocation.  krs_gemv_t allocates its per-CTA partial sums on the
// stream; this variant keeps them in one fixed array in device global memory instead and
// otherwise launches the very same kernels with the very same partition, so its result is
// bitwise krs_gemv_t's.
//
// The array: kNoallocScratchDoubles doubles (2 MiB), a file-scope __device__ variable, so
// every GPU on which the library is loaded holds it until the process exits.  It holds one
// partial sum per (row block, column): at most kNoallocMaxK columns and kNoallocMaxBlocks
// row blocks.  Host code cannot use the symbol itself (in host code it names a host-side
// stand-in), so its device address is looked up with cudaGetSymbolAddress, on the device
// that is current, by the first call made there, and cached together with the context it
// was found in; a call made under another context (after cudaDeviceReset, say) looks it
// up again.
//
// Every call shares the array and it keeps the previous call's contents.  Nothing in it
// has to start at zero: the first kernel writes every partial the second one reads.  Two
// calls whose kernels overlap on the GPU (different streams, or different host threads
// without ordering) race on the array and give wrong results.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "krs.h"
#include "krs_internal.h"

namespace krs {

constexpr int kNoallocMaxK = 1024;
constexpr int kNoallocMaxBlocks = 256;
constexpr size_t kNoallocScratchDoubles = (size_t)kNoallocMaxK * kNoallocMaxBlocks;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
struct ScratchSlot {
  CUcontext ctx;   // context the address was looked up in
  double* addr;    // device address of g_noalloc_scratch there
};
static ScratchSlot g_scratch[kMaxDevices] = {};
static std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// The calling thread's current context, through the driver entry point the runtime hands
// out (no link-time dependency on the driver library).  nullptr when it is unavailable.
static CUcontext current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array on the current device, looked up again whenever the
// current context is not the one of the cached address (or no context handle is known).
static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSlot& s = g_scratch[dev];
  if (!s.addr || !ctx || s.ctx != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    s.addr = static_cast<double*>(p);
    s.ctx = current_context();  // the lookup may have made the primary context current
  }
  *out = s.addr;
  return cudaSuccess;
}

}  // namespace krs

using namespace krs;

extern "C" krs_status krs_gemv_t_noalloc(int64_t n, int32_t k, const double* V, int64_t ldv, const double* u,
                                         double* t, void* stream) {
  if (n < 0 || k < 0 || (k > 0 && (!t || (n > 0 && (!V || !u)))))
    return set_error(KRS_ERR_INVALID_ARG, "krs_gemv_t_noalloc: bad argument");
  if (k > kNoallocMaxK)
    return set_error(KRS_ERR_INVALID_ARG, "krs_gemv_t_noalloc: k exceeds the 1024 columns its fixed scratch holds");
  if (k == 0) return KRS_OK;
  if (ldv % 4 != 0 || ldv < ((n + 3) / 4) * 4)
    return set_error(KRS_ERR_INVALID_ARG, "krs_gemv_t_noalloc: ldv must be a multiple of 4 and >= n rounded up to 4");
  if (((uintptr_t)V & 31) || ((uintptr_t)u & 31))
    return set_error(KRS_ERR_INVALID_ARG, "krs_gemv_t_noalloc: V and u must be 32-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  int P = 0;
  int64_t rpc = 0;
  if (gemv_rows_partition(n, &P, &rpc) != cudaSuccess)
    return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: no current CUDA device");
  if (P > kNoallocMaxBlocks)
    return set_error(KRS_ERR_INVALID_ARG, "krs_gemv_t_noalloc: too many row blocks for its fixed scratch");
  double* part = nullptr;
  if (n > 0 && scratch_address(&part) != cudaSuccess)
    return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: cudaGetSymbolAddress of the scratch array failed");
  // krs_gemv_t's kernels and partition with the partials in the fixed array (n == 0: t = 0)
  if (launch_gemv_t_rows(n, k, V, ldv, u, t, part, P, rpc, st) != cudaSuccess)
    return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: launch failed");
  return KRS_OK;
}
