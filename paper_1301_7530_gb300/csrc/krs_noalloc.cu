// krs_noalloc.cu -- krs_gemv_t_noalloc: the tall-skinny product t = V^T u without any
// device allocation.
//
// Who needs it: callers that must not touch the CUDA allocator at all -- a framework that
// has reserved the whole device for its own pool (any cudaMalloc / cudaMallocAsync outside
// it fails or fragments that pool), a latency-bound loop that cannot afford an
// allocation's cost or its implicit synchronisation, or code running where another
// component owns every allocation.  krs_gemv_t allocates its per-CTA partial sums on the
// stream; this variant keeps them in one fixed array in device global memory instead.
//
// The array: kNoallocScratchDoubles doubles (2 MiB), a file-scope __device__ variable, so
// every GPU on which the library is loaded holds it until the process exits.  It holds one
// partial sum per (CTA, column): at most kNoallocMaxK columns and kNoallocMaxCtas CTAs.
// Host code cannot use the symbol itself (in host code it names a host-side stand-in), so
// its device address is looked up once per device with cudaGetSymbolAddress, on that
// device, by the first call made there, and cached.
//
// Every call shares the array and it keeps the previous call's contents.  Nothing in it
// has to start at zero: the first kernel writes every partial the second one reads.  Two
// calls whose kernels overlap on the GPU (different streams, or different host threads
// without ordering) race on the array and give wrong results.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "krs.h"
#include "krs_device.cuh"
#include "krs_internal.h"

namespace krs {

constexpr int kNoallocMaxK = 1024;
constexpr int kNoallocMaxCtas = 256;
constexpr size_t kNoallocScratchDoubles = (size_t)kNoallocMaxK * kNoallocMaxCtas;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void __launch_bounds__(TPB, 1) k_noalloc_gemv_t_part(const double* V, int64_t ld, int k,
                                                                const double* u, int64_t n, int64_t rpc,
                                                                double* part) {
  extern __shared__ double4_32a smem_na[];
  double* base = reinterpret_cast<double*>(smem_na);
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = kmin64(n, r0 + rpc);
  cta_gemv_t<true>(V, ld, k, u, r0, r1, part + (int64_t)blockIdx.x * k, base, base + ROW_CHUNK);
}

__global__ void k_noalloc_reduce(const double* part, int P, int k, double* t) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= k) return;
  const double v = warp_sum_strided(part + warp, P, k);
  if ((threadIdx.x & 31) == 0) t[warp] = v;
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
  if (n == 0)
    return cudaMemsetAsync(t, 0, sizeof(double) * k, st) == cudaSuccess
               ? KRS_OK
               : set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: cudaMemsetAsync failed");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: no current CUDA device");
  int64_t rpc = ((n + sms - 1) / (sms > 0 ? sms : 1) + 3) / 4 * 4;
  if (rpc < 64) rpc = 64;
  const int64_t P = (n + rpc - 1) / rpc;
  if (P > kNoallocMaxCtas)
    return set_error(KRS_ERR_INVALID_ARG, "krs_gemv_t_noalloc: too many row blocks for its fixed scratch");
  double* part = nullptr;
  if (scratch_address(&part) != cudaSuccess)
    return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: cudaGetSymbolAddress of the scratch array failed");
  const size_t sm = sizeof(double) * (size_t)(ROW_CHUNK + 4 * TPB);  // cta_gemv_t's staging and partials
  if (cudaFuncSetAttribute((const void*)k_noalloc_gemv_t_part, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess)
    return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: cudaFuncSetAttribute failed");
  k_noalloc_gemv_t_part<<<(unsigned)P, TPB, sm, st>>>(V, ldv, k, u, n, rpc, part);
  k_noalloc_reduce<<<(k * 32 + 255) / 256, 256, 0, st>>>(part, (int)P, k, t);
  if (cudaGetLastError() != cudaSuccess) return set_error(KRS_ERR_CUDA, "krs_gemv_t_noalloc: launch failed");
  return KRS_OK;
}
