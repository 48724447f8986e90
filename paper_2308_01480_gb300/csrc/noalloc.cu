// Gram-apply pass Y = C (C^T X) that needs no caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they want
// this product: code running inside another framework's stream capture or
// memory pool, real-time loops where cudaMalloc would synchronise the device
// and stall, or plugins whose host application owns all device memory.
// This entry point serves them: its per-CTA partial sums live in one
// fixed, file-scope device array that is created when the library is loaded
// on a device and stays there until the process exits.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

// 4 Mi floats = 16 MiB of partial sums, shared by every call on a device.
constexpr int64_t kScratchFloats = int64_t(4) << 20;
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
cudaError_t scratch_for_current_device(float** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

tt_status noalloc_fail(tt_status s, const char* msg) {
  ttr::set_last_error(msg);   // reported by tt_rbki_last_error()
  return s;
}

}  // namespace

extern "C" tt_status tt_gram_apply_noalloc(const void* C, int c_dtype, int64_t m, int64_t n, int b,
                                           const float* x, float* y, void* stream) {
  if (!C || !x || !y) return noalloc_fail(TT_EINVAL, "tt_gram_apply_noalloc: NULL pointer");
  if (c_dtype != TT_F32 && c_dtype != TT_BF16)
    return noalloc_fail(TT_EINVAL, "tt_gram_apply_noalloc: c_dtype must be TT_F32 or TT_BF16");
  if (m < 1 || n < 1 || b < 1) return noalloc_fail(TT_EINVAL, "tt_gram_apply_noalloc: m, n, b must be >= 1");
  if (m > 256 || b > 48 || !ttr::simt_ga_fused_ok(m, b))
    return noalloc_fail(TT_EUNSUPPORTED,
                        "tt_gram_apply_noalloc: needs m <= 256 and b <= 48 (the fixed scratch holds "
                        "at most one m x b partial per CTA)");
  float* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return noalloc_fail(TT_ECUDA, cudaGetErrorString(e));
  const int64_t max_ctas = kScratchFloats / (m * b);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c_dtype == TT_BF16)
    e = ttr::simt_ga_with_ctas<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(C), m, n, x, b, b, scratch,
                                              max_ctas, y, b, st);
  else
    e = ttr::simt_ga_with_ctas<float>(static_cast<const float*>(C), m, n, x, b, b, scratch, max_ctas, y, b, st);
  if (e != cudaSuccess) return noalloc_fail(TT_ECUDA, cudaGetErrorString(e));
  return TT_OK;
}
