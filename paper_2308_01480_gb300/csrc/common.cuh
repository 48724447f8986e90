// Shared definitions for the TT-rBKI CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/tt_rbki.h"

namespace ttr {

// Device status word values (mirrors tt_status where they overlap).
enum : int { DEV_OK = 0, DEV_BREAKDOWN = TT_EBREAKDOWN, DEV_NONFINITE = TT_ENONFINITE };

// Record the first non-OK status (later ones do not overwrite it).
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, DEV_OK, code);
}

// Element loads/stores for the two storage types.
__device__ __forceinline__ float ld_elem(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld_elem(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
__device__ __forceinline__ void st_elem(float* p, int64_t i, float v) { p[i] = v; }
__device__ __forceinline__ void st_elem(__nv_bfloat16* p, int64_t i, float v) {
  p[i] = __float2bfloat16_rn(v);
}

// Deterministic pseudo-random value in [-1, 1) from two 64-bit words (a
// SplitMix64-style finaliser), for replacing numerically vanished basis
// columns by directions that carry no information of their own.
__device__ __forceinline__ float hash_uniform(uint64_t a, uint64_t b) {
  uint64_t z = a * 0x9E3779B97F4A7C15ull + b + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (1.0f / 8388608.0f) - 1.0f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the whole CTA; `red` holds >= 32 floats of shared scratch.
// Every thread receives the total.  Contains two __syncthreads().
__device__ __forceinline__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = (lane < nw) ? red[lane] : 0.f;
  return warp_sum(t);
}

// Raises a kernel's dynamic shared-memory limit, once per kernel, to the
// largest the device allows next to the kernel's static shared memory.  One
// fixed limit (rather than one per launch) keeps every launch captured in a
// CUDA graph valid however the launches of other sizes that follow set it.
cudaError_t raise_smem_limit_ptr(const void* kernel);
template <typename Kernel>
inline cudaError_t raise_smem_limit(Kernel kernel) {
  return raise_smem_limit_ptr(reinterpret_cast<const void*>(kernel));
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

}  // namespace ttr
