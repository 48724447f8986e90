// Input-side kernels: the Gaussian test matrices of Alg. 3 step 3 drawn on
// the device, and the canonicalising permute/convert of a strided tensor.
#include "common.cuh"
#include "kernels.h"

namespace ttr {

// Philox4x32 with 10 rounds, from its published definition (Salmon, Moraes,
// Dror, Shaw, SC'11): per round the two multiplications give high and low
// halves that are mixed with the other two words and the round key; the key
// advances by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// (0,1) uniform with 24 significant bits: exact in binary32.
__device__ __forceinline__ float u01(uint32_t x) {
  return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
}

// Box-Muller (1958): (u1, u2) -> sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  const float rad = sqrtf(-2.f * logf(u01(a)));
  float s, c;
  sincospif(2.f * u01(b), &s, &c);
  return make_float2(rad * c, rad * s);
}

// Omega_k entry (i, c) written at out[i * si + c * sc], i < n, c < b.  With
// a slab (w > 0) the n local rows are the rows (i / w) nd + lo + i % w of
// the full Omega_k: the columns of the unfolding whose last index lies in
// [lo, lo + w) of a last mode of size nd, in their order.
template <typename T>
__global__ void k_omega(uint64_t seed, uint32_t mode, int64_t n, int b, T* __restrict__ out, int64_t si,
                        int64_t sc, int64_t w, int64_t nd, int64_t lo) {
  const int groups = (b + 3) >> 2;
  const int64_t total = n * groups;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;            // consecutive threads -> consecutive rows
    const int g = (int)(e / n);
    const int64_t gi = (w > 0) ? (i / w) * nd + lo + i % w : i;   // row of the full Omega_k
    const uint4 x =
        philox4x32_10(make_uint4((uint32_t)gi, (uint32_t)((uint64_t)gi >> 32), (uint32_t)g, mode), k0, k1);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 4 * g + t;
      if (c < b) st_elem(out, i * si + (int64_t)c * sc, z[t]);
    }
  }
}

cudaError_t launch_omega(uint64_t seed, int mode, int64_t n, int b, void* out, int dtype, int64_t si,
                         int64_t sc, cudaStream_t st, int64_t slab_w, int64_t slab_nd, int64_t slab_lo) {
  const int64_t total = n * ((b + 3) / 4);
  const int blocks = (int)imin(ceil_div(total, 256), 152 * 16);
  ProfScope prof("omega_philox", st, (double)n * b * (dtype == TT_BF16 ? 2 : 4), 0);
  note_launch("omega_philox");
  if (dtype == TT_BF16)
    k_omega<__nv_bfloat16><<<blocks, 256, 0, st>>>(seed, (uint32_t)mode, n, b, (__nv_bfloat16*)out, si, sc, slab_w,
                                                   slab_nd, slab_lo);
  else
    k_omega<float><<<blocks, 256, 0, st>>>(seed, (uint32_t)mode, n, b, (float*)out, si, sc, slab_w, slab_nd,
                                           slab_lo);
  return cudaGetLastError();
}

// Transposed copy of an explicit Omega (n x b, row-major) into the b x n
// layout read by the sketch pass, with dtype conversion.
template <typename T>
__global__ void k_transpose_in(const float* __restrict__ src, int64_t n, int b, T* __restrict__ dst) {
  __shared__ float tile[32][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    int r = e / 32, c = e % 32;
    if (c < b && r0 + r < n) tile[c][r] = src[(r0 + r) * b + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    int c = e / 64, r = e % 64;
    if (c < b && r0 + r < n) st_elem(dst, (int64_t)c * n + r0 + r, tile[c][r]);
  }
}

cudaError_t launch_omega_transpose(const float* src, int64_t n, int b, void* dst, int dtype, cudaStream_t st) {
  if (b > 32) {
    // two passes of at most 32 columns each would need a strided source; use
    // the simple element-wise form for wide Omega
    return cudaErrorInvalidValue;
  }
  dim3 grid((unsigned)ceil_div(n, 64));
  note_launch("omega_transpose");
  if (dtype == TT_BF16)
    k_transpose_in<__nv_bfloat16><<<grid, 256, 0, st>>>(src, n, b, (__nv_bfloat16*)dst);
  else
    k_transpose_in<float><<<grid, 256, 0, st>>>(src, n, b, (float*)dst);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_transpose_in_wide(const float* __restrict__ src, int64_t n, int b, T* __restrict__ dst) {
  const int64_t total = n * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, r = e % n;
    st_elem(dst, e, src[r * b + c]);
  }
}

cudaError_t launch_omega_transpose_any(const float* src, int64_t n, int b, void* dst, int dtype, cudaStream_t st) {
  if (b <= 32) return launch_omega_transpose(src, n, b, dst, dtype, st);
  const int blocks = (int)imin(ceil_div(n * b, 256), 152 * 16);
  note_launch("omega_transpose");
  if (dtype == TT_BF16)
    k_transpose_in_wide<__nv_bfloat16><<<blocks, 256, 0, st>>>(src, n, b, (__nv_bfloat16*)dst);
  else
    k_transpose_in_wide<float><<<blocks, 256, 0, st>>>(src, n, b, (float*)dst);
  return cudaGetLastError();
}

// ------------------------------------------------------------ permute/convert
struct PermArgs {
  int d;
  int64_t ddims[8];     // destination mode sizes
  int64_t sstride[8];   // source stride of destination mode j
};

template <typename TS, typename TD>
__global__ void k_permute(const TS* __restrict__ src, TD* __restrict__ dst, int64_t total, PermArgs a) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e, off = 0;
    for (int j = a.d - 1; j >= 0; --j) {
      const int64_t idx = rem % a.ddims[j];
      rem /= a.ddims[j];
      off += idx * a.sstride[j];
    }
    st_elem(dst, e, ld_elem(src, off));
  }
}

cudaError_t launch_permute(const void* src, int sdt, void* dst, int ddt, const int64_t* dims,
                           const int64_t* sstrides, const int* perm, int d, cudaStream_t st) {
  PermArgs a;
  a.d = d;
  int64_t total = 1;
  for (int j = 0; j < d; ++j) {
    const int s = perm ? perm[j] : j;
    a.ddims[j] = dims[s];
    a.sstride[j] = sstrides[s];
    total *= dims[s];
  }
  if (total == 0) return cudaSuccess;
  const int blocks = (int)imin(ceil_div(total, 256), 152 * 32);
  note_launch("permute_convert");
  if (sdt == TT_F32 && ddt == TT_F32)
    k_permute<float, float><<<blocks, 256, 0, st>>>((const float*)src, (float*)dst, total, a);
  else if (sdt == TT_F32 && ddt == TT_BF16)
    k_permute<float, __nv_bfloat16><<<blocks, 256, 0, st>>>((const float*)src, (__nv_bfloat16*)dst, total, a);
  else if (sdt == TT_BF16 && ddt == TT_BF16)
    k_permute<__nv_bfloat16, __nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)src, (__nv_bfloat16*)dst, total, a);
  else if (sdt == TT_BF16 && ddt == TT_F32)
    k_permute<__nv_bfloat16, float><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)src, (float*)dst, total, a);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace ttr

// ---------------------------------------------------------------- test aid
namespace ttr {

// Every CTA fills its whole dynamic shared memory with `value`; with one
// maximal CTA per SM and several waves, each SM's shared memory ends up
// holding the pattern, so a later kernel that reads shared memory it never
// wrote sees it.
__global__ void k_fill_shared(uint32_t bits, int words) {
  extern __shared__ uint32_t fill_sm[];
  volatile uint32_t* p = fill_sm;   // volatile: the stores are the point
  for (int i = threadIdx.x; i < words; i += blockDim.x) p[i] = bits;
}

}  // namespace ttr

extern "C" tt_status tt_debug_fill_shared(uint32_t bits, void* stream) {
  int dev = 0, sms = 0, maxsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    ttr::set_last_error("tt_debug_fill_shared: device query failed");
    return TT_ECUDA;
  }
  const size_t bytes = (size_t)maxsm / 16 * 16;
  if (cudaFuncSetAttribute(ttr::k_fill_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
      cudaSuccess) {
    ttr::set_last_error("tt_debug_fill_shared: cudaFuncSetAttribute failed");
    return TT_ECUDA;
  }
  ttr::k_fill_shared<<<4 * sms, 1024, bytes, (cudaStream_t)stream>>>(bits, (int)(bytes / 4));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ttr::set_last_error(cudaGetErrorString(e));
    return TT_ECUDA;
  }
  return TT_OK;
}
