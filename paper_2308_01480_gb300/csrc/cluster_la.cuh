// Building blocks for block orthonormalisation on one thread-block cluster
// (orth_cluster.cu, krylov_cluster.cu): register-tiled products over
// shared-memory row blocks and the rank-ordered sum of per-CTA shares
// through distributed shared memory.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace ttr {

namespace cg = cooperative_groups;

__host__ __device__ inline int pad4(int x) { return (x + 3) & ~3; }

// 4-byte asynchronous global -> shared copy; with ok = false it reads
// nothing and writes zero (src-size 0)
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// out[t][j] = sum_{i < rows} A[i][t] B[i][j], t < ta (multiple of 4), j < bp;
// row strides lda, ldb, ldo are multiples of 4 (16-byte aligned rows).
static __device__ void tn_tile(const float* A, int lda, int ta, const float* B, int ldb, int bp, int rows, float* out,
                        int ldo) {
  const int tt = ta >> 2, tj = bp >> 2;
  for (int tile = threadIdx.x; tile < tt * tj; tile += blockDim.x) {
    const int t0 = (tile / tj) * 4, j0 = (tile % tj) * 4;
    float acc[4][4] = {};
    for (int i = 0; i < rows; ++i) {
      const float4 x = *reinterpret_cast<const float4*>(A + i * lda + t0);
      const float4 v = *reinterpret_cast<const float4*>(B + i * ldb + j0);
      const float av[4] = {x.x, x.y, x.z, x.w}, bv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(av[u], bv[w], acc[u][w]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      *reinterpret_cast<float4*>(out + (t0 + u) * ldo + j0) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  }
}

// Y[i][j] = scale * sum_{t < kk} X[i][t] M[t][j] (+ Y0[i][j]), i < rows
// (multiple of 4), j < bp; row strides multiples of 4.
static __device__ void nn_tile(const float* X, int ldx, int kk, const float* M, int ldm, int rows, int bp, float* Y,
                        int ldy, const float* Y0, float scale) {
  const int ti = rows >> 2, tj = bp >> 2;
  for (int tile = threadIdx.x; tile < ti * tj; tile += blockDim.x) {
    const int i0 = (tile / tj) * 4, j0 = (tile % tj) * 4;
    float acc[4][4] = {};
    for (int t = 0; t < kk; ++t) {
      const float4 v = *reinterpret_cast<const float4*>(M + t * ldm + j0);
      const float bv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float x = X[(i0 + u) * ldx + t];
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(x, bv[w], acc[u][w]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float4 r = make_float4(acc[u][0] * scale, acc[u][1] * scale, acc[u][2] * scale, acc[u][3] * scale);
      if (Y0) {
        const float4 y = *reinterpret_cast<const float4*>(Y0 + (i0 + u) * ldy + j0);
        r.x += y.x; r.y += y.y; r.z += y.z; r.w += y.w;
      }
      *reinterpret_cast<float4*>(Y + (i0 + u) * ldy + j0) = r;
    }
  }
}

// Sums element e of the NC CTAs' shares (rank order, the same in every CTA)
// for e0 <= e < e1 and hands each sum to put(e, s); four elements per
// thread at a time, so that 4 NC remote loads are in flight together.
template <int NC, typename Put>
__device__ __forceinline__ void sum_ranks(cg::cluster_group& cl, float* mine, int e0, int e1, Put& put) {
  const float* src[NC];
#pragma unroll
  for (int r = 0; r < NC; ++r) src[r] = cl.map_shared_rank(mine, r);
  const int stride = blockDim.x;
  for (int base = e0 + threadIdx.x; base < e1; base += 4 * stride) {
    float x[4][NC];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * stride;
#pragma unroll
      for (int r = 0; r < NC; ++r) x[u][r] = (e < e1) ? src[r][e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * stride;
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < NC; ++r) s += x[u][r];
      if (e < e1) put(e, s);
    }
  }
}


// Cluster-wide sum of the shares in two steps, so that each CTA reads only
// twice as many remote values as there are elements (instead of NC times):
// CTA r sums the slice [r S, r S + S) of the elements (S = ceil((e1 - e0) / NC))
// over all ranks in rank order into its own buffer `slice` (S floats), one
// cluster barrier, then every CTA reads every slice from its owner and hands
// each sum to put(e, s).  `slice` must not be reused by the next call before
// a cluster barrier has passed (callers alternate two buffers).
template <typename Put>
__device__ __forceinline__ void cluster_reduce_scatter_gather(cg::cluster_group& cl, float* mine, float* slice, int e0,
                                                              int e1, Put& put) {
  const int nc = (int)cl.num_blocks();
  const int r = (int)cl.block_rank();
  const int n = e1 - e0;
  const int S = (n + nc - 1) / nc;
  const int s0 = e0 + r * S, s1 = min(e1, s0 + S);
  for (int e = s0 + (int)threadIdx.x; e < s1; e += blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < nc; ++q) s += cl.map_shared_rank(mine, q)[e];
    slice[e - s0] = s;
  }
  cl.sync();
  for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) {
    const int owner = (e - e0) / S;
    put(e, cl.map_shared_rank(slice, owner)[e - e0 - owner * S]);
  }
}

// Sums element e of the cluster's shares for e0 <= e < e1 (rank order) for
// any cluster size up to 16.
template <typename Put>
__device__ __forceinline__ void sum_ranks_any(cg::cluster_group& cl, float* mine, int e0, int e1, Put& put) {
  switch (cl.num_blocks()) {
    case 16: sum_ranks<16>(cl, mine, e0, e1, put); break;
    case 8: sum_ranks<8>(cl, mine, e0, e1, put); break;
    case 4: sum_ranks<4>(cl, mine, e0, e1, put); break;
    case 2: sum_ranks<2>(cl, mine, e0, e1, put); break;
    default: sum_ranks<1>(cl, mine, e0, e1, put); break;
  }
}

}  // namespace ttr
