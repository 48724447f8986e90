// The Gram matrix G = C C^T of an m x n unfolding with 128 < m <= 2048 rows
// and the Krylov power W = G X with it (the Gram-power route of Alg. 3 step
// 4: span{X, G X, ..., G^q X} is the block Krylov space of C C^T, so once G
// is formed every power reads the L2-resident m x m matrix instead of C).
//
// tcgen05 Gram (BF16 C, n % 8 == 0): G is cut into tiles of 128 rows
// (MMA M) by 256 columns (MMA N <= 256), only the tiles that meet the upper
// triangle.  Each CTA owns one tile and one contiguous range of 64-column
// k-boxes of C (split-K); per k-box TMA brings the A box (128 rows) and one or
// two B boxes (128 rows each) into a four-stage ring, one thread issues four
// 128 x N x 16 MMAs accumulating in TMEM (chunks of four k-boxes, double
// buffered), and eight epilogue warps add the chunks in FP32 registers and
// write the tile to a partial slot.  When the A rows lie inside the B rows (tiles
// on the diagonal) the A operand is read from the B box, not loaded again.
// A second kernel sums each tile's split partials in a fixed order and
// writes both triangles of G (deterministic, bit-reproducible).
//
// SIMT Gram (FP32 C, or BF16 shapes the tensor-core path does not take):
// 64 x 64 upper-triangular tiles with 4 x 4 register tiles, split-K, the same
// fixed-order reduction.
//
// Power: W (m x c) = G X, FP32, X a 16-byte-aligned padded block; 8 rows of
// W per CTA over many CTAs, four 128-row K chunks in flight by 16-byte
// asynchronous copies, 2 x 4 register tiles, a fixed-order sum over the
// CTA's K groups.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace ttr {

using namespace tc;

namespace {

constexpr int GT_THREADS = 320;             // producer, MMA, 8 epilogue warps
constexpr int GT_STAGES = 4;
constexpr int GT_BOX = 128 * 128;           // bytes of one 64-column x 128-row BF16 box
constexpr int GT_STAGE = 3 * GT_BOX;        // A box + two B boxes
constexpr int GT_CHUNK = 4;                 // k-boxes (16 MMAs) per TMEM accumulation chunk
constexpr int GT_MAX_TILES = 80;            // m <= 2048: 72 tiles
constexpr int GT_MAX_ITEMS = 320;
constexpr int GT_MAX_J = 9;

struct GtParams {
  int64_t m, n;
  int nitems, ntiles, nI, nJ;
  int* status;
  float* part;                      // nitems x 128 x 256 floats
  int tile_base[GT_MAX_J];          // first tile of column block J
  int4 tile[GT_MAX_TILES];          // I, J, N (MMA N), nbB | (a_box + 1) << 4
  int2 tile_items[GT_MAX_TILES];    // first item, count
  int4 item[GT_MAX_ITEMS];          // tile, kb0, kb1, 0
};

struct GtShared {
  uint64_t full[GT_STAGES];
  uint64_t empty[GT_STAGES];
  uint64_t cfull[2];
  uint64_t cempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

__device__ __forceinline__ void gt_abort(GtShared* sh, int* status) {
  sh->abort_flag = 1;
  set_status(status, TT_ETIMEOUT);
}

// The MMAs accumulate GT_CHUNK k-boxes at a time into one of two TMEM
// buffers (256 columns each); the eight epilogue warps add each finished
// chunk into FP32 registers (one row and 128 columns per thread) while the
// MMAs fill the other buffer.  The tensor cores' FP32 accumulation does
// not round to nearest, so its error grows with the number of MMAs that
// add into one accumulator; chunking bounds that number by 4 GT_CHUNK and
// the chunk sums are added with round-to-nearest.
__global__ void __launch_bounds__(GT_THREADS, 1)
k_gram_tiles(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ GtParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  GtShared* sh = reinterpret_cast<GtShared*>(ring + (size_t)GT_STAGES * GT_STAGE);
  volatile int* abortp = &sh->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 it4 = p.item[blockIdx.x];
  const int4 tl = p.tile[it4.x];
  const int I = tl.x, J = tl.y, N = tl.z, nbB = tl.w & 15, a_box = (tl.w >> 4) - 1;
  const int kb0 = it4.y, kb1 = it4.z;
  const int nchunks = (kb1 - kb0 + GT_CHUNK - 1) / GT_CHUNK;
  const uint32_t tmem_cols = 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < GT_STAGES; ++s) { mbar_init(&sh->full[s], 1); mbar_init(&sh->empty[s], 1); }
    for (int i = 0; i < 2; ++i) { mbar_init(&sh->cfull[i], 1); mbar_init(&sh->cempty[i], 8); }
    mbar_init(&sh->drain, 1);
    sh->abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&mapC);
  }
  if (warp == 1) {
    tmem_alloc(&sh->tmem_base, tmem_cols);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)((a_box < 0 ? 1 : 0) + nbB) * GT_BOX;
      int64_t fill = 0;
      for (int kb = kb0; kb < kb1; ++kb, ++fill) {
        const int s = (int)(fill % GT_STAGES);
        if (!mbar_wait(&sh->empty[s], (uint32_t)(((fill / GT_STAGES) & 1) ^ 1), abortp)) {
          gt_abort(sh, p.status);
          break;
        }
        uint8_t* st = ring + (size_t)s * GT_STAGE;
        mbar_arrive_expect_tx(&sh->full[s], bytes);
        if (a_box < 0) tma_load_2d(st, &mapC, &sh->full[s], kb * 64, I * 128);
        for (int bb = 0; bb < nbB; ++bb)
          tma_load_2d(st + (size_t)(1 + bb) * GT_BOX, &mapC, &sh->full[s], kb * 64, J * 256 + bb * 128);
      }
      // every issued copy lands before the CTA may exit
      for (int s = 0; s < GT_STAGES; ++s)
        if (s < fill) {
          const int64_t last = s + (int64_t)GT_STAGES * ((fill - 1 - s) / GT_STAGES);
          int zero = 0;
          mbar_wait(&sh->full[s], (uint32_t)((last / GT_STAGES) & 1), &zero);
        }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t ring_s = smem_u32(ring);
      const DescGen gK(ring_s, 16, 1024, SW_128B);
      const uint32_t idesc = idesc_bf16(128, N, 0, 0);
      const uint32_t a_rel = (a_box < 0) ? 0u : (uint32_t)(1 + a_box) * GT_BOX;
      int64_t fill = 0;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int buf = c & 1;
        if (!mbar_wait(&sh->cempty[buf], (uint32_t)(((c >> 1) & 1) ^ 1), abortp)) {
          gt_abort(sh, p.status);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 256);
        const int kbe = min(kb1, kb0 + (c + 1) * GT_CHUNK);
        for (int kb = kb0 + c * GT_CHUNK; kb < kbe; ++kb, ++fill) {
          const int s = (int)(fill % GT_STAGES);
          if (!mbar_wait(&sh->full[s], (uint32_t)((fill / GT_STAGES) & 1), abortp)) {
            gt_abort(sh, p.status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t soff = (uint32_t)s * GT_STAGE;
          const bool first = kb == kb0 + c * GT_CHUNK;
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4)
            mma_bf16(d, gK.at(soff + a_rel + 32 * k4), gK.at(soff + GT_BOX + 32 * k4), idesc,
                     (!first || k4 > 0) ? 1u : 0u);
          mma_commit(&sh->empty[s]);
        }
        mma_commit(&sh->cfull[buf]);
      }
      mma_commit(&sh->drain);
      int zero = 0;
      mbar_wait(&sh->drain, 0, &zero);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                       // TMEM lane quarter of this warp
    const int h = (warp - 2) >> 2;                // column half
    const int lrow = q * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      if (!mbar_wait(&sh->cfull[buf], (uint32_t)((c >> 1) & 1), abortp)) {
        gt_abort(sh, p.status);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + lane_addr + (uint32_t)(buf * 256 + h * 128);
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        if (h * 128 + g * 16 < N) {
          uint32_t r[16];
          tmem_ld16<0>(ta + (uint32_t)(g * 16), r);
          tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[g * 16 + t] += __uint_as_float(r[t]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh->cempty[buf]);
    }
    if (ok && !*abortp) {
      float* out = p.part + (size_t)blockIdx.x * (128 * 256) + (size_t)lrow * 256 + h * 128;
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (h * 128 + g * 16 < N) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            *reinterpret_cast<float4*>(out + g * 16 + 4 * v) =
                make_float4(acc[g * 16 + 4 * v], acc[g * 16 + 4 * v + 1], acc[g * 16 + 4 * v + 2],
                            acc[g * 16 + 4 * v + 3]);
        }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// G[i][j] = G[j][i] = sum over the splits of tile(i, j), i <= j, in split order.
__global__ void k_gram_tiles_reduce(const __grid_constant__ GtParams p, float* __restrict__ G) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < i || j >= p.m) return;
  const int I = i >> 7, J = j >> 8;
  const int t = p.tile_base[J] + I;
  const int2 ti = p.tile_items[t];
  const float* src = p.part + (size_t)ti.x * (128 * 256) + (size_t)(i - 128 * I) * 256 + (j - 256 * J);
  float s0 = 0.f, s1 = 0.f;
  int k = 0;
  for (; k + 2 <= ti.y; k += 2) {
    s0 += src[(size_t)k * (128 * 256)];
    s1 += src[(size_t)(k + 1) * (128 * 256)];
  }
  if (k < ti.y) s0 += src[(size_t)k * (128 * 256)];
  const float s = s0 + s1;
  G[(int64_t)i * p.m + j] = s;
  if (j != i) G[(int64_t)j * p.m + i] = s;
}

int num_sms_gram() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

// Tile list, per-tile split counts (proportional to each tile's per-k-box
// cost: bytes loaded or MMA width, whichever binds) and the work items.
bool gt_plan(int64_t m, int64_t n, GtParams& p) {
  std::memset(&p, 0, sizeof(p));
  p.m = m;
  p.n = n;
  p.nI = (int)ceil_div(m, 128);
  p.nJ = (int)ceil_div(m, 256);
  if (p.nJ > GT_MAX_J) return false;
  std::vector<double> cost;
  int t = 0;
  for (int J = 0; J < p.nJ; ++J) {
    p.tile_base[J] = t;
    const int rowsB = (int)imin(256, m - 256 * J);
    const int N = (rowsB + 15) / 16 * 16;
    const int nbB = (rowsB + 127) / 128;
    for (int I = 0; I < p.nI && I <= 2 * J + 1; ++I) {
      if (t >= GT_MAX_TILES) return false;
      const int a_box = (I == 2 * J || I == 2 * J + 1) ? I - 2 * J : -1;
      p.tile[t] = make_int4(I, J, N, nbB | ((a_box + 1) << 4));
      const double load = (double)((a_box < 0 ? 1 : 0) + nbB) / 3.0;
      cost.push_back(std::max(load, (double)N / 256.0));
      ++t;
    }
  }
  p.ntiles = t;
  const int64_t kboxes = ceil_div(n, 64);
  double total = 0;
  for (double c : cost) total += c;
  const int target = num_sms_gram();
  int items = 0;
  for (int i = 0; i < t; ++i) {
    int S = (int)std::max(1.0, std::floor(target * cost[i] / total));
    S = (int)imin(S, kboxes);
    if (items + S > GT_MAX_ITEMS) return false;
    p.tile_items[i] = make_int2(items, S);
    for (int s = 0; s < S; ++s) {
      const int kb0 = (int)(kboxes * s / S), kb1 = (int)(kboxes * (s + 1) / S);
      p.item[items++] = make_int4(i, kb0, kb1, 0);
    }
  }
  p.nitems = items;
  return true;
}

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;
std::mutex g_enc_mu;

cudaError_t map_rows128(CUtensorMap* map, const void* base, int64_t rows, int64_t cols) {
  {
    std::lock_guard<std::mutex> lk(g_enc_mu);
    if (!g_enc) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess) return e;
      if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
      g_enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {64u, 128u};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = g_enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ------------------------------------------------------------ SIMT Gram
constexpr int GS_T = 64;     // tile edge
constexpr int GS_K = 32;     // columns of C per smem chunk

// P[item] (64 x 64) = rows I of C times rows J of C, transposed, over the
// item's column range; tiles I <= J enumerated J-major.
template <typename TIn>
__global__ void __launch_bounds__(256) k_gram_simt_tiles(const TIn* __restrict__ C, int64_t m, int64_t n,
                                                         int splits, float* __restrict__ P) {
  __shared__ __align__(16) float As[GS_K][GS_T + 4];
  __shared__ __align__(16) float Bs[GS_K][GS_T + 4];
  const int item = blockIdx.x;
  const int t = item / splits, s = item % splits;
  int J = 0;
  while ((J + 1) * (J + 2) / 2 <= t) ++J;
  const int I = t - J * (J + 1) / 2;
  const int64_t chunks = ceil_div(n, GS_K);
  const int64_t c0 = chunks * s / splits * GS_K, c1 = imin(n, chunks * (s + 1) / splits * GS_K);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t ra = (int64_t)I * GS_T, rb = (int64_t)J * GS_T;
  float acc[4][4] = {};
  for (int64_t k0 = c0; k0 < c1; k0 += GS_K) {
    __syncthreads();
    for (int e = threadIdx.x; e < GS_T * GS_K; e += 256) {
      const int r = e / GS_K, kk = e % GS_K;
      const int64_t col = k0 + kk;
      As[kk][r] = (ra + r < m && col < c1) ? ld_elem(C, (ra + r) * n + col) : 0.f;
      Bs[kk][r] = (rb + r < m && col < c1) ? ld_elem(C, (rb + r) * n + col) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GS_K; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(av[u], bv[w], acc[u][w]);
    }
  }
  float* out = P + (size_t)item * GS_T * GS_T;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<float4*>(out + (4 * ty + u) * GS_T + 4 * tx) =
        make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
}

__global__ void k_gram_simt_reduce(const float* __restrict__ P, int64_t m, int splits, float* __restrict__ G) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < i || j >= m) return;
  const int I = i / GS_T, J = j / GS_T;
  const int t = J * (J + 1) / 2 + I;
  const float* src = P + (size_t)t * splits * GS_T * GS_T + (size_t)(i - GS_T * I) * GS_T + (j - GS_T * J);
  float s0 = 0.f, s1 = 0.f;
  int k = 0;
  for (; k + 2 <= splits; k += 2) {
    s0 += src[(size_t)k * GS_T * GS_T];
    s1 += src[(size_t)(k + 1) * GS_T * GS_T];
  }
  if (k < splits) s0 += src[(size_t)k * GS_T * GS_T];
  const float s = s0 + s1;
  G[(int64_t)i * m + j] = s;
  if (j != i) G[(int64_t)j * m + i] = s;
}

void gs_plan(int64_t m, int64_t n, int* tiles, int* splits) {
  const int nT = (int)ceil_div(m, GS_T);
  *tiles = nT * (nT + 1) / 2;
  const int64_t chunks = ceil_div(n, GS_K);
  const int want = (int)ceil_div(4 * (int64_t)num_sms_gram(), *tiles);
  *splits = (int)imax(1, imin(imin(want, chunks), 64));
}

// ------------------------------------------------------------ power W = G X
// X is a padded block (m x ldx, ldx % 4 == 0, 16-byte aligned), so both
// operands arrive by 16-byte asynchronous copies, GP_ST chunks of 128 rows of
// K in flight (the work per SM is small and latency decides it).  Each CTA
// owns 8 rows of W; a thread owns a 2 x 4 tile and one of KG groups that
// split each chunk, summed in group order at the end (fixed order).
constexpr int GP_RB = 8;      // rows of W per CTA
constexpr int GP_KC = 128;    // K chunk
constexpr int GP_ST = 4;      // chunks in flight
constexpr int GP_GLD = GP_KC + 4;

__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool ok) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4z(float* dst, const float* src, bool ok) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(256) k_gram_power(const float* __restrict__ G, int64_t m,
                                                    const float* __restrict__ X, int64_t ldx, int c,
                                                    float* __restrict__ W, int64_t ldw) {
  extern __shared__ __align__(16) float gp_sm[];
  const int CP = (c + 3) & ~3;
  const int tcq = CP / 4, ntl = (GP_RB / 2) * tcq;
  const int KG = 256 / ntl;
  float* Gs = gp_sm;                                  // [GP_ST][GP_RB][GP_GLD]
  float* Xs = Gs + GP_ST * GP_RB * GP_GLD;            // [GP_ST][GP_KC][CP]
  float* Rd = Xs + GP_ST * GP_KC * CP;                // [KG][GP_RB][CP]
  const int64_t r0 = (int64_t)blockIdx.x * GP_RB;
  const int tid = threadIdx.x;
  const int tl = tid % ntl, g = tid / ntl;
  const int rp = tl / tcq, cq = tl % tcq;
  const bool active = g < KG;
  const int64_t nchunks = ceil_div(m, GP_KC);
  const bool gvec = (m % 4) == 0 && (reinterpret_cast<uintptr_t>(G) % 16) == 0;
  auto load = [&](int64_t ch, int buf) {
    const int64_t k0 = ch * GP_KC;
    float* gs = Gs + buf * GP_RB * GP_GLD;
    float* xs = Xs + buf * GP_KC * CP;
    if (gvec) {
      for (int e = tid; e < GP_RB * (GP_KC / 4); e += 256) {
        const int r = e / (GP_KC / 4), k4 = (e % (GP_KC / 4)) * 4;
        const bool ok = r0 + r < m && k0 + k4 < m;   // m % 4 == 0: all four or none
        cp_async16z(gs + r * GP_GLD + k4, ok ? G + (r0 + r) * m + k0 + k4 : G, ok);
      }
    } else {
      for (int e = tid; e < GP_RB * GP_KC; e += 256) {
        const int r = e / GP_KC, kk = e % GP_KC;
        const bool ok = r0 + r < m && k0 + kk < m;
        cp_async4z(gs + r * GP_GLD + kk, ok ? G + (r0 + r) * m + k0 + kk : G, ok);
      }
    }
    for (int e = tid; e < GP_KC * tcq; e += 256) {
      const int kk = e / tcq, j4 = (e % tcq) * 4;
      const bool ok = k0 + kk < m;
      cp_async16z(xs + kk * CP + j4, ok ? X + (k0 + kk) * ldx + j4 : X, ok);
    }
    cp_commit();
  };
  float acc[2][4] = {};
  for (int64_t ch = 0; ch < GP_ST - 1; ++ch) {
    if (ch < nchunks) load(ch, (int)ch);
    else cp_commit();
  }
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int buf = (int)(ch % GP_ST);
    const int64_t nx = ch + GP_ST - 1;
    if (nx < nchunks) load(nx, (int)(nx % GP_ST));
    else cp_commit();
    cp_wait<GP_ST - 1>();
    __syncthreads();
    if (active) {
      const float* gs = Gs + buf * GP_RB * GP_GLD + (2 * rp) * GP_GLD;
      const float* xs = Xs + buf * GP_KC * CP + 4 * cq;
#pragma unroll 4
      for (int kk = g; kk < GP_KC; kk += KG) {
        const float4 x4 = *reinterpret_cast<const float4*>(xs + kk * CP);
        const float g0 = gs[kk], g1 = gs[GP_GLD + kk];
        acc[0][0] = fmaf(g0, x4.x, acc[0][0]); acc[0][1] = fmaf(g0, x4.y, acc[0][1]);
        acc[0][2] = fmaf(g0, x4.z, acc[0][2]); acc[0][3] = fmaf(g0, x4.w, acc[0][3]);
        acc[1][0] = fmaf(g1, x4.x, acc[1][0]); acc[1][1] = fmaf(g1, x4.y, acc[1][1]);
        acc[1][2] = fmaf(g1, x4.z, acc[1][2]); acc[1][3] = fmaf(g1, x4.w, acc[1][3]);
      }
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int u = 0; u < 2; ++u)
      *reinterpret_cast<float4*>(Rd + ((size_t)g * GP_RB + 2 * rp + u) * CP + 4 * cq) =
          make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  }
  __syncthreads();
  for (int e = tid; e < GP_RB * c; e += 256) {
    const int r = e / c, j = e % c;
    if (r0 + r >= m) continue;
    float s = 0.f;
    for (int gg = 0; gg < KG; ++gg) s += Rd[((size_t)gg * GP_RB + r) * CP + j];
    W[(r0 + r) * ldw + j] = s;
  }
}

size_t gp_smem_bytes(int c) {
  const int CP = (c + 3) & ~3;
  const int KG = 256 / ((GP_RB / 2) * (CP / 4));
  return sizeof(float) * ((size_t)GP_ST * GP_RB * GP_GLD + (size_t)GP_ST * GP_KC * CP + (size_t)KG * GP_RB * CP);
}

}  // namespace

// ------------------------------------------------------------ public launchers
bool gram_tiled_ok(int64_t m) { return m >= 1 && m <= 2048; }

bool gram_tc_tiled_ok(int64_t m, int64_t n) { return m > 128 && m <= 2048 && tc_shape_ok(m, n); }

size_t gram_tiled_partials(int64_t m, int64_t n, int c_bf16) {
  if (c_bf16 && gram_tc_tiled_ok(m, n)) {
    GtParams p;
    if (!gt_plan(m, n, p)) return 0;
    return (size_t)p.nitems * 128 * 256;
  }
  int tiles, splits;
  gs_plan(m, n, &tiles, &splits);
  return (size_t)tiles * splits * GS_T * GS_T;
}

cudaError_t gram_tiled(const void* C, int c_bf16, int64_t m, int64_t n, float* partials, float* G, int* status,
                       cudaStream_t st) {
  if (!gram_tiled_ok(m)) return cudaErrorInvalidValue;
  const double bytes = (double)m * n * (c_bf16 ? 2 : 4), flops = 2.0 * m * m * n;
  if (c_bf16 && gram_tc_tiled_ok(m, n)) {
    GtParams p;
    if (!gt_plan(m, n, p)) return cudaErrorInvalidValue;
    p.status = status;
    p.part = partials;
    CUtensorMap mc;
    cudaError_t e = map_rows128(&mc, C, m, n);
    if (e != cudaSuccess) return e;
    const size_t smem = 1024 + (size_t)GT_STAGES * GT_STAGE + sizeof(GtShared) + 64;
    e = raise_smem_limit(k_gram_tiles);
    if (e != cudaSuccess) return e;
    {
      ProfScope prof("gram_tc_tiled", st, bytes, flops);
      note_launch("gram_tc_tiled");
      k_gram_tiles<<<p.nitems, GT_THREADS, smem, st>>>(mc, p);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    note_launch("gram_reduce");
    k_gram_tiles_reduce<<<dim3((unsigned)ceil_div(m, 256), (unsigned)m), 256, 0, st>>>(p, G);
    return cudaGetLastError();
  }
  int tiles, splits;
  gs_plan(m, n, &tiles, &splits);
  {
    ProfScope prof("gram_simt_tiled", st, bytes, flops);
    note_launch("gram_simt_tiled");
    if (c_bf16)
      k_gram_simt_tiles<__nv_bfloat16><<<tiles * splits, 256, 0, st>>>((const __nv_bfloat16*)C, m, n, splits,
                                                                        partials);
    else
      k_gram_simt_tiles<float><<<tiles * splits, 256, 0, st>>>((const float*)C, m, n, splits, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  note_launch("gram_reduce");
  k_gram_simt_reduce<<<dim3((unsigned)ceil_div(m, 256), (unsigned)m), 256, 0, st>>>(partials, m, splits, G);
  return cudaGetLastError();
}

bool gram_power_ok(int64_t m, int c) { return m >= 1 && c >= 1 && c <= 64; }

// X must be 16-byte aligned with ldx % 4 == 0 (the caller's padded copy of
// the block).
cudaError_t gram_power(const float* G, int64_t m, const float* X, int64_t ldx, int c, float* W, int64_t ldw,
                       cudaStream_t st) {
  if (!gram_power_ok(m, c) || ldx % 4 != 0 || ldx < ((c + 3) & ~3) || reinterpret_cast<uintptr_t>(X) % 16 != 0)
    return cudaErrorInvalidValue;
  const size_t smem = gp_smem_bytes(c);
  cudaError_t e = raise_smem_limit(k_gram_power);
  if (e != cudaSuccess) return e;
  // G (at most 16 MB) is read from L2 by every power: no HBM bytes counted
  ProfScope prof("gram_power", st, 0.0, 2.0 * m * m * c);
  note_launch("gram_power");
  k_gram_power<<<(unsigned)ceil_div(m, GP_RB), 256, smem, st>>>(G, m, X, ldx, c, W, ldw);
  return cudaGetLastError();
}

}  // namespace ttr
