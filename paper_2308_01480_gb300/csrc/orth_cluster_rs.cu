// Orthonormalisation of one Krylov block against the basis, on one
// thread-block cluster (Alg. 3 step 5; Alg. 4 step 8 with an empty basis).
//
// The NC CTAs of the cluster (NC <= 16) own consecutive blocks of at most 64
// rows of the block Z and of the basis Q, and exchange only the b x b and
// kq x b block products: each CTA forms its share in shared memory, and the
// cluster sums the shares in rank order by a reduce-scatter (each CTA sums a
// slice over all ranks through distributed shared memory) and an all-gather,
// so every CTA holds identical sums and repeats the small factorisations
// itself.  The new block is appended to Q and, when asked, also written to a
// 16-byte-aligned padded buffer for the Gram-power product that follows.
//
// Sequence (BCGS2 and Cholesky QR, as in orth_cluster.cu with one reduction
// fewer): a block Gram-Schmidt projection against the basis, then a second
// projection whose reduction also forms the Gram for a shifted Cholesky QR
// (or, under the Krylov dimension cap, a greedy pivoted selection of the c
// kept columns), a Cholesky QR with a third projection, and a last Cholesky
// QR or first-order polar correction.
// A Cholesky pivot below 1e-6 of its diagonal marks its column.  The block
// (still spanning the same space: a marked pivot is replaced by 1, not
// dropped) is then orthonormalised once more as it stands, which settles
// weak but genuine directions of an ill-conditioned block; a column marked
// again lies numerically inside the span of the basis and the earlier
// columns, and is replaced by a deterministic pseudo-random vector before
// the next pass (at most twice), inside the same launch.  A column still
// marked after that records TT_EBREAKDOWN in the status.
#include <map>
#include <mutex>
#include <utility>

#include "chol.cuh"
#include "cluster_la.cuh"
#include "kernels.h"

namespace ttr {

namespace {

constexpr int KC_THREADS = 512;
constexpr int KC_MAX_ROWS = 64;
constexpr int KC_SMEM_MAX = 218 * 1024;

struct OrthRsArgs {
  const float* Y;       // the block, m x zc0, row stride ldy
  int64_t ldy;
  float* Q;             // basis, row stride ldq: columns [kq0, kq0 + c) written
  int64_t ldq;
  float* Xg;            // optional padded copy of the new block, m x xld
  int xld;
  int64_t m;
  int rows;             // rows per CTA
  int kq0;              // basis columns already in Q
  int zc0;              // columns of Y
  int c;                // columns kept
  int kqmax;            // kq0 + c
  int zmax;             // zc0
  int* status;
  uint64_t seed;
  // grid form only: per-rank shares (2 x nranks x E), sums (2 x E), barrier
  float* gparts;
  float* gsums;
  unsigned* gbar;
  int eslot;            // E: floats per share
};

struct KcLayout {
  int KP, ZP, RP;
  size_t share, slice, P, Gm, T, R, misc, Zc, Zn, Qc, tmp, total;
  int slice_len;
  int share_bufs;       // 2 for a cluster (other ranks read the shares), 1 for the grid form
};

// nc: cluster size; nc = 0 for the grid form (shares and sums in global
// memory, no slice buffers).
__host__ __device__ inline KcLayout kc_layout(int kqmax, int zmax, int rows, int nc) {
  KcLayout L;
  L.KP = pad4(kqmax);
  L.ZP = pad4(zmax);
  L.RP = pad4(rows);
  size_t o = 0;
  auto take = [&](size_t n) { size_t r = o; o += (n + 3) & ~size_t(3); return r; };
  L.share_bufs = nc > 0 ? 2 : 1;
  L.share = take((size_t)L.share_bufs * (L.KP + L.ZP) * L.ZP);
  L.slice_len = nc > 0 ? ((L.KP + L.ZP) * L.ZP + nc - 1) / nc + 4 : 0;
  L.slice = take(2 * (size_t)L.slice_len);
  L.P = take((size_t)L.KP * L.ZP);
  L.Gm = take((size_t)zmax * (zmax + 1));
  L.T = take((size_t)L.ZP * L.ZP);
  L.R = take((size_t)zmax * zmax);
  L.misc = take(256);
  L.Zc = take((size_t)L.RP * L.ZP);
  L.Zn = take((size_t)L.RP * L.ZP);
  L.Qc = take((size_t)L.RP * L.KP);
  L.tmp = take(8 * (size_t)L.ZP * L.ZP);   // split partial products of the Gram
  L.total = o;
  return L;
}

// Y[i][j] = scale * sum_{t < kk} X[i][t] M[t][j] (+ Y0[i][j]) for i < rows
// (multiple of 4), j < bp (multiple of 4), with TR x 4 register tiles so
// that short blocks still occupy every thread (row strides multiples of 4).
template <int TR>
__device__ void nn_rows(const float* X, int ldx, int kk, const float* M, int ldm, int rows, int bp, float* Y, int ldy,
                        const float* Y0, float scale) {
  const int ti = rows / TR, tj = bp >> 2;
  for (int tile = threadIdx.x; tile < ti * tj; tile += blockDim.x) {
    const int i0 = (tile / tj) * TR, j0 = (tile % tj) * 4;
    float acc[TR][4] = {};
    for (int t = 0; t < kk; ++t) {
      const float4 v = *reinterpret_cast<const float4*>(M + t * ldm + j0);
#pragma unroll
      for (int u = 0; u < TR; ++u) {
        const float x = X[(i0 + u) * ldx + t];
        acc[u][0] = fmaf(x, v.x, acc[u][0]); acc[u][1] = fmaf(x, v.y, acc[u][1]);
        acc[u][2] = fmaf(x, v.z, acc[u][2]); acc[u][3] = fmaf(x, v.w, acc[u][3]);
      }
    }
#pragma unroll
    for (int u = 0; u < TR; ++u) {
      float4 r = make_float4(acc[u][0] * scale, acc[u][1] * scale, acc[u][2] * scale, acc[u][3] * scale);
      if (Y0) {
        const float4 y = *reinterpret_cast<const float4*>(Y0 + (i0 + u) * ldy + j0);
        r.x += y.x; r.y += y.y; r.z += y.z; r.w += y.w;
      }
      *reinterpret_cast<float4*>(Y + (i0 + u) * ldy + j0) = r;
    }
  }
}

__device__ __forceinline__ void nn_any(const float* X, int ldx, int kk, const float* M, int ldm, int rows, int bp,
                                       float* Y, int ldy, const float* Y0, float scale) {
  const int t4 = (rows / 4) * (bp / 4);
  if (2 * t4 >= (int)blockDim.x) nn_rows<4>(X, ldx, kk, M, ldm, rows, bp, Y, ldy, Y0, scale);
  else if (4 * t4 >= (int)blockDim.x || (rows & 3)) nn_rows<2>(X, ldx, kk, M, ldm, rows, bp, Y, ldy, Y0, scale);
  else nn_rows<1>(X, ldx, kk, M, ldm, rows, bp, Y, ldy, Y0, scale);
}

// out[t][j] = sum_{i < rows} A[i][t] B[i][j] (t < ta, j < bp, multiples of 4)
// with the rows split over KS groups of threads when there are few output
// tiles; the KS partial tiles (in tmp) are summed in group order.  Ends
// with a __syncthreads().
__device__ void tn_split(const float* A, int lda, int ta, const float* B, int ldb, int bp, int rows, float* out,
                         int ldo, float* tmp) {
  const int tt = ta >> 2, tj = bp >> 2, tiles = tt * tj;
  const int KS = imax(1, imin(8, (int)blockDim.x / tiles));
  if (KS == 1) {
    tn_tile(A, lda, ta, B, ldb, bp, rows, out, ldo);
    __syncthreads();
    return;
  }
  const int tid = threadIdx.x;
  if (tid < tiles * KS) {
    const int tile = tid % tiles, g = tid / tiles;
    const int t0 = (tile / tj) * 4, j0 = (tile % tj) * 4;
    float acc[4][4] = {};
    for (int i = g; i < rows; i += KS) {
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
      *reinterpret_cast<float4*>(tmp + ((size_t)g * ta + t0 + u) * bp + j0) =
          make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  }
  __syncthreads();
  for (int e = tid; e < ta * bp; e += blockDim.x) {
    float sacc = 0.f;
    for (int g = 0; g < KS; ++g) sacc += tmp[(size_t)g * ta * bp + e];
    out[(e / bp) * ldo + (e % bp)] = sacc;
  }
  __syncthreads();
}

// The ranks of one cluster: shares summed through distributed shared memory.
struct ClusterComm {
  cg::cluster_group cl;
  float* slices;        // two buffers of slice_len floats
  int slice_len;
  __device__ int nranks() { return (int)cl.num_blocks(); }
  __device__ int rank() { return (int)cl.block_rank(); }
  template <typename Put>
  __device__ void reduce(float* mine, int phase, int e0, int e1, Put& put) {
    cl.sync();
    cluster_reduce_scatter_gather(cl, mine, slices + (size_t)(phase & 1) * slice_len, e0, e1, put);
  }
  __device__ void finish() { cl.sync(); }   // no CTA leaves while others may read its shares
};

// Barrier over all CTAs of a cooperative launch (every CTA resident): an
// arrival counter and a generation word in global memory.  The wait gives up
// after about two seconds, records TT_ETIMEOUT and marks the CTA dead, after
// which its barriers return at once (results are then garbage, the status
// says so).
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned n, int* status, int* dead) {
  __syncthreads();
  if (threadIdx.x == 0 && !*dead) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == n - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint64_t t0 = 0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (*gen == g) {
        uint64_t t = 0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) {
          set_status(status, TT_ETIMEOUT);
          *dead = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// All CTAs of a cooperative launch: each writes its share to global memory,
// CTA q sums the slice [q S, q S + S) over the ranks in rank order (the
// ranks split over thread groups, the group partials added in group order),
// and every CTA reads all sums back.
struct GridComm {
  int nr, rk;
  float* parts;         // two buffers of nr x E floats
  float* sums;          // two buffers of E floats
  int E;
  unsigned* bar;
  int* status;
  int* dead;            // shared-memory flag
  float* tmp;           // shared scratch, at least blockDim.x floats
  __device__ int nranks() { return nr; }
  __device__ int rank() { return rk; }
  template <typename Put>
  __device__ void reduce(float* mine, int phase, int e0, int e1, Put& put) {
    float* P = parts + (size_t)(phase & 1) * nr * E;
    float* S = sums + (size_t)(phase & 1) * E;
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) __stcg(P + (size_t)rk * E + e, mine[e]);
    grid_barrier(bar, nr, status, dead);
    const int n = e1 - e0, sl = (n + nr - 1) / nr;
    const int s0 = e0 + rk * sl, ns = max(0, min(e1, s0 + sl) - s0);
    if (2 * ns > (int)blockDim.x) {
      for (int x = threadIdx.x; x < ns; x += blockDim.x) {
        float acc = 0.f;
        for (int q = 0; q < nr; ++q) acc += __ldcg(P + (size_t)q * E + s0 + x);
        __stcg(S + s0 + x, acc);
      }
    } else if (ns > 0) {
      const int groups = min(nr, (int)blockDim.x / ns);   // >= 2
      const int t = threadIdx.x, el = t % ns, g = t / ns;
      if (g < groups) {
        float acc = 0.f;
        for (int q = g; q < nr; q += groups) acc += __ldcg(P + (size_t)q * E + s0 + el);
        tmp[g * ns + el] = acc;
      }
      __syncthreads();
      for (int x = threadIdx.x; x < ns; x += blockDim.x) {
        float acc = 0.f;
        for (int q = 0; q < groups; ++q) acc += tmp[q * ns + x];
        __stcg(S + s0 + x, acc);
      }
    }
    grid_barrier(bar, nr, status, dead);
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) put(e, __ldcg(S + e));
  }
  __device__ void finish() {}
};

template <class Comm>
__device__ __forceinline__ void orth_rs_body(const OrthRsArgs& a, Comm& comm, float* sm, const KcLayout& L,
                                             unsigned long long& badmask) {
  const int tid = threadIdx.x;
  const int KP = L.KP, ZP = L.ZP, RP = L.RP;
  const unsigned rank = (unsigned)comm.rank();
  const int64_t r0 = (int64_t)rank * a.rows;
  const int rc = (int)imax(0, imin(a.rows, a.m - r0));
  float* share0 = sm + L.share;
  float* P = sm + L.P;
  float* Gm = sm + L.Gm;
  float* T = sm + L.T;
  float* R = sm + L.R;
  float* diag0 = sm + L.misc;
  float* red = diag0 + 64;
  int* perm = reinterpret_cast<int*>(red + 64);
  float* dsw = red + 128;
  float* Zc = sm + L.Zc;
  float* Zn = sm + L.Zn;
  float* Qc = sm + L.Qc;
  float* tmp = sm + L.tmp;        // split partial products (orthonormalisation)

  // prologue: the CTA's rows of the existing basis and of the first block
  // (zero padded), all copies in flight together
  {
    const int lane = tid & 31, nw = blockDim.x >> 5;
    for (int i = tid >> 5; i < RP; i += nw) {
      const bool row_ok = i < rc;
      const float* qrow = row_ok ? a.Q + (r0 + i) * a.ldq : a.Q;
      const float* yrow = row_ok ? a.Y + (r0 + i) * a.ldy : a.Y;
      for (int t = lane; t < KP; t += 32) {
        const bool ok = row_ok && t < a.kq0;
        cp_async4(&Qc[i * KP + t], ok ? qrow + t : a.Q, ok);
      }
      for (int j = lane; j < ZP; j += 32) {
        const bool ok = row_ok && j < a.zc0;
        cp_async4(&Zc[i * ZP + j], ok ? yrow + j : a.Y, ok);
        Zn[i * ZP + j] = 0.f;
      }
    }
    cp_async_wait_all();
  }
  for (int x = tid; x < ZP * ZP; x += blockDim.x) T[x] = 0.f;
  for (int x = tid; x < KP * ZP; x += blockDim.x) P[x] = 0.f;
  __syncthreads();

  int phase = 0;
  // Orthonormalises the zc columns of Zc against Qc[:, :kq], keeping c
  // columns; the result is in Zc[:, :c] (columns c..ZP zero).
  auto orth = [&](int kq, int zc, int c, int bidx) {
    for (int attempt = 0; attempt < 4; ++attempt) {
      const int kp = pad4(kq), bz = pad4(zc);
      const int E = (kp + bz) * bz;
      if (tid == 0) badmask = 0ull;
      __syncthreads();
      auto reduce = [&](bool qz, bool zz) {
        float* mine = share0 + (size_t)(L.share_bufs == 2 ? (phase & 1) : 0) * (KP + ZP) * ZP;
        if (qz) tn_tile(Qc, KP, kp, Zc, ZP, bz, RP, mine, bz);
        if (zz) tn_split(Zc, ZP, bz, Zc, ZP, bz, RP, mine + kp * bz, bz, tmp);
        __syncthreads();
        const int e0 = qz ? 0 : kp * bz, e1 = zz ? E : kp * bz;
        auto put = [&](int e, float s) {
          const int row = e / bz, j = e % bz;
          if (row < kp) P[e] = s;
          else if (row - kp < zc && j < zc) Gm[(row - kp) * (zc + 1) + j] = s;
        };
        comm.reduce(mine, phase, e0, e1, put);
        __syncthreads();
        ++phase;
      };
      auto swap = [&]() { float* t = Zc; Zc = Zn; Zn = t; };
      auto sub_q = [&]() {     // Z = Z - Q P
        nn_any(Qc, KP, kp, P, bz, RP, bz, Zn, ZP, Zc, -1.f);
        __syncthreads();
        swap();
      };
      auto mul_t = [&]() {     // Z = Z T
        nn_any(Zc, ZP, bz, T, bz, RP, bz, Zn, ZP, nullptr, 1.f);
        __syncthreads();
        swap();
      };
      auto set_diag0 = [&]() {
        for (int i = tid; i < zc; i += blockDim.x) diag0[i] = Gm[i * (zc + 1) + i];
        __syncthreads();
      };
      auto factor = [&](int bc) {
        for (int x = tid; x < bz * bz; x += blockDim.x) T[x] = 0.f;
        __syncthreads();
        chol_inv_fast(Gm, zc + 1, bc, diag0, R, zc, T, bz, nullptr, false, &badmask);
      };
      if (kq > 0) {
        reduce(true, false);                     // A
        sub_q();
      }
      for (int pass = 0; pass < 3; ++pass) {     // B+C, D, E
        // pass 0 also forms the second projection Q^T Z; the Gram of
        // Z - Q P then differs from Z^T Z by P^T P, second order in the
        // rounding-level P and far below the shift
        reduce((pass == 0 || pass == 1) && kq > 0, true);
        set_diag0();
        if (pass == 0) {
          float tr = 0.f;
          for (int i = tid; i < zc; i += blockDim.x) tr += Gm[i * (zc + 1) + i];
          tr = block_sum(tr, red);
          const float shift = 11.f * ((float)a.m * zc + (float)zc * (zc + 1)) * 5.9604645e-08f * tr;
          __syncthreads();
          for (int i = tid; i < zc; i += blockDim.x) Gm[i * (zc + 1) + i] += shift;
        }
        bool polar = false;
        if (pass == 2) {
          float e = 0.f;
          for (int x = tid; x < c * c; x += blockDim.x) {
            const int i = x / c, j = x % c;
            e = fmaxf(e, fabsf(Gm[i * (zc + 1) + j] - (i == j ? 1.f : 0.f)));
          }
          e = warp_max(e);
          __syncthreads();
          if ((tid & 31) == 0) red[tid >> 5] = e;
          __syncthreads();
          e = warp_max((tid & 31) < (int)(blockDim.x >> 5) ? red[tid & 31] : 0.f);
          polar = e < 1e-4f;
          if (polar) {
            for (int x = tid; x < bz * bz; x += blockDim.x) {
              const int i = x / bz, j = x % bz;
              T[x] = (i < c && j < c) ? (i == j ? 1.5f : 0.f) - 0.5f * Gm[i * (zc + 1) + j] : 0.f;
            }
            __syncthreads();
          }
        }
        if (pass == 0 && c < zc)
          pchol_select_cta(Gm, zc + 1, zc, c, diag0, R, zc, T, bz, bz, perm, dsw, nullptr, false, &badmask);
        else if (!polar)
          factor(pass == 0 ? zc : c);
        if (pass <= 1 && kq > 0) sub_q();
        mul_t();
      }
      __syncthreads();
      const unsigned long long bad = badmask;
      if (bad == 0ull) return;
      if (attempt == 3) {
        if (rank == 0 && tid == 0) set_status(a.status, DEV_BREAKDOWN);
        return;
      }
      if (attempt >= 1) {
        // marked again: replace those columns by pseudo-random vectors
        for (int x = tid; x < rc * c; x += blockDim.x) {
          const int i = x / c, j = x % c;
          if ((bad >> j) & 1ull)
            Zc[i * ZP + j] = hash_uniform(a.seed ^ ((uint64_t)(bidx * 64 + j) << 40) ^ ((uint64_t)attempt << 58),
                                          (uint64_t)(r0 + i));
        }
        __syncthreads();
      }
      zc = c;
    }
  };

  const int c = a.c, base = a.kq0;
  orth(a.kq0, a.zc0, c, 0);
  for (int x = tid; x < rc * c; x += blockDim.x) {
    const int i = x / c, t = x % c;
    a.Q[(r0 + i) * a.ldq + base + t] = Zc[i * ZP + t];
  }
  if (a.Xg) {
    const int bzc = pad4(c);
    for (int x = tid; x < rc * bzc; x += blockDim.x) {
      const int i = x / bzc, t = x % bzc;
      a.Xg[(r0 + i) * a.xld + t] = (t < c) ? Zc[i * ZP + t] : 0.f;
    }
  }
  comm.finish();
}

__global__ void __launch_bounds__(KC_THREADS, 1) k_orth_cluster_rs(const __grid_constant__ OrthRsArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ unsigned long long badmask;
  ClusterComm comm{cg::this_cluster(), nullptr, 0};
  const KcLayout L = kc_layout(a.kqmax, a.zmax, a.rows, comm.nranks());
  comm.slices = sm + L.slice;
  comm.slice_len = L.slice_len;
  orth_rs_body(a, comm, sm, L, badmask);
}

// The same sequence over all CTAs of a cooperative launch, for blocks with
// more rows than one cluster holds; the shares go through global memory.
__global__ void __launch_bounds__(KC_THREADS, 1) k_orth_grid_rs(const __grid_constant__ OrthRsArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ unsigned long long badmask;
  __shared__ int dead;
  __shared__ float gtmp[KC_THREADS];
  if (threadIdx.x == 0) dead = 0;
  __syncthreads();
  GridComm comm{(int)gridDim.x, (int)blockIdx.x, a.gparts, a.gsums, a.eslot, a.gbar, a.status, &dead, gtmp};
  const KcLayout L = kc_layout(a.kqmax, a.zmax, a.rows, 0);
  orth_rs_body(a, comm, sm, L, badmask);
}

}  // namespace

// ------------------------------------------------------------ launcher
namespace {

struct KcConfig {
  int nc = 0, rows = 0;
  size_t smem = 0;
};

bool kc_config(int64_t m, int kqmax, int zmax, KcConfig* cfg) {
  if (m < 1 || zmax < 1 || zmax > 64 || kqmax > 256) return false;
  int nc = 1;
  while (nc < 16 && ceil_div(m, nc) > KC_MAX_ROWS) nc *= 2;
  const int64_t rows = ceil_div(m, nc);
  if (rows > KC_MAX_ROWS) return false;
  const KcLayout L = kc_layout(kqmax, zmax, (int)rows, nc);
  const size_t smem = L.total * sizeof(float);
  if (smem > (size_t)KC_SMEM_MAX) return false;
  cfg->nc = nc;
  cfg->rows = (int)rows;
  cfg->smem = smem;
  return true;
}

// Whether the device can hold one cluster of nc CTAs with this shared memory.
bool kc_schedulable(int nc, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, bool> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev * 64 + nc, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  bool ok = false;
  if (raise_smem_limit(k_orth_cluster_rs) == cudaSuccess &&
      cudaFuncSetAttribute(k_orth_cluster_rs, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc);
    cfg.blockDim = dim3(KC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    ok = cudaOccupancyMaxActiveClusters(&clusters, k_orth_cluster_rs, &cfg) == cudaSuccess && clusters > 0;
  }
  cudaGetLastError();
  cache[key] = ok;
  return ok;
}

// Grid form: one CTA per SM at most (every CTA of the cooperative launch
// resident), at least 16 rows each.
struct KgConfig {
  int nr = 0, rows = 0, E = 0;
  size_t smem = 0;
};

int kg_device_ctas() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 0;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) sms = 0;
  cudaGetLastError();
  cache[dev] = sms;
  return sms;
}

bool kg_config(int64_t m, int kqmax, int zmax, KgConfig* cfg) {
  if (m < 1 || zmax < 1 || zmax > 64 || kqmax > 256) return false;
  const int maxr = kg_device_ctas();
  if (maxr < 1) return false;
  const int64_t nr0 = imin((int64_t)maxr, imax((int64_t)1, ceil_div(m, 16)));
  const int64_t rows = ceil_div(m, nr0);
  const KcLayout L = kc_layout(kqmax, zmax, (int)rows, 0);
  const size_t smem = L.total * sizeof(float);
  if (smem > (size_t)KC_SMEM_MAX) return false;
  cfg->rows = (int)rows;
  cfg->nr = (int)ceil_div(m, rows);
  cfg->E = (L.KP + L.ZP) * L.ZP;
  cfg->smem = smem;
  return true;
}

}  // namespace

bool orth_grid_rs_ok(int64_t m, int kq0, int zc, int c) {
  KgConfig cfg;
  return c >= 1 && c <= zc && kg_config(m, kq0 + c, zc, &cfg);
}

size_t orth_grid_rs_scratch_floats(int64_t m, int kq0, int zc) {
  KgConfig cfg;
  if (!kg_config(m, kq0 + zc, zc, &cfg)) return 0;
  return 4 + 2 * (size_t)cfg.nr * cfg.E + 2 * (size_t)cfg.E;
}

cudaError_t launch_orth_grid_rs(const float* Y, int64_t ldy, int zc, int64_t m, int c, int kq0, float* Q,
                                int64_t ldq, float* Xg, int xld, uint64_t seed, float* scratch, int* status,
                                cudaStream_t st) {
  if (c < 1 || c > zc || (Xg && xld < pad4(c)) || !scratch) return cudaErrorInvalidValue;
  OrthRsArgs a = {};
  a.Y = Y; a.ldy = ldy; a.Q = Q; a.ldq = ldq; a.Xg = Xg; a.xld = xld; a.m = m;
  a.kq0 = kq0; a.zc0 = zc; a.c = c; a.status = status; a.seed = seed;
  a.kqmax = kq0 + c;
  a.zmax = zc;
  KgConfig cfg;
  if (!kg_config(m, a.kqmax, zc, &cfg)) return cudaErrorInvalidValue;
  a.rows = cfg.rows;
  a.eslot = cfg.E;
  a.gbar = reinterpret_cast<unsigned*>(scratch);
  a.gparts = scratch + 4;
  a.gsums = a.gparts + 2 * (size_t)cfg.nr * cfg.E;
  cudaError_t e = raise_smem_limit(k_orth_grid_rs);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.gbar, 0, 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.nr);
  lc.blockDim = dim3(KC_THREADS);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  ProfScope prof("orth_grid", st, 0, 0);
  note_launch("orth_grid");
  e = cudaLaunchKernelEx(&lc, k_orth_grid_rs, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

bool orth_cluster_rs_ok(int64_t m, int kq0, int zc, int c) {
  KcConfig cfg;
  return c >= 1 && c <= zc && kc_config(m, kq0 + c, zc, &cfg);
}

cudaError_t launch_orth_cluster_rs(const float* Y, int64_t ldy, int zc, int64_t m, int c, int kq0, float* Q,
                                  int64_t ldq, float* Xg, int xld, uint64_t seed, int* status, cudaStream_t st) {
  if (c < 1 || c > zc || (Xg && xld < pad4(c))) return cudaErrorInvalidValue;
  OrthRsArgs a = {};
  a.Y = Y; a.ldy = ldy; a.Q = Q; a.ldq = ldq; a.Xg = Xg; a.xld = xld; a.m = m;
  a.kq0 = kq0; a.zc0 = zc; a.c = c; a.status = status; a.seed = seed;
  a.kqmax = kq0 + c;
  a.zmax = zc;
  KcConfig cfg;
  if (!kc_config(m, a.kqmax, zc, &cfg)) return cudaErrorInvalidValue;
  if (!kc_schedulable(cfg.nc, cfg.smem)) return cudaErrorNotSupported;
  a.rows = cfg.rows;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.nc);
  lc.blockDim = dim3(KC_THREADS);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cfg.nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  ProfScope prof("orth_cluster", st, 0, 0);
  note_launch("orth_cluster");
  cudaError_t e = cudaLaunchKernelEx(&lc, k_orth_cluster_rs, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ttr
