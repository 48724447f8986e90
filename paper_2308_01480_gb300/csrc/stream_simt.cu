// CUDA-core (SIMT) streaming passes over an unfolding C (m x n, row-major).
//
// These are the plain FP32 form of the four passes of Alg. 3 (and the form
// used for shapes the tensor-core kernels do not cover):
//   proj  : S = X^T C              (Alg. 3 step 10, and the first half of a
//                                   Krylov power for tall unfoldings)
//   cs    : Y = C S^T              (Alg. 3 step 4: the sketch C W with
//                                   S = W^T, or the second half of a power)
//   ga    : Y = C (C^T X)          (Alg. 3 step 4: one Krylov power, fused so
//                                   each column tile of C is read once)
//   gram  : G = C C^T              (exhaustion route: all of R^m is Krylov)
// Reductions over n are split across CTAs into per-CTA partials that a
// second kernel sums in a fixed order, so results are bit-reproducible.
#include "common.cuh"
#include "kernels.h"

namespace ttr {

// ---------------------------------------------------------------- proj
// S[c][col] = sum_i X[i][c] C[i][col];  256 threads = 16 (cols) x 16 (c).
// With gridDim.y > 1 each CTA row covers rows [y * rows_per, ...) and writes
// its partial sums to S + y * split_stride (the tall-thin form).
template <typename TIn, typename TOut, int VB>
__global__ void __launch_bounds__(256) k_proj(const TIn* __restrict__ C, int64_t m, int64_t n,
                                              const float* __restrict__ X, int ldx, int b,
                                              TOut* __restrict__ S, int64_t lds, int64_t rows_per,
                                              int64_t split_stride) {
  constexpr int TN = 64, RC = 32;
  __shared__ float Cs[RC][TN];
  __shared__ float Xs[RC][16 * VB];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t col0 = (int64_t)blockIdx.x * TN;
  const int64_t rbeg = (int64_t)blockIdx.y * rows_per;
  const int64_t rend = imin(m, rbeg + rows_per);
  S += (int64_t)blockIdx.y * split_stride;
  float acc[VB][4];
#pragma unroll
  for (int v = 0; v < VB; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[v][u] = 0.f;
  constexpr int NC = RC * TN / 256, NX = RC * 16 * VB / 256;   // tile entries per thread
  for (int64_t i0 = rbeg; i0 < rend; i0 += RC) {
    // every load of the chunk in flight before the first store
    float cl[NC], xl[NX];
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      const int e = threadIdx.x + 256 * u, r = e / TN, c = e % TN;
      const int64_t gi = i0 + r, gc = col0 + c;
      cl[u] = (gi < rend && gc < n) ? ld_elem(C, gi * n + gc) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int e = threadIdx.x + 256 * u, r = e / (16 * VB), c = e % (16 * VB);
      const int64_t gi = i0 + r;
      xl[u] = (gi < rend && c < b) ? X[gi * ldx + c] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      const int e = threadIdx.x + 256 * u;
      Cs[e / TN][e % TN] = cl[u];
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int e = threadIdx.x + 256 * u;
      Xs[e / (16 * VB)][e % (16 * VB)] = xl[u];
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < RC; ++r) {
      float cv[4], xv[VB];
#pragma unroll
      for (int u = 0; u < 4; ++u) cv[u] = Cs[r][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < VB; ++v) xv[v] = Xs[r][ty + 16 * v];
#pragma unroll
      for (int v = 0; v < VB; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[v][u] = fmaf(xv[v], cv[u], acc[v][u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < VB; ++v) {
    int c = ty + 16 * v;
    if (c >= b) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int64_t gc = col0 + tx + 16 * u;
      if (gc < n) st_elem(S, (int64_t)c * lds + gc, acc[v][u]);
    }
  }
}

// ---------------------------------------------------------------- cs
// P[split][i][c] = sum_{col in split} C[i][col] S[c][col] for the CTA's
// 32-row tile; grid = (row tiles, splits).
template <typename TIn, int VB>
__global__ void __launch_bounds__(256) k_cs(const TIn* __restrict__ C, int64_t m, int64_t n,
                                            const float* __restrict__ S, int64_t lds, int b,
                                            float* __restrict__ P, int64_t cols_per_split) {
  constexpr int TN = 64, RM = 32;
  __shared__ float Cs[RM][TN + 1];
  __shared__ float Ss[16 * VB][TN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * RM;
  const int64_t cbeg = (int64_t)blockIdx.y * cols_per_split;
  const int64_t cend = min(n, cbeg + cols_per_split);
  float acc[2][VB];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int v = 0; v < VB; ++v) acc[a][v] = 0.f;
  for (int64_t c0 = cbeg; c0 < cend; c0 += TN) {
    for (int e = threadIdx.x; e < RM * TN; e += 256) {
      int r = e / TN, c = e % TN;
      int64_t gi = row0 + r, gc = c0 + c;
      Cs[r][c] = (gi < m && gc < cend) ? ld_elem(C, gi * n + gc) : 0.f;
    }
    for (int e = threadIdx.x; e < 16 * VB * TN; e += 256) {
      int r = e / TN, c = e % TN;
      int64_t gc = c0 + c;
      Ss[r][c] = (r < b && gc < cend) ? S[(int64_t)r * lds + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < TN; ++t) {
      float ci[2], sv[VB];
#pragma unroll
      for (int a = 0; a < 2; ++a) ci[a] = Cs[ty + 16 * a][t];
#pragma unroll
      for (int v = 0; v < VB; ++v) sv[v] = Ss[tx + 16 * v][t];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int v = 0; v < VB; ++v) acc[a][v] = fmaf(ci[a], sv[v], acc[a][v]);
    }
    __syncthreads();
  }
  float* out = P + (int64_t)blockIdx.y * m * b;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int64_t i = row0 + ty + 16 * a;
    if (i >= m) continue;
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      int c = tx + 16 * v;
      if (c < b) out[i * b + c] = acc[a][v];
    }
  }
}

// ---------------------------------------------------------------- ga (fused)
// P[cta] = sum over the CTA's column tiles C_j (C_j^T X), m <= 256, b <= 48.
// Each 32-column tile of C is loaded once into shared memory and used by both
// products.  Accumulator rows i = ty + 16 a, columns c = tx + 16 v.
template <typename TIn, int MA, int VB>
__global__ void __launch_bounds__(256) k_ga_fused(const TIn* __restrict__ C, int64_t m, int64_t n,
                                                  const float* __restrict__ X, int ldx, int b,
                                                  float* __restrict__ P, int64_t tiles_per_cta) {
  constexpr int TN = 32;
  constexpr int MP = 16 * MA;            // padded row count
  constexpr int BP = 16 * VB;            // padded column count
  extern __shared__ float sm[];
  float* Cs = sm;                        // [MP][TN + 1]
  float* Xs = Cs + MP * (TN + 1);        // [MP][BP + 1]
  float* Ts = Xs + MP * (BP + 1);        // [TN][BP + 1]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int e = threadIdx.x; e < MP * BP; e += 256) {
    int r = e / BP, c = e % BP;
    Xs[r * (BP + 1) + c] = (r < m && c < b) ? X[(int64_t)r * ldx + c] : 0.f;
  }
  float acc[MA][VB];
#pragma unroll
  for (int a = 0; a < MA; ++a)
#pragma unroll
    for (int v = 0; v < VB; ++v) acc[a][v] = 0.f;
  const int64_t ntiles = (n + TN - 1) / TN;
  const int64_t t_beg = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t t_end = min(ntiles, t_beg + tiles_per_cta);
  for (int64_t tile = t_beg; tile < t_end; ++tile) {
    const int64_t c0 = tile * TN;
    __syncthreads();
    for (int e = threadIdx.x; e < MP * TN; e += 256) {
      int r = e / TN, c = e % TN;
      int64_t gc = c0 + c;
      Cs[r * (TN + 1) + c] = (r < m && gc < n) ? ld_elem(C, (int64_t)r * n + gc) : 0.f;
    }
    __syncthreads();
    // T[t][c] = sum_i C[i][t] X[i][c]; thread -> t = tx + 16 u (u < 2), c = ty + 16 v
    {
      float tacc[2][VB];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < VB; ++v) tacc[u][v] = 0.f;
      for (int i = 0; i < MP; ++i) {
        float cv0 = Cs[i * (TN + 1) + tx], cv1 = Cs[i * (TN + 1) + tx + 16];
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          float xv = Xs[i * (BP + 1) + ty + 16 * v];
          tacc[0][v] = fmaf(cv0, xv, tacc[0][v]);
          tacc[1][v] = fmaf(cv1, xv, tacc[1][v]);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < VB; ++v) Ts[(tx + 16 * u) * (BP + 1) + ty + 16 * v] = tacc[u][v];
    }
    __syncthreads();
    // acc[i][c] += sum_t C[i][t] T[t][c]
#pragma unroll 4
    for (int t = 0; t < TN; ++t) {
      float tv[VB];
#pragma unroll
      for (int v = 0; v < VB; ++v) tv[v] = Ts[t * (BP + 1) + tx + 16 * v];
#pragma unroll
      for (int a = 0; a < MA; ++a) {
        float cv = Cs[(ty + 16 * a) * (TN + 1) + t];
#pragma unroll
        for (int v = 0; v < VB; ++v) acc[a][v] = fmaf(cv, tv[v], acc[a][v]);
      }
    }
  }
  float* out = P + (int64_t)blockIdx.x * m * b;
#pragma unroll
  for (int a = 0; a < MA; ++a) {
    int i = ty + 16 * a;
    if (i >= m) continue;
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      int c = tx + 16 * v;
      if (c < b) out[(int64_t)i * b + c] = acc[a][v];
    }
  }
}

// ---------------------------------------------------------------- gram
// P[cta] = sum over the CTA's column tiles C_j C_j^T, m <= 128.
template <typename TIn, int MA>
__global__ void __launch_bounds__(256) k_gram(const TIn* __restrict__ C, int64_t m, int64_t n,
                                              float* __restrict__ P, int64_t tiles_per_cta) {
  constexpr int TN = 32, MP = 16 * MA;
  __shared__ float Cs[MP][TN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[MA][MA];
#pragma unroll
  for (int a = 0; a < MA; ++a)
#pragma unroll
    for (int l = 0; l < MA; ++l) acc[a][l] = 0.f;
  const int64_t ntiles = (n + TN - 1) / TN;
  const int64_t t_beg = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t t_end = min(ntiles, t_beg + tiles_per_cta);
  for (int64_t tile = t_beg; tile < t_end; ++tile) {
    const int64_t c0 = tile * TN;
    __syncthreads();
    for (int e = threadIdx.x; e < MP * TN; e += 256) {
      int r = e / TN, c = e % TN;
      int64_t gc = c0 + c;
      Cs[r][c] = (r < m && gc < n) ? ld_elem(C, (int64_t)r * n + gc) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < TN; ++t) {
      float ci[MA], cj[MA];
#pragma unroll
      for (int a = 0; a < MA; ++a) ci[a] = Cs[ty + 16 * a][t];
#pragma unroll
      for (int l = 0; l < MA; ++l) cj[l] = Cs[tx + 16 * l][t];
#pragma unroll
      for (int a = 0; a < MA; ++a)
#pragma unroll
        for (int l = 0; l < MA; ++l) acc[a][l] = fmaf(ci[a], cj[l], acc[a][l]);
    }
  }
  float* out = P + (int64_t)blockIdx.x * m * m;
#pragma unroll
  for (int a = 0; a < MA; ++a) {
    int i = ty + 16 * a;
    if (i >= m) continue;
#pragma unroll
    for (int l = 0; l < MA; ++l) {
      int j = tx + 16 * l;
      if (j < m) out[(int64_t)i * m + j] = acc[a][l];
    }
  }
}

// ---------------------------------------------------------------- reduce
// out[r * ldo + c] = sum_{s < S} P[s][r][c] (fixed order), r < rows, c < cols.
// A block takes 32 consecutive elements (lane = element, each load of a warp
// one 128-byte row of a partial); warp w sums the partials w, w + 8, ... in
// four interleaved chains, and the eight warp sums are added in a fixed
// tree: every element sees the same order whatever the grid, so reruns are
// bit-identical, and a short element range still spreads over eight warps.
constexpr int RED_WARPS = 8;

__device__ __forceinline__ float strided_sum_warp(const float* __restrict__ p, int n, int64_t stride, int w) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int k = w;
  for (; k + 3 * RED_WARPS < n; k += 4 * RED_WARPS) {
    a0 += p[(int64_t)k * stride];
    a1 += p[(int64_t)(k + RED_WARPS) * stride];
    a2 += p[(int64_t)(k + 2 * RED_WARPS) * stride];
    a3 += p[(int64_t)(k + 3 * RED_WARPS) * stride];
  }
  for (; k < n; k += RED_WARPS) a0 += p[(int64_t)k * stride];
  return (a0 + a1) + (a2 + a3);
}

// base(e) + k * stride is partial k of element e (k < n); out[e] = the sum.
template <typename Base>
__device__ __forceinline__ void reduce_elements(Base base, int n, int64_t stride, int64_t E, int cols,
                                                float* __restrict__ out, int64_t ldo) {
  __shared__ float red[RED_WARPS][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < E; e0 += (int64_t)gridDim.x * 32) {
    const int64_t e = e0 + lane;
    red[w][lane] = (e < E) ? strided_sum_warp(base(e), n, stride, w) : 0.f;
    __syncthreads();
    if (w == 0 && e < E) {
      const float t = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                      ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
      out[(e / cols) * ldo + e % cols] = t;
    }
    __syncthreads();
  }
}

struct PartialsFlat {
  const float* P;
  __device__ const float* operator()(int64_t e) const { return P + e; }
};
struct PartialsGrouped {   // element e's row group g = e / cols / group_rows starts at slot g
  const float* P;
  int64_t E, cols, group_rows;
  __device__ const float* operator()(int64_t e) const { return P + (e / cols / group_rows) * E + e; }
};

__global__ void __launch_bounds__(32 * RED_WARPS) k_reduce_partials(const float* __restrict__ P, int S, int64_t rows,
                                                                    int cols, float* __restrict__ out, int64_t ldo) {
  const int64_t E = rows * cols;
  reduce_elements(PartialsFlat{P}, S, E, E, cols, out, ldo);
}

// out[r][c] = sum over the CTAs of r's row group (slot j * groups + g) of
// their partials; the CTAs of a group write only that group's rows.
__global__ void __launch_bounds__(32 * RED_WARPS) k_reduce_grouped(const float* __restrict__ P, int per, int groups,
                                                                   int64_t rows, int cols, int64_t group_rows,
                                                                   float* __restrict__ out, int64_t ldo) {
  const int64_t E = rows * cols;
  reduce_elements(PartialsGrouped{P, E, cols, group_rows}, per, (int64_t)groups * E, E, cols, out, ldo);
}

// ======================================================================
// Launchers
// ======================================================================
static int target_ctas() { return 4 * 152; }

static void reduce_launch(const float* P, int S, int64_t rows, int cols, float* out, int64_t ldo,
                          cudaStream_t st) {
  int64_t E = rows * cols;
  int blocks = (int)imin(ceil_div(E, 32), 4096);
  k_reduce_partials<<<blocks, 32 * RED_WARPS, 0, st>>>(P, S, rows, cols, out, ldo);
  note_launch("reduce_partials");
}

cudaError_t launch_reduce_partials(const float* P, int S, int64_t rows, int cols, float* out, int64_t ldo,
                                   cudaStream_t st) {
  reduce_launch(P, S, rows, cols, out, ldo, st);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials_grouped(const float* P, int per, int groups, int64_t rows, int cols,
                                           int64_t group_rows, float* out, int64_t ldo, cudaStream_t st) {
  const int64_t E = rows * cols;
  note_launch("reduce_partials");
  k_reduce_grouped<<<(int)imin(ceil_div(E, 32), 4096), 32 * RED_WARPS, 0, st>>>(P, per, groups, rows, cols,
                                                                                group_rows, out, ldo);
  return cudaGetLastError();
}

// S (b x n) = sum over row splits of the partials P[y] (b x n), fixed order.
template <typename TOut>
__global__ void k_sum_splits(const float* __restrict__ P, int splits, int b, int64_t n, TOut* __restrict__ S,
                             int64_t lds) {
  const int64_t E = (int64_t)b * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    // eight loads in flight, added in split order
    float acc = 0.f;
    int y = 0;
    for (; y + 8 <= splits; y += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = P[(int64_t)(y + u) * E + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; y < splits; ++y) acc += P[(int64_t)y * E + e];
    st_elem(S, (e / n) * lds + e % n, acc);
  }
}

// Row splits of the tall-thin form: 32 rows (one tile chunk) per CTA, at most
// 64 splits.
int64_t simt_proj_splits(int64_t m, int64_t n) {
  if (n > 512 || m < 256) return 1;
  return imin(ceil_div(m, 32), 64);
}

template <typename TIn, typename TOut>
cudaError_t simt_proj(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b, TOut* S,
                      int64_t lds, cudaStream_t st, float* partials) {
  const int64_t splits = partials ? simt_proj_splits(m, n) : 1;
  if (splits > 1) {
    // tall-thin unfolding: rows split across CTAs, then a fixed-order sum
    const int64_t rows_per = ceil_div(m, splits);
    dim3 grid((unsigned)ceil_div(n, 64), (unsigned)splits);
    ProfScope prof("proj_simt", st, (double)m * n * sizeof(TIn) + (double)m * b * 4 + (double)b * n * sizeof(TOut),
                   2.0 * m * n * b);
    note_launch("proj_simt", 2);
#define TTR_PS(VB) k_proj<TIn, float, VB><<<grid, 256, 0, st>>>(C, m, n, X, ldx, b, partials, n, rows_per, (int64_t)b * n)
    if (b <= 16) TTR_PS(1); else if (b <= 32) TTR_PS(2); else if (b <= 48) TTR_PS(3); else if (b <= 64) TTR_PS(4);
    else return cudaErrorInvalidValue;
#undef TTR_PS
    const int64_t E = (int64_t)b * n;
    k_sum_splits<TOut><<<(int)imin(ceil_div(E, 256), 256), 256, 0, st>>>(partials, (int)splits, b, n, S, lds);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)ceil_div(n, 64));
  ProfScope prof("proj_simt", st, (double)m * n * sizeof(TIn) + (double)m * b * 4 + (double)b * n * sizeof(TOut),
                 2.0 * m * n * b);
  note_launch("proj_simt");
  if (b <= 16)
    k_proj<TIn, TOut, 1><<<grid, 256, 0, st>>>(C, m, n, X, ldx, b, S, lds, m, 0);
  else if (b <= 32)
    k_proj<TIn, TOut, 2><<<grid, 256, 0, st>>>(C, m, n, X, ldx, b, S, lds, m, 0);
  else if (b <= 48)
    k_proj<TIn, TOut, 3><<<grid, 256, 0, st>>>(C, m, n, X, ldx, b, S, lds, m, 0);
  else if (b <= 64)
    k_proj<TIn, TOut, 4><<<grid, 256, 0, st>>>(C, m, n, X, ldx, b, S, lds, m, 0);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int64_t simt_cs_splits(int64_t m, int64_t n) {
  int64_t rt = ceil_div(m, 32);
  int64_t s = imax(1, target_ctas() / rt);
  s = imin(s, imax(1, ceil_div(n, 256)));
  return s;
}

template <typename TIn>
cudaError_t simt_cs(const TIn* C, int64_t m, int64_t n, const float* S, int64_t lds, int b,
                    float* partials, float* out, int64_t ldo, cudaStream_t st) {
  int64_t splits = simt_cs_splits(m, n);
  int64_t per = ceil_div(ceil_div(n, 64), splits) * 64;
  dim3 grid((unsigned)ceil_div(m, 32), (unsigned)splits);
  {
  ProfScope prof("cs_simt", st, (double)m * n * sizeof(TIn) + (double)b * n * 4, 2.0 * m * n * b);
  note_launch("cs_simt");
  if (b <= 16)
    k_cs<TIn, 1><<<grid, 256, 0, st>>>(C, m, n, S, lds, b, partials, per);
  else if (b <= 32)
    k_cs<TIn, 2><<<grid, 256, 0, st>>>(C, m, n, S, lds, b, partials, per);
  else if (b <= 48)
    k_cs<TIn, 3><<<grid, 256, 0, st>>>(C, m, n, S, lds, b, partials, per);
  else if (b <= 64)
    k_cs<TIn, 4><<<grid, 256, 0, st>>>(C, m, n, S, lds, b, partials, per);
  else
    return cudaErrorInvalidValue;
  }
  reduce_launch(partials, (int)splits, m, b, out, ldo, st);
  return cudaGetLastError();
}

int64_t simt_tiles_split(int64_t n, int64_t tn) {
  int64_t tiles = ceil_div(n, tn);
  int64_t ctas = imin(tiles, target_ctas());
  return ceil_div(tiles, ctas);   // tiles per CTA
}

template <typename TIn, int MA, int VB>
static void ga_launch(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b, float* P,
                      int64_t tpc, int ctas, cudaStream_t st) {
  size_t smem = sizeof(float) * ((16 * MA) * 33 + (16 * MA) * (16 * VB + 1) + 32 * (16 * VB + 1));
  auto kern = k_ga_fused<TIn, MA, VB>;
  raise_smem_limit(kern);
  kern<<<ctas, 256, smem, st>>>(C, m, n, X, ldx, b, P, tpc);
}

template <typename TIn, int VB>
static cudaError_t ga_dispatch_m(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b,
                                 float* P, int64_t tpc, int ctas, cudaStream_t st) {
  int ma = (int)ceil_div(m, 16);
  switch (ma) {
#define TTR_GA_CASE(K) \
  case K: ga_launch<TIn, K, VB>(C, m, n, X, ldx, b, P, tpc, ctas, st); break;
    TTR_GA_CASE(1) TTR_GA_CASE(2) TTR_GA_CASE(3) TTR_GA_CASE(4) TTR_GA_CASE(5) TTR_GA_CASE(6)
    TTR_GA_CASE(7) TTR_GA_CASE(8) TTR_GA_CASE(9) TTR_GA_CASE(10) TTR_GA_CASE(11) TTR_GA_CASE(12)
    TTR_GA_CASE(13) TTR_GA_CASE(14) TTR_GA_CASE(15) TTR_GA_CASE(16)
#undef TTR_GA_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

bool simt_ga_fused_ok(int64_t m, int b) { return m <= 256 && b <= 48 && ceil_div(m, 16) * ceil_div(b, 16) <= 48; }

template <typename TIn>
cudaError_t simt_ga(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b,
                    float* partials, float* out, int64_t ldo, cudaStream_t st) {
  if (!simt_ga_fused_ok(m, b)) return cudaErrorInvalidValue;
  int64_t tpc = simt_tiles_split(n, 32);
  int ctas = (int)ceil_div(ceil_div(n, 32), tpc);
  cudaError_t e;
  {
  ProfScope prof("gram_apply_simt", st, (double)m * n * sizeof(TIn) + (double)m * b * 4, 4.0 * m * n * b);
  note_launch("gram_apply_simt");
  if (b <= 16)
    e = ga_dispatch_m<TIn, 1>(C, m, n, X, ldx, b, partials, tpc, ctas, st);
  else if (b <= 32)
    e = ga_dispatch_m<TIn, 2>(C, m, n, X, ldx, b, partials, tpc, ctas, st);
  else
    e = ga_dispatch_m<TIn, 3>(C, m, n, X, ldx, b, partials, tpc, ctas, st);
  }
  if (e != cudaSuccess) return e;
  reduce_launch(partials, ctas, m, b, out, ldo, st);
  return cudaGetLastError();
}

// Fused Gram-apply with at most max_ctas CTAs, so that the partials fit a
// caller-given buffer of max_ctas * m * b floats.
template <typename TIn>
cudaError_t simt_ga_with_ctas(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b,
                              float* partials, int64_t max_ctas, float* out, int64_t ldo, cudaStream_t st) {
  if (!simt_ga_fused_ok(m, b) || max_ctas < 1) return cudaErrorInvalidValue;
  const int64_t tiles = ceil_div(n, 32);
  const int64_t ctas0 = imin(imin(tiles, target_ctas()), max_ctas);
  const int64_t tpc = ceil_div(tiles, ctas0);
  const int ctas = (int)ceil_div(tiles, tpc);
  cudaError_t e;
  {
    ProfScope prof("gram_apply_simt", st, (double)m * n * sizeof(TIn) + (double)m * b * 4, 4.0 * m * n * b);
    note_launch("gram_apply_simt");
    if (b <= 16)
      e = ga_dispatch_m<TIn, 1>(C, m, n, X, ldx, b, partials, tpc, ctas, st);
    else if (b <= 32)
      e = ga_dispatch_m<TIn, 2>(C, m, n, X, ldx, b, partials, tpc, ctas, st);
    else
      e = ga_dispatch_m<TIn, 3>(C, m, n, X, ldx, b, partials, tpc, ctas, st);
  }
  if (e != cudaSuccess) return e;
  reduce_launch(partials, ctas, m, b, out, ldo, st);
  return cudaGetLastError();
}
template cudaError_t simt_ga_with_ctas<float>(const float*, int64_t, int64_t, const float*, int, int, float*, int64_t, float*, int64_t, cudaStream_t);
template cudaError_t simt_ga_with_ctas<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t, const float*, int, int, float*, int64_t, float*, int64_t, cudaStream_t);

int64_t simt_ga_partials(int64_t m, int64_t n, int b) {
  int64_t tpc = simt_tiles_split(n, 32);
  return ceil_div(ceil_div(n, 32), tpc) * m * b;
}
int64_t simt_cs_partials(int64_t m, int64_t n, int b) { return simt_cs_splits(m, n) * m * b; }
int64_t simt_gram_partials(int64_t m, int64_t n) {
  int64_t tpc = simt_tiles_split(n, 32);
  return ceil_div(ceil_div(n, 32), tpc) * m * m;
}

template <typename TIn>
cudaError_t simt_gram(const TIn* C, int64_t m, int64_t n, float* partials, float* out, cudaStream_t st) {
  int64_t tpc = simt_tiles_split(n, 32);
  int ctas = (int)ceil_div(ceil_div(n, 32), tpc);
  int ma = (int)ceil_div(m, 16);
  {
  ProfScope prof("gram_simt", st, (double)m * n * sizeof(TIn), 2.0 * m * m * n);
  note_launch("gram_simt");
  switch (ma) {
#define TTR_GR_CASE(K) \
  case K: k_gram<TIn, K><<<ctas, 256, 0, st>>>(C, m, n, partials, tpc); break;
    TTR_GR_CASE(1) TTR_GR_CASE(2) TTR_GR_CASE(3) TTR_GR_CASE(4) TTR_GR_CASE(5) TTR_GR_CASE(6)
    TTR_GR_CASE(7) TTR_GR_CASE(8)
#undef TTR_GR_CASE
    default: return cudaErrorInvalidValue;
  }
  }
  reduce_launch(partials, ctas, m, (int)m, out, m, st);
  return cudaGetLastError();
}

// Explicit instantiations.
template cudaError_t simt_proj<float, float>(const float*, int64_t, int64_t, const float*, int, int, float*, int64_t, cudaStream_t, float*);
template cudaError_t simt_proj<float, __nv_bfloat16>(const float*, int64_t, int64_t, const float*, int, int, __nv_bfloat16*, int64_t, cudaStream_t, float*);
template cudaError_t simt_proj<__nv_bfloat16, float>(const __nv_bfloat16*, int64_t, int64_t, const float*, int, int, float*, int64_t, cudaStream_t, float*);
template cudaError_t simt_proj<__nv_bfloat16, __nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t, const float*, int, int, __nv_bfloat16*, int64_t, cudaStream_t, float*);
template cudaError_t simt_cs<float>(const float*, int64_t, int64_t, const float*, int64_t, int, float*, float*, int64_t, cudaStream_t);
template cudaError_t simt_cs<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t, const float*, int64_t, int, float*, float*, int64_t, cudaStream_t);
template cudaError_t simt_ga<float>(const float*, int64_t, int64_t, const float*, int, int, float*, float*, int64_t, cudaStream_t);
template cudaError_t simt_ga<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t, const float*, int, int, float*, float*, int64_t, cudaStream_t);
template cudaError_t simt_gram<float>(const float*, int64_t, int64_t, float*, float*, cudaStream_t);
template cudaError_t simt_gram<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t, float*, float*, cudaStream_t);

}  // namespace ttr
