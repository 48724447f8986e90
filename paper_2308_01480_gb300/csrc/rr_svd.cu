// Rayleigh-Ritz through the singular vectors of B = Q^T C without squaring
// them in single precision (Alg. 3 steps 6-8, option accurate_rr).
//
// The default Rayleigh-Ritz forms H = Q^T C C^T Q from the FP32 powers and
// takes its eigenvectors in FP32: H holds squared singular values, so a
// direction with sigma_j / sigma_1 below about sqrt(u) = 2.4e-4 drowns in
// the rounding of H.  Here B = Q^T C (k x n) is projected in FP32 (its
// error is u ||C||, not u ||C||^2), and
//   1. H = B B^T is accumulated with exact FP32 products (p = a b plus
//      fma(a, b, -p)) and compensated sums (double-FP32 pairs over 256
//      columns at a time), the pairs summed in FP64 in a fixed order: H is
//      accurate to ~64 u^2 ||B||^2;
//   2. P H P^T = L L^T by a Cholesky factorisation in FP64 with diagonal
//      pivoting, stopped at a pivot below 64 eps max H_ii (one CTA);
//   3. L, rounded to FP32 (error u ||L|| = u sigma_1, again unsquared), is
//      diagonalised by one-sided Jacobi in FP32: rotations of column pairs
//      until every pair is orthogonal to u, so L J = Y Sigma with Y the left
//      singular vectors of L, i.e. the eigenvectors of H, and Sigma the
//      singular values of B;
//   4. U = Q Y[:, top r] (or Y itself when Q is the identity, the
//      exhaustion route).
// A factorisation stopped at numerical rank j (B rank-deficient to working
// accuracy) leaves zero columns in L and zero singular values; a wanted
// vector whose singular value is zero is completed by Gram-Schmidt against
// the others from unit vectors, so U stays orthonormal.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace ttr {

namespace {

constexpr int DF_TILE = 16;         // output tile of H per CTA (16 x 16, one entry per thread)
constexpr int DF_CHUNK = 64;        // columns of B staged per step
constexpr int DF_FLUSH = 4;         // chunks between flushes of the FP32 pairs into FP64
constexpr int RS_THREADS = 512;

// s (hi, lo) += a b with the product exact and the sum compensated.  The
// _rn intrinsics keep the compiler from contracting a b + hi into one FMA,
// which would break the error terms' exactness.
__device__ __forceinline__ void df_fma(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  const float t = __fadd_rn(hi, p);
  const float bb = __fsub_rn(t, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

// Upper-triangle tiles (I <= J) of the k x k output, I-major.
__host__ __device__ inline int df_tiles(int k) {
  const int t = (k + DF_TILE - 1) / DF_TILE;
  return t * (t + 1) / 2;
}
__device__ inline void df_tile_ij(int idx, int k, int& I, int& J) {
  const int t = (k + DF_TILE - 1) / DF_TILE;
  int i = 0;
  while (idx >= t - i) { idx -= t - i; ++i; }
  I = i;
  J = i + idx;
}

template <typename T>
__device__ __forceinline__ float df_ld(const T* p) {
  if constexpr (sizeof(T) == 2) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  else return *p;
}

// partials[item] (16 x 16 doubles) for item = tile * splits + split: the
// tile's entries summed over the split's columns [c0, c1).
template <typename T>
__global__ void __launch_bounds__(256) k_gram_df(const T* __restrict__ B, int k, int64_t n, int64_t ldb, int splits,
                                                 double* __restrict__ partials) {
  __shared__ float As[DF_TILE][DF_CHUNK + 1];
  __shared__ float Bs[DF_TILE][DF_CHUNK + 1];
  const int tile = blockIdx.x / splits, split = blockIdx.x % splits;
  int I, J;
  df_tile_ij(tile, k, I, J);
  const int64_t per = (n + splits - 1) / splits;
  const int64_t c0 = (int64_t)split * per, c1 = c0 + per < n ? c0 + per : n;
  const int tid = threadIdx.x, ti = tid / DF_TILE, tj = tid % DF_TILE;
  // four interleaved compensated pairs (columns c mod 4, independent
  // dependency chains), flushed into an FP64 total every DF_FLUSH chunks:
  // lo itself rounds in FP32, so over n_c terms its error grows like
  // n_c u^2 |H|, which for n_c in the tens of thousands reaches the squared
  // tail singular values; a period of 64 terms a chain keeps it near
  // 64 u^2 |H| (the FP64 adds run at a small fraction of the FP32 rate,
  // hence the period of several chunks)
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
  double tot = 0.0;
  int pending = 0;
  for (int64_t cb = c0; cb < c1; cb += DF_CHUNK) {
    for (int x = tid; x < 2 * DF_TILE * DF_CHUNK; x += blockDim.x) {
      const int which = x / (DF_TILE * DF_CHUNK), rr = (x / DF_CHUNK) % DF_TILE, cc = x % DF_CHUNK;
      const int row = (which ? J : I) * DF_TILE + rr;
      const int64_t col = cb + cc;
      const float v = (row < k && col < c1) ? df_ld(B + (int64_t)row * ldb + col) : 0.f;
      if (which) Bs[rr][cc] = v;
      else As[rr][cc] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < DF_CHUNK; c += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) df_fma(As[ti][c + u], Bs[tj][c + u], hi[u], lo[u]);
    }
    __syncthreads();
    if (++pending == DF_FLUSH) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        tot += (double)hi[u] + (double)lo[u];
        hi[u] = 0.f;
        lo[u] = 0.f;
      }
      pending = 0;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) tot += (double)hi[u] + (double)lo[u];
  partials[(size_t)blockIdx.x * DF_TILE * DF_TILE + tid] = tot;
}

// H (k x k doubles, both triangles) from the partials, splits in order.
__global__ void k_gram_df_reduce(const double* __restrict__ partials, int k, int splits, double* __restrict__ H) {
  const int tile = blockIdx.x;
  int I, J;
  df_tile_ij(tile, k, I, J);
  const int tid = threadIdx.x, ti = tid / DF_TILE, tj = tid % DF_TILE;
  double s = 0.0;
  for (int q = 0; q < splits; ++q) s += partials[((size_t)tile * splits + q) * DF_TILE * DF_TILE + tid];
  const int i = I * DF_TILE + ti, j = J * DF_TILE + tj;
  if (i < k && j < k) {
    H[(size_t)i * k + j] = s;
    H[(size_t)j * k + i] = s;
  }
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (lane < nw) ? red[lane] : 0.0;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// Shared memory: packed lower triangle of H / L in FP64, k (k + 1) / 2
// doubles; W = L^T rows (k x ldw floats, ldw = k | 1); order, sigma.
__host__ __device__ inline size_t rs_smem_bytes(int k) {
  const size_t tri = (size_t)k * (k + 1) / 2 * sizeof(double);
  const size_t w = (((size_t)k * (size_t)(k | 1) + 1) & ~(size_t)1) * sizeof(float);
  return tri + w + 64 * sizeof(double) + 2 * (size_t)k * sizeof(float) + 3 * (size_t)k * sizeof(int) + 64 +
         64 * 64 * sizeof(float);   // the kept vectors' Gram (r <= 64)
}

__global__ void __launch_bounds__(RS_THREADS, 1)
k_rr_svd(const double* __restrict__ Hg, int k, int r, const float* __restrict__ Q, int64_t m, int64_t ldq,
         float* __restrict__ U, float* __restrict__ core, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* Lp = reinterpret_cast<double*>(smraw);                      // packed lower, row i at i (i + 1) / 2
  const int ldw = k | 1;
  float* Wt = reinterpret_cast<float*>(Lp + (size_t)k * (k + 1) / 2);   // Wt[j][i] = W[i][j] (column j of W)
  double* redd = reinterpret_cast<double*>(Wt + (((size_t)k * ldw + 1) & ~(size_t)1));   // [64], 8-byte aligned
  float* sig = reinterpret_cast<float*>(redd + 64);                     // [k]
  float* tmpv = sig + k;                                                // [k]
  int* order = reinterpret_cast<int*>(tmpv + k);                        // [k]
  int* perm = order + k;                                                // [k] pivot order: row i of L is H's perm[i]
  int* iperm = perm + k;                                                // [k] its inverse
  float* Gs = reinterpret_cast<float*>(iperm + k + 16);                 // [r][r]
  __shared__ int s_rot, s_piv;
  __shared__ double s_pval, s_tol;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5, NW = RS_THREADS / 32;
  for (int i = ty; i < k; i += NW)
    for (int t = lane; t <= i; t += 32) Lp[(size_t)i * (i + 1) / 2 + t] = Hg[(size_t)i * k + t];
  for (int i = tid; i < k; i += RS_THREADS) perm[i] = i;
  if (ty == 0) {
    double dm = 0.0;
    for (int i = lane; i < k; i += 32) dm = fmax(dm, Hg[(size_t)i * k + i]);
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) s_tol = 64.0 * DBL_EPSILON * dm;
  }
  __syncthreads();
  // 2. Cholesky P H P^T = L L^T in FP64, right-looking, column by column,
  // with diagonal pivoting: H is semidefinite to working accuracy (its
  // trailing eigenvalues are rounding), and an unpivoted factorisation that
  // meets a pivot of rounding size divides rounding by its square root,
  // which fills L with entries of order sigma_1.  The largest remaining
  // diagonal is taken instead, and the factorisation stops once it falls
  // below 64 eps max_i H_ii (the rest of L is zero: a numerical rank of j).
  const double tol = s_tol;
  for (int j = 0; j < k; ++j) {
    if (ty == 0) {
      double bv = -1.0;
      int bi = j;
      for (int i = j + lane; i < k; i += 32) {
        const double d = Lp[(size_t)i * (i + 1) / 2 + i];
        if (d > bv) { bv = d; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) { s_piv = bi; s_pval = bv; }
    }
    __syncthreads();
    const int pv = s_piv;
    if (!(s_pval > tol)) {
      for (int i = j + ty; i < k; i += NW)
        for (int c = j + lane; c <= i; c += 32) Lp[(size_t)i * (i + 1) / 2 + c] = 0.0;
      __syncthreads();
      break;
    }
    if (pv != j) {
      // symmetric swap of indices j < pv in the packed lower triangle (the
      // computed columns of L swap rows; (pv, j) stays)
      const size_t rp = (size_t)pv * (pv + 1) / 2, rj0 = (size_t)j * (j + 1) / 2;
      for (int t = tid; t < k; t += RS_THREADS) {
        size_t a, b;
        if (t < j) { a = rj0 + t; b = rp + t; }
        else if (t == j) { a = rj0 + j; b = rp + pv; }
        else if (t < pv) { a = (size_t)t * (t + 1) / 2 + j; b = rp + t; }
        else if (t > pv) { a = (size_t)t * (t + 1) / 2 + j; b = (size_t)t * (t + 1) / 2 + pv; }
        else continue;
        const double va = Lp[a];
        Lp[a] = Lp[b];
        Lp[b] = va;
      }
      if (tid == 0) { const int tp = perm[j]; perm[j] = perm[pv]; perm[pv] = tp; }
      __syncthreads();
    }
    const size_t rj = (size_t)j * (j + 1) / 2;
    const double djj = Lp[rj + j];
    const double ljj = djj > 0.0 ? sqrt(djj) : 0.0;
    const double inv = ljj > 0.0 ? 1.0 / ljj : 0.0;
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += RS_THREADS) Lp[(size_t)i * (i + 1) / 2 + j] *= inv;
    if (tid == 0) Lp[rj + j] = ljj;
    __syncthreads();
    // trailing update: L[i][l] -= L[i][j] L[l][j], j < l <= i (a warp per row)
    for (int i = j + 1 + ty; i < k; i += NW) {
      const size_t ri = (size_t)i * (i + 1) / 2;
      const double lij = Lp[ri + j];
      for (int l = j + 1 + lane; l <= i; l += 32) Lp[ri + l] = fma(-lij, Lp[(size_t)l * (l + 1) / 2 + j], Lp[ri + l]);
    }
    __syncthreads();
  }
  for (int i = tid; i < k; i += RS_THREADS) iperm[perm[i]] = i;
  // 3. W = L in FP32, stored by columns: Wt[c][i] = L[i][c] (i >= c)
  for (int x = tid; x < k * k; x += RS_THREADS) {
    const int c = x / k, i = x % k;
    Wt[(size_t)c * ldw + i] = (i >= c) ? (float)Lp[(size_t)i * (i + 1) / 2 + c] : 0.f;
  }
  __syncthreads();
  // one-sided Jacobi on the columns of W: round-robin pairs, a warp per pair
  const int K = (k + 1) & ~1, half = K / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < K - 1; ++rnd) {
      for (int j = ty; j < half; j += NW) {
        int p = (j == 0) ? 0 : 1 + (rnd + j) % (K - 1);
        int q = (j == 0) ? 1 + rnd % (K - 1) : 1 + (rnd - j + (K - 1)) % (K - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= k) continue;
        float* wp = Wt + (size_t)p * ldw;
        float* wq = Wt + (size_t)q * ldw;
        // the norms have no cancellation; the inner product does, and an
        // FP32 sum of k products would carry k u |w_p||w_q| of rounding, far
        // above the 1.2e-7 test: it is accumulated compensated
        float al = 0.f, be = 0.f, ghi = 0.f, glo = 0.f;
        for (int i = lane; i < k; i += 32) {
          const float x = wp[i], y = wq[i];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          df_fma(x, y, ghi, glo);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          const float oh = __shfl_xor_sync(0xffffffffu, ghi, o);
          const float ol = __shfl_xor_sync(0xffffffffu, glo, o);
          const float t = __fadd_rn(ghi, oh), bb = __fsub_rn(t, ghi);
          glo = __fadd_rn(glo, __fadd_rn(ol, __fadd_rn(__fsub_rn(ghi, __fsub_rn(t, bb)), __fsub_rn(oh, bb))));
          ghi = t;
        }
        const float ga = ghi + glo;
        if (fabsf(ga) > 1.2e-7f * sqrtf(al * be) && fabsf(ga) > FLT_MIN) {
          const float ze = (be - al) / (2.f * ga);
          const float t = copysignf(1.f, ze) / (fabsf(ze) + sqrtf(fmaf(ze, ze, 1.f)));
          const float c = rsqrtf(fmaf(t, t, 1.f)), s = c * t;
          for (int i = lane; i < k; i += 32) {
            const float x = wp[i], y = wq[i];
            wp[i] = fmaf(c, x, -s * y);
            wq[i] = fmaf(s, x, c * y);
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  // singular values (column norms) and the descending order
  for (int c = ty; c < k; c += NW) {
    float s = 0.f;
    for (int i = lane; i < k; i += 32) s = fmaf(Wt[(size_t)c * ldw + i], Wt[(size_t)c * ldw + i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sig[c] = sqrtf(s);
  }
  __syncthreads();
  for (int t = tid; t < k; t += RS_THREADS) {
    const float st = sig[t];
    int rank = 0;
    for (int s2 = 0; s2 < k; ++s2) {
      const float ss = sig[s2];
      rank += (ss > st) || (ss == st && s2 < t);
    }
    order[rank] = t;
  }
  __syncthreads();
  // Y columns (normalised W columns) in place; a zero one is completed by
  // Gram-Schmidt from unit vectors against the earlier ones
  const float smax = sig[order[0]];
  for (int jj = 0; jj < r; ++jj) {
    float* y = Wt + (size_t)order[jj] * ldw;
    const float sj = sig[order[jj]];
    if (sj > 1e-30f && sj > 1e-30f * smax) {
      const float inv = 1.f / sj;
      for (int i = tid; i < k; i += RS_THREADS) y[i] *= inv;
      __syncthreads();
      continue;
    }
    for (int e = 0; e < k; ++e) {
      for (int i = tid; i < k; i += RS_THREADS) y[i] = (i == e) ? 1.f : 0.f;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int j2 = ty; j2 < jj; j2 += NW) {
          const float* z = Wt + (size_t)order[j2] * ldw;
          float d = 0.f;
          for (int i = lane; i < k; i += 32) d = fmaf(z[i], y[i], d);
          for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          if (lane == 0) tmpv[j2] = d;
        }
        __syncthreads();
        for (int i = tid; i < k; i += RS_THREADS) {
          float v = y[i];
          for (int j2 = 0; j2 < jj; ++j2) v = fmaf(-tmpv[j2], Wt[(size_t)order[j2] * ldw + i], v);
          y[i] = v;
        }
        __syncthreads();
      }
      double nn = 0.0;
      for (int i = tid; i < k; i += RS_THREADS) nn += (double)y[i] * y[i];
      nn = block_sum_d(nn, redd);
      if (nn > 0.25) {
        const float inv = (float)(1.0 / sqrt(nn));
        for (int i = tid; i < k; i += RS_THREADS) y[i] *= inv;
        __syncthreads();
        break;
      }
      __syncthreads();
    }
  }
  // the kept vectors' Jacobi rotations stop at the FP32 dot accuracy: one
  // first-order polar step, Y <- Y (3 I - Y^T Y) / 2, makes them orthonormal
  // to second order (the new columns are staged where L was)
  float* Yn = reinterpret_cast<float*>(Lp);                             // [r][k]
  for (int x = ty; x < r * r; x += NW) {
    const int a = x / r, b2 = x % r;
    const float* ya = Wt + (size_t)order[a] * ldw;
    const float* yb = Wt + (size_t)order[b2] * ldw;
    float dsum = 0.f;
    for (int i = lane; i < k; i += 32) dsum = fmaf(ya[i], yb[i], dsum);
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lane == 0) Gs[a * r + b2] = (a == b2 ? 1.5f : 0.f) - 0.5f * dsum;
  }
  __syncthreads();
  for (int x = tid; x < r * k; x += RS_THREADS) {
    const int j = x / k, i = x % k;
    float acc = 0.f;
    for (int l = 0; l < r; ++l) acc = fmaf(Wt[(size_t)order[l] * ldw + i], Gs[l * r + j], acc);
    Yn[(size_t)j * k + i] = acc;
  }
  __syncthreads();
  for (int x = tid; x < r * k; x += RS_THREADS) {
    const int j = x / k, i = x % k;
    Wt[(size_t)order[j] * ldw + i] = Yn[(size_t)j * k + i];
  }
  __syncthreads();
  // 4. U = Q P^T Y[:, top r] (m x r, row stride r), or P^T Y when Q is the
  // identity: row t of Y belongs to H's index perm[t]
  for (int64_t x = tid; x < m * r; x += RS_THREADS) {
    const int64_t i = x / r;
    const int j = (int)(x % r);
    const float* y = Wt + (size_t)order[j] * ldw;
    float s;
    if (Q) {
      s = 0.f;
      for (int t = 0; t < k; ++t) s = fmaf(Q[i * ldq + perm[t]], y[t], s);
    } else {
      s = y[iperm[i]];
    }
    U[x] = s;
    if (core) core[x] = s;
  }
  (void)status;
}

}  // namespace

int gram_df_splits(int k, int64_t n) {
  const int tiles = df_tiles(k);
  int64_t s = (2 * 152 + tiles - 1) / tiles;
  s = s < 1 ? 1 : s;
  const int64_t maxs = (n + DF_CHUNK - 1) / DF_CHUNK;
  if (s > maxs) s = maxs < 1 ? 1 : maxs;
  return (int)s;
}

size_t gram_df_partial_doubles(int k, int64_t n) {
  return (size_t)df_tiles(k) * gram_df_splits(k, n) * DF_TILE * DF_TILE;
}

template <typename T>
cudaError_t gram_df(const T* B, int k, int64_t n, int64_t ldb, double* partials, double* H, cudaStream_t st) {
  if (k < 1 || k > RR_SVD_KMAX || n < 1) return cudaErrorInvalidValue;
  const int tiles = df_tiles(k), splits = gram_df_splits(k, n);
  ProfScope prof("gram_df", st, (double)k * n * sizeof(T), 2.0 * k * k * n);
  note_launch("gram_df");
  k_gram_df<T><<<tiles * splits, 256, 0, st>>>(B, k, n, ldb, splits, partials);
  note_launch("gram_df");
  k_gram_df_reduce<<<tiles, 256, 0, st>>>(partials, k, splits, H);
  return cudaGetLastError();
}
template cudaError_t gram_df<float>(const float*, int, int64_t, int64_t, double*, double*, cudaStream_t);
template cudaError_t gram_df<__nv_bfloat16>(const __nv_bfloat16*, int, int64_t, int64_t, double*, double*,
                                            cudaStream_t);

bool rr_svd_ok(int k, int r) {
  return k >= 1 && k <= RR_SVD_KMAX && r >= 1 && r <= k && r <= 64 && rs_smem_bytes(k) <= 227 * 1024 - 1024;
}

cudaError_t launch_rr_svd(const double* H, int k, int r, const float* Q, int64_t m, int64_t ldq, float* U,
                          float* core, int* status, cudaStream_t st) {
  if (!rr_svd_ok(k, r)) return cudaErrorInvalidValue;
  const size_t smem = rs_smem_bytes(k);
  cudaError_t e = raise_smem_limit(k_rr_svd);
  if (e != cudaSuccess) return e;
  ProfScope prof("rr_svd", st, 0, 0);
  note_launch("rr_svd");
  k_rr_svd<<<1, RS_THREADS, smem, st>>>(H, k, r, Q, m, ldq, U, core, status);
  return cudaGetLastError();
}

}  // namespace ttr
