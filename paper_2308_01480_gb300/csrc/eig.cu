// Rayleigh-Ritz of one mode (Alg. 3 steps 6-8): the top-r eigenpairs of the
// small symmetric matrix H = Q^T C C^T Q (or of the Gram C C^T on the
// exhaustion route), then U = Q V_r.
//
// The eigensolver runs in one CTA in FP32: Householder reduction of H to a
// tridiagonal T, bisection by Sturm counts for the r largest eigenvalues
// (one warp per eigenvalue, 32-point multisection), inverse iteration on T
// with a pivoted tridiagonal LU for their eigenvectors, modified
// Gram-Schmidt across them, and the back-transformation by the stored
// reflectors.  Only the r wanted eigenvectors are ever formed.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace ttr {

constexpr int EIG_THREADS = 1024;
constexpr int EIG_KMAX = 224;   // H (k x (k+1) floats) must fit shared memory

// ------------------------------------------------------------ partial A^T B
// P[y][s][t] = sum_{i in row range y} A[i][s] B[i][t] for the 32 x 32 output
// tile blockIdx.x (s < ka, t < kb); 64 threads, each with a 4 x 4 register
// tile fed by two float4 shared-memory broadcasts per row.
template <typename TA, typename TB>
__global__ void __launch_bounds__(64) k_tn_partials(const TA* __restrict__ A, int64_t lda, int ka,
                                                    const TB* __restrict__ B, int64_t ldb, int kb, int64_t m,
                                                    int64_t rows_per_split, float* __restrict__ P) {
  __shared__ __align__(16) float As[32][32];
  __shared__ __align__(16) float Bs[32][32];
  const int tiles_t = (kb + 31) / 32;
  const int s0 = (int)(blockIdx.x / tiles_t) * 32, t0 = (int)(blockIdx.x % tiles_t) * 32;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split, r1 = imin(m, r0 + rows_per_split);
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float acc[4][4] = {};
  for (int64_t i0 = r0; i0 < r1; i0 += 32) {
    __syncthreads();
    // all sixteen loads of a thread in flight at once
#pragma unroll
    for (int x = threadIdx.x; x < 32 * 32; x += 64) {
      const int r = x >> 5, c = x & 31;
      const int64_t i = i0 + r;
      As[r][c] = (i < r1 && s0 + c < ka) ? ld_elem(A, i * lda + s0 + c) : 0.f;
      Bs[r][c] = (i < r1 && t0 + c < kb) ? ld_elem(B, i * ldb + t0 + c) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[r][4 * ty]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[r][4 * tx]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(av[u], bv[w], acc[u][w]);
    }
  }
  float* out = P + (int64_t)blockIdx.y * ka * kb;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int sidx = s0 + 4 * ty + u, tidx = t0 + 4 * tx + w;
      if (sidx < ka && tidx < kb) out[(int64_t)sidx * kb + tidx] = acc[u][w];
    }
}

// out[e] = sum_{c < nparts} P[c][e] (fixed order: four interleaved chains
// over c mod 4, then ((0 + 1) + (2 + 3)))
__global__ void k_sum_parts(const float* __restrict__ P, int nparts, int64_t E, float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int c = 0;
    for (; c + 4 <= nparts; c += 4) {
      a0 += P[(int64_t)c * E + e];
      a1 += P[(int64_t)(c + 1) * E + e];
      a2 += P[(int64_t)(c + 2) * E + e];
      a3 += P[(int64_t)(c + 3) * E + e];
    }
    for (; c < nparts; ++c) a0 += P[(int64_t)c * E + e];
    out[e] = (a0 + a1) + (a2 + a3);
  }
}

// ------------------------------------------------------------ eigensolver
struct EigSmem {
  float* H;      // [k][k+1]
  float* d;      // [k]
  float* e;      // [k]
  float* tau;    // [k]
  float* v;      // [k]
  float* p;      // [k]
  float* red;    // [64]
  float* lam;    // [r]
};

// Householder tridiagonalisation of the symmetric H (full storage, row
// stride ld).  Afterwards d/e hold T, and column j of H below the
// subdiagonal holds the reflector v_j (with implicit leading 1), tau[j] its
// scale: P_j = I - tau_j v_j v_j^T acting on indices j+1..k-1.
// Three barriers per column: warp 0 forms the reflector and v; then
// p = tau A v (groups of 8 lanes per row); then the rank-2 update
// A -= v w^T + w v^T with w = p - (tau/2)(v^T p) v (a warp per row).
__device__ void householder_tridiag(EigSmem& S, int k, int ld) {
  float* H = S.H;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x, nw = nt >> 5;
  const int grp = tid >> 3, sl = tid & 7, ngrp = nt >> 3;
  for (int j = 0; j + 2 < k; ++j) {
    const int L = k - j - 1;                   // reflector length
    float* col = H + (j + 1) * ld + j;         // x_i = col[i * ld]
    if (wid == 0) {
      float part = 0.f;
#pragma unroll 4
      for (int i = 1 + lane; i < L; i += 32) {
        const float x = col[i * ld];
        part = fmaf(x, x, part);
      }
      const float sigma = warp_sum(part);
      const float x0 = col[0];
      float t = 0.f, iv = 0.f, beta = x0;
      if (sigma > 0.f) {
        const float mu = sqrtf(x0 * x0 + sigma);
        const float v0 = (x0 <= 0.f) ? x0 - mu : -sigma / (x0 + mu);
        t = 2.f * v0 * v0 / (sigma + v0 * v0);
        beta = mu;
        iv = 1.f / v0;
      }
      if (t != 0.f)
        for (int i = lane; i < L; i += 32) S.v[i] = (i == 0) ? 1.f : col[i * ld] * iv;
      if (lane == 0) {
        S.tau[j] = t;
        S.e[j] = beta;
        S.d[j] = H[j * ld + j];
      }
    }
    __syncthreads();
    const float t = S.tau[j];
    if (t == 0.f) continue;                    // column already reduced
    for (int r0 = 0; r0 < L; r0 += ngrp) {
      const int r = r0 + grp;
      float s0 = 0.f, s1 = 0.f;
      if (r < L) {
        const float* hr = H + (j + 1 + r) * ld + (j + 1);
        int c = sl;
        for (; c + 8 < L; c += 16) {
          s0 = fmaf(hr[c], S.v[c], s0);
          s1 = fmaf(hr[c + 8], S.v[c + 8], s1);
        }
        if (c < L) s0 = fmaf(hr[c], S.v[c], s0);
      }
      s0 += s1;
      s0 += __shfl_xor_sync(0xffffffffu, s0, 4);
      s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
      s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
      if (r < L && sl == 0) S.p[r] = t * s0;
    }
    __syncthreads();
    float kp = 0.f;
    for (int i = lane; i < L; i += 32) kp = fmaf(S.v[i], S.p[i], kp);
    const float K = 0.5f * t * warp_sum(kp);
    for (int r = wid; r < L; r += nw) {
      const float vr = S.v[r], wr = S.p[r] - K * vr;
      float* hr = H + (j + 1 + r) * ld + (j + 1);
#pragma unroll 4
      for (int c = lane; c < L; c += 32) {
        const float vc = S.v[c];
        hr[c] -= vr * (S.p[c] - K * vc) + wr * vc;
      }
    }
    for (int i = 1 + tid; i < L; i += nt) col[i * ld] = S.v[i];   // keep v_j
    __syncthreads();
  }
  if (tid == 0) {
    if (k >= 2) {
      S.d[k - 2] = H[(k - 2) * ld + (k - 2)];
      S.e[k - 2] = H[(k - 1) * ld + (k - 2)];
      S.tau[k - 2] = 0.f;
    }
    S.d[k - 1] = H[(k - 1) * ld + (k - 1)];
    S.e[k - 1] = 0.f;
    S.tau[k - 1] = 0.f;
  }
  __syncthreads();
}

// Number of eigenvalues of T (d, e) smaller than x (Sturm sequence).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int k, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < k; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// LU factorisation with row exchanges of the tridiagonal T - lam I, stored
// in w[0..5k): reciprocal pivots, the two superdiagonals of the upper factor,
// the multipliers and the exchange flags.  Tiny pivots are replaced by tiny
// (the usual inverse-iteration safeguard).
__device__ void tri_factor(const float* d, const float* e, int k, float lam, float tiny, float* w) {
  float* r0 = w;
  float* u1 = w + k;
  float* u2 = w + 2 * k;
  float* l = w + 3 * k;
  float* sw = w + 4 * k;
  float alpha = d[0] - lam, beta = (k > 1) ? e[0] : 0.f;
  for (int i = 0; i + 1 < k; ++i) {
    const float sub = e[i];
    const float a1 = d[i + 1] - lam, c1 = (i + 2 < k) ? e[i + 1] : 0.f;
    if (fabsf(alpha) >= fabsf(sub)) {
      const float piv = (fabsf(alpha) < tiny) ? copysignf(tiny, alpha) : alpha;
      const float rp = 1.f / piv;
      const float li = sub * rp;
      r0[i] = rp; u1[i] = beta; u2[i] = 0.f; l[i] = li; sw[i] = 0.f;
      alpha = a1 - li * beta;
      beta = c1;
    } else {
      const float li = alpha / sub;
      const float piv = (fabsf(sub) < tiny) ? copysignf(tiny, sub) : sub;
      r0[i] = 1.f / piv; u1[i] = a1; u2[i] = c1; l[i] = li; sw[i] = 1.f;
      alpha = beta - li * a1;
      beta = -li * c1;
    }
  }
  r0[k - 1] = 1.f / ((fabsf(alpha) < tiny) ? copysignf(tiny, alpha) : alpha);
  // the last row has no superdiagonal entries: the back substitution reads
  // them (times zero), so they must be finite
  u1[k - 1] = 0.f; u2[k - 1] = 0.f; l[k - 1] = 0.f; sw[k - 1] = 0.f;
}

// x <- (T - lam I)^{-1} x with the factors of tri_factor.
__device__ void tri_solve(const float* w, int k, float* x) {
  const float* r0 = w;
  const float* u1 = w + k;
  const float* u2 = w + 2 * k;
  const float* l = w + 3 * k;
  const float* sw = w + 4 * k;
  for (int i = 0; i + 1 < k; ++i) {
    if (sw[i] != 0.f) { const float t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
    x[i + 1] -= l[i] * x[i];
  }
  float x1 = 0.f, x2 = 0.f;                 // x[i+1], x[i+2]
  for (int i = k - 1; i >= 0; --i) {
    const float v = (x[i] - u1[i] * x1 - u2[i] * x2) * r0[i];
    x[i] = v;
    x2 = x1;
    x1 = v;
  }
}

// Top-r eigenpairs of the symmetric k x k matrix held in S.H (ld = k+1).
// Writes eigenvectors as columns of Vout (k x r, row stride ldv) in global
// memory and eigenvalues (descending) to S.lam.  work: 6 * k * r floats,
// in shared memory whenever it fits (the inverse iterations are dependent
// chains, so their latency decides the kernel's time).
__device__ void sym_eig_top(EigSmem& S, int k, int r, float* Vout, int ldv, float* scratch) {
  const int ld = k + 1;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
  householder_tridiag(S, k, ld);
  float* e2 = S.p;                        // reuse: squared off-diagonals
  for (int i = tid; i < k; i += blockDim.x) e2[i] = S.e[i] * S.e[i];
  __syncthreads();
  // Gershgorin interval and scale
  float glo = FLT_MAX, ghi = -FLT_MAX, amax = 0.f;
  for (int i = tid; i < k; i += blockDim.x) {
    const float off = (i > 0 ? fabsf(S.e[i - 1]) : 0.f) + (i + 1 < k ? fabsf(S.e[i]) : 0.f);
    glo = fminf(glo, S.d[i] - off);
    ghi = fmaxf(ghi, S.d[i] + off);
    amax = fmaxf(amax, fmaxf(fabsf(S.d[i]), fabsf(S.e[i])));
  }
  for (int o = 16; o > 0; o >>= 1) {
    glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  __syncthreads();
  if (lane == 0) { S.red[wid] = glo; S.red[32 + wid] = ghi; }
  __syncthreads();
  if (tid == 0) {
    float a = FLT_MAX, bb = -FLT_MAX;
    for (int w = 0; w < nw; ++w) { a = fminf(a, S.red[w]); bb = fmaxf(bb, S.red[32 + w]); }
    S.red[0] = a; S.red[1] = bb;
  }
  __syncthreads();
  glo = S.red[0];
  ghi = S.red[1];
  __syncthreads();
  if (lane == 0) S.red[wid] = amax;
  __syncthreads();
  if (tid == 0) { float a = 0.f; for (int w = 0; w < nw; ++w) a = fmaxf(a, S.red[w]); S.red[2] = a; }
  __syncthreads();
  const float tnorm = fmaxf(S.red[2], FLT_MIN);
  const float pivmin = FLT_MIN * fmaxf(1.f, tnorm * tnorm);
  const float pad = 2.f * FLT_EPSILON * tnorm + pivmin;
  // bisection: a warp per eigenvalue evaluates Sturm counts at 32 interior
  // points of the current interval (33-fold shrink per round)
  for (int j = wid; j < r; j += nw) {
    const int t = k - 1 - j;                   // ascending index
    float lo = glo - pad, hi = ghi + pad;
    for (int it = 0; it < 7; ++it) {
      const float x = lo + (hi - lo) * (float)(lane + 1) * (1.f / 33.f);
      const int cnt = sturm_count(S.d, e2, k, x, pivmin);
      const unsigned ge = __ballot_sync(0xffffffffu, cnt >= t + 1);
      const int sidx = ge ? (__ffs(ge) - 1) : 32;
      const float xs = __shfl_sync(0xffffffffu, x, sidx < 32 ? sidx : 31);
      const float xprev = __shfl_sync(0xffffffffu, x, sidx > 0 ? sidx - 1 : 0);
      if (sidx == 32) lo = xs;
      else { hi = xs; if (sidx > 0) lo = xprev; }
    }
    if (lane == 0) S.lam[j] = 0.5f * (lo + hi);
  }
  __syncthreads();
  // inverse iteration: one thread per wanted eigenvector, vectors in scratch
  float* X = scratch;                  // [r][k]
  float* Wk = scratch + (size_t)r * k; // [r][5k]
  const float tiny = FLT_EPSILON * tnorm + pivmin;
  for (int j = tid; j < r; j += blockDim.x) {
    float* x = X + (size_t)j * k;
    float* w = Wk + (size_t)j * 5 * k;
    tri_factor(S.d, S.e, k, S.lam[j], tiny, w);
    for (int i = 0; i < k; ++i) x[i] = 1.f + 0.01f * (float)((i * 7 + j * 13) % 11);
    for (int it = 0; it < 2; ++it) {
      tri_solve(w, k, x);
      float mx = 0.f;
      for (int i = 0; i < k; ++i) mx = fmaxf(mx, fabsf(x[i]));
      const float sc = mx > 0.f ? 1.f / mx : 0.f;
      for (int i = 0; i < k; ++i) x[i] *= sc;
    }
  }
  __syncthreads();
  // Gram-Schmidt (classical, twice) across the r vectors in descending
  // eigenvalue order; restores orthogonality inside clusters
  float* dots = S.v;                   // [r] (r <= k)
  for (int j = 0; j < r; ++j) {
    float* xj = X + (size_t)j * k;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      for (int i2 = wid; i2 < j; i2 += nw) {
        const float* xi = X + (size_t)i2 * k;
        float pp = 0.f;
        for (int i = lane; i < k; i += 32) pp = fmaf(xi[i], xj[i], pp);
        pp = warp_sum(pp);
        if (lane == 0) dots[i2] = pp;
      }
      __syncthreads();
      for (int i = tid; i < k; i += nt) {
        float s0 = xj[i], s1 = 0.f;
        int i2 = 0;
        for (; i2 + 1 < j; i2 += 2) {
          s0 -= dots[i2] * X[(size_t)i2 * k + i];
          s1 -= dots[i2 + 1] * X[(size_t)(i2 + 1) * k + i];
        }
        if (i2 < j) s0 -= dots[i2] * X[(size_t)i2 * k + i];
        xj[i] = s0 + s1;
      }
      __syncthreads();
    }
    float pp = 0.f;
    for (int i = tid; i < k; i += nt) pp = fmaf(xj[i], xj[i], pp);
    const float nrm = sqrtf(block_sum(pp, S.red));
    const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
    for (int i = tid; i < k; i += nt) xj[i] *= inv;
    __syncthreads();
  }
  // back-transformation x <- P_0 P_1 ... P_{k-3} x; a warp per vector,
  // reflectors applied from the last to the first
  for (int j = wid; j < r; j += nw) {
    float* x = X + (size_t)j * k;
    for (int h = k - 3; h >= 0; --h) {
      const float t = S.tau[h];
      if (t == 0.f) continue;
      const int L = k - h - 1;
      float s0 = 0.f, s1 = 0.f;
      int i = lane;
      for (; i + 32 < L; i += 64) {
        s0 = fmaf((i == 0) ? 1.f : S.H[(h + 1 + i) * ld + h], x[h + 1 + i], s0);
        s1 = fmaf(S.H[(h + 1 + i + 32) * ld + h], x[h + 1 + i + 32], s1);
      }
      if (i < L) s0 = fmaf((i == 0) ? 1.f : S.H[(h + 1 + i) * ld + h], x[h + 1 + i], s0);
      const float sc = warp_sum(s0 + s1) * t;
      for (int i2 = lane; i2 < L; i2 += 32) {
        const float vi = (i2 == 0) ? 1.f : S.H[(h + 1 + i2) * ld + h];
        x[h + 1 + i2] -= sc * vi;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int x = tid; x < k * r; x += blockDim.x) {
    const int i = x / r, j = x % r;
    Vout[(size_t)i * ldv + j] = X[(size_t)j * k + i];
  }
  __syncthreads();
}

// H (k x k, global, row stride ldh) -> top-r eigenvectors V (k x r, ld r).
__global__ void __launch_bounds__(EIG_THREADS) k_eig_top(const float* __restrict__ Hin, int64_t ldh, int k, int r,
                                                        float* __restrict__ V, float* __restrict__ scratch,
                                                        float* __restrict__ evals, int work_in_smem) {
  extern __shared__ float sm[];
  EigSmem S;
  S.H = sm;
  S.d = S.H + (size_t)k * (k + 1);
  S.e = S.d + k;
  S.tau = S.e + k;
  S.v = S.tau + k;
  S.p = S.v + k;
  S.red = S.p + k;
  S.lam = S.red + 64;
  for (int x = threadIdx.x; x < k * k; x += blockDim.x) {
    const int i = x / k, j = x % k;
    S.H[i * (k + 1) + j] = 0.5f * (Hin[(int64_t)i * ldh + j] + Hin[(int64_t)j * ldh + i]);
  }
  __syncthreads();
  float* work = work_in_smem ? (S.lam + ((r + 3) & ~3)) : scratch;
  sym_eig_top(S, k, r, V, r, work);
  if (evals)
    for (int j = threadIdx.x; j < r; j += blockDim.x) evals[j] = S.lam[j];
}

// U (m x r) = Q (m x k, ld ldq) V (k x r); also written to core (same layout).
// V and the CTA's rows of Q are staged in shared memory with sixteen loads
// of each thread in flight at a time; each U entry is then one FMA chain over
// t = 0..k-1.
template <typename TQ>
__global__ void __launch_bounds__(256) k_apply_basis(const TQ* __restrict__ Q, int64_t ldq, int64_t m, int k,
                                                     const float* __restrict__ V, int r, float* __restrict__ U,
                                                     float* __restrict__ core, int64_t rows_per_cta) {
  constexpr int NT = 256, NL = 16;
  extern __shared__ float sm[];
  float* Vs = sm;                     // [k][r]
  float* Qs = sm + (size_t)k * r;     // [rows][k]
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = imin(m, r0 + rows_per_cta);
  const int nv = k * r, nq = (int)(r1 - r0) * k;
  for (int base = threadIdx.x; base < nv; base += NT * NL) {
    float v[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) v[u] = (base + NT * u < nv) ? V[base + NT * u] : 0.f;
#pragma unroll
    for (int u = 0; u < NL; ++u)
      if (base + NT * u < nv) Vs[base + NT * u] = v[u];
  }
  for (int base = threadIdx.x; base < nq; base += NT * NL) {
    float v[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int x = base + NT * u;
      v[u] = (x < nq) ? ld_elem(Q + (r0 + x / k) * ldq, x % k) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NL; ++u)
      if (base + NT * u < nq) Qs[base + NT * u] = v[u];
  }
  __syncthreads();
  for (int64_t x = threadIdx.x; x < (r1 - r0) * r; x += NT) {
    const int64_t i = r0 + x / r;
    const int j = (int)(x % r);
    const float* qi = Qs + (x / r) * k;
    float s = 0.f;
    for (int t = 0; t < k; ++t) s = fmaf(qi[t], Vs[t * r + j], s);
    U[i * r + j] = s;
    if (core) core[i * r + j] = s;
  }
}

// ------------------------------------------------------------ launchers
size_t eig_scratch_floats(int k, int r) { return (size_t)k * k + (size_t)7 * k * r + 64; }

bool eig_top_ok(int k) { return k >= 1 && k <= EIG_KMAX; }

static size_t eig_smem(int k, int r) { return sizeof(float) * ((size_t)k * (k + 1) + 5 * (size_t)k + 64 + r + 8); }
static size_t eig_work_bytes(int k, int r) { return sizeof(float) * 6 * (size_t)k * r; }

cudaError_t launch_eig_top(const float* H, int64_t ldh, int k, int r, float* V, float* scratch, float* evals,
                           cudaStream_t st) {
  if (!eig_top_ok(k) || r > k || r < 1) return cudaErrorInvalidValue;
  if (eig_reg_ok(k, r)) return launch_eig_reg(H, ldh, k, r, V, r, evals, scratch, st);
  size_t smem = eig_smem(k, r);
  const int work_in_smem = (smem + eig_work_bytes(k, r) + 16 <= 226 * 1024) ? 1 : 0;
  if (work_in_smem) smem += eig_work_bytes(k, r) + 16;
  raise_smem_limit(k_eig_top);
  ProfScope prof("eig_top", st, 0, 0);
  note_launch("eig_top");
  k_eig_top<<<1, EIG_THREADS, smem, st>>>(H, ldh, k, r, V, scratch, evals, work_in_smem);
  return cudaGetLastError();
}

// Row ranges of the partial products: about 32 rows each (one shared-memory
// tile per CTA up to m = 2048), at most 64.
static int rows_split(int64_t m, int64_t* rows_per_split) {
  const int64_t splits = imax(1, imin(ceil_div(m, 32), 64));
  *rows_per_split = ceil_div(m, splits);
  return (int)ceil_div(m, *rows_per_split);
}

size_t tn_parts_floats(int64_t m, int ka, int kb) {
  int64_t rpc;
  return (size_t)rows_split(m, &rpc) * ka * kb;
}

template <typename TA, typename TB>
static cudaError_t launch_tn(const TA* A, int64_t lda, int ka, const TB* B, int64_t ldb, int kb, int64_t m,
                             float* parts, float* out, cudaStream_t st) {
  int64_t rps;
  const int splits = rows_split(m, &rps);
  const dim3 grid((unsigned)(ceil_div(ka, 32) * ceil_div(kb, 32)), (unsigned)splits);
  {
    ProfScope prof("tn_small", st, 0, 2.0 * m * ka * kb);
    note_launch("tn_small");
    k_tn_partials<TA, TB><<<grid, 64, 0, st>>>(A, lda, ka, B, ldb, kb, m, rps, parts);
  }
  const int64_t E = (int64_t)ka * kb;
  note_launch("sum_parts");
  k_sum_parts<<<(int)imin(ceil_div(E, 256), 256), 256, 0, st>>>(parts, splits, E, out);
  return cudaGetLastError();
}

template <typename TQ>
static cudaError_t apply_basis_t(const TQ* Q, int64_t ldq, int64_t m, int k, const float* V, int r, float* U,
                                 float* core, cudaStream_t st) {
  int64_t rpc = 8;
  const int ctas = (int)ceil_div(m, rpc);
  const size_t smem = sizeof(float) * ((size_t)k * r + (size_t)rpc * k);
  raise_smem_limit(k_apply_basis<TQ>);
  ProfScope prof("apply_basis", st, 0, 2.0 * m * k * r);
  note_launch("apply_basis");
  k_apply_basis<TQ><<<ctas, 256, smem, st>>>(Q, ldq, m, k, V, r, U, core, rpc);
  return cudaGetLastError();
}

cudaError_t launch_apply_basis(const float* Q, int64_t ldq, int64_t m, int k, const float* V, int r, float* U,
                               float* core, cudaStream_t st) {
  return apply_basis_t(Q, ldq, m, k, V, r, U, core, st);
}

// Rayleigh-Ritz: H = Q^T W (or H = G when Q is the identity), top-r
// eigenvectors, U = Q V.  scratch holds rr_fast_scratch_floats(m, k, r).
size_t rr_fast_scratch_floats(int64_t m, int k, int r) {
  return tn_parts_floats(m, k, k) + (size_t)k * k + (size_t)k * r + eig_scratch_floats(k, r);
}

cudaError_t launch_rr_fast(const float* Q, const float* W, int64_t ld, int64_t m, int k, int r, int identity_q,
                           float* scratch, float* U, float* core, cudaStream_t st) {
  float* parts = scratch;
  float* H = parts + tn_parts_floats(m, k, k);
  float* V = H + (size_t)k * k;
  float* es = V + (size_t)k * r;
  cudaError_t e;
  const float* Hsrc;
  int64_t ldh;
  if (identity_q) {
    Hsrc = W;
    ldh = ld;
  } else {
    e = launch_tn(Q, ld, k, W, ld, k, m, parts, H, st);
    if (e != cudaSuccess) return e;
    Hsrc = H;
    ldh = k;
  }
  e = launch_eig_top(Hsrc, ldh, k, r, V, es, nullptr, st);
  if (e != cudaSuccess) return e;
  if (identity_q) {
    // Q = I (m == k): U = V
    e = cudaMemcpyAsync(U, V, sizeof(float) * (size_t)m * r, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && core)
      e = cudaMemcpyAsync(core, V, sizeof(float) * (size_t)m * r, cudaMemcpyDeviceToDevice, st);
    return e;
  }
  return launch_apply_basis(Q, ld, m, k, V, r, U, core, st);
}

// Exhaustion with D = n < m (the Krylov basis would span range(C)): the
// top-r right singular vectors V' of C from its n x n Gram C^T C, and
// Y = C V' (m x r), whose orthonormalisation (left to the caller) gives
// the top-r left singular vectors.
size_t colgram_scratch_floats(int64_t m, int n, int r) {
  return tn_parts_floats(m, n, n) + (size_t)n * n + (size_t)n * r + eig_scratch_floats(n, r);
}

template <typename T>
cudaError_t launch_colgram(const T* C, int64_t m, int n, int r, float* scratch, float* Y, cudaStream_t st) {
  float* parts = scratch;
  float* G = parts + tn_parts_floats(m, n, n);
  float* V = G + (size_t)n * n;
  float* es = V + (size_t)n * r;
  cudaError_t e = launch_tn(C, n, n, C, n, n, m, parts, G, st);
  if (e != cudaSuccess) return e;
  e = launch_eig_top(G, n, n, r, V, es, nullptr, st);
  if (e != cudaSuccess) return e;
  return apply_basis_t(C, n, m, n, V, r, Y, nullptr, st);
}

template cudaError_t launch_colgram<float>(const float*, int64_t, int, int, float*, float*, cudaStream_t);
template cudaError_t launch_colgram<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int, int, float*, float*,
                                                   cudaStream_t);

}  // namespace ttr
