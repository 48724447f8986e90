// Cholesky factorisation of a small symmetric positive definite Gram matrix
// and the inverse of its triangular factor, by one CTA in shared memory
// (used by the block orthonormalisation of Alg. 3 step 5).
#pragma once

#include "common.cuh"

namespace ttr {

// G (b x b, row stride ldg, upper triangle used) = R^T R.  R is written to
// R (row stride ldr, upper triangle; its lower triangle is zeroed) and
// T = R^{-1} (b x b, row stride ldt, upper triangular) to T.  G is destroyed.
// A pivot below 1e-6 of diag0[j] (or non-positive) raises *flag (when
// report) and is replaced by 1 so the factorisation completes.
// One barrier per column: row j of R is formed from the unscaled row j of G
// while the trailing block (rows and columns > j) is updated in place.
__device__ inline void chol_inv_cta(float* G, int ldg, int b, const float* diag0, float* R, int ldr, float* T,
                                    int ldt, int* flag, bool report, unsigned long long* badmask = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    float dj = G[j * ldg + j];
    if (!(dj > 1e-6f * diag0[j])) {
      if (report && tid == 0 && flag) atomicExch(flag, 1);
      if (badmask && tid == 0) atomicOr(badmask, 1ull << j);
      dj = 1.f;
    }
    const float rj = sqrtf(dj), inv = 1.f / rj, inv2 = inv * inv;
    for (int l = j + tid; l < b; l += blockDim.x) R[j * ldr + l] = (l == j) ? rj : G[j * ldg + l] * inv;
    for (int l = tid; l < j; l += blockDim.x) R[j * ldr + l] = 0.f;
    for (int i = j + 1 + wid; i < b; i += nw) {
      const float gi = G[j * ldg + i] * inv2;
      for (int l = i + lane; l < b; l += 32) G[i * ldg + l] -= gi * G[j * ldg + l];
    }
    __syncthreads();
  }
  // T = R^{-1}: one thread per column, back substitution in shared memory
  for (int c = tid; c < b; c += blockDim.x) {
    for (int i = b - 1; i > c; --i) T[i * ldt + c] = 0.f;
    for (int i = c; i >= 0; --i) {
      float s0 = (i == c) ? 1.f : 0.f, s1 = 0.f;
      int l = i + 1;
      for (; l + 1 <= c; l += 2) {
        s0 -= R[i * ldr + l] * T[l * ldt + c];
        s1 -= R[i * ldr + l + 1] * T[(l + 1) * ldt + c];
      }
      if (l <= c) s0 -= R[i * ldr + l] * T[l * ldt + c];
      T[i * ldt + c] = (s0 + s1) / R[i * ldr + i];
    }
  }
  __syncthreads();
}


// Cholesky factorisation and triangular inverse of a b x b Gram, b <= 32,
// by one warp (the calling warp, all 32 lanes; one warp of a CTA at a time,
// since the routine keeps its rows of R in static shared arrays), in one
// sweep.  Lane l holds column l of the upper triangle of G in a register
// window that slides down one row per step: at step j, a[s] = G[j + s][l],
// so the pivot row is always a[0] and every register index is a
// compile-time constant while the column loop runs at run time.  Row j of
// R goes to R and, shifted so that it starts at R[j][j + 1], to a
// 16-byte-aligned shared row Rs[j], which every lane reads back as eight
// vector broadcasts.  The same row updates row l of V (started as the
// identity), held as the window v[s] = V[l][j + s]: T[l][j] = V[l][j] /
// R[j][j] is final at step j, and V[l][j + s] -= R[j][j + s] T[l][j]
// (T[:, c] = (e_c - sum_{j < c} R[j][c] T[:, j]) / R[c][c], i.e. T R = I),
// so no triangular solve follows.  T is staged transposed (conflict-free)
// and written row by row at the end.  Entries past row or column b are
// exact zeros in Rs and in the windows, so the sums run over full vectors
// without changing a bit of the result.  Pivot square roots and
// reciprocals use the hardware reciprocal square root (a few ulp), which
// the following Cholesky QR passes absorb.  A pivot below 1e-6 of diag0
// (or non-positive) raises *flag when report and is replaced by 1.
// Callers use the out-of-line copy below.
__device__ __forceinline__ void chol_inv_warp(const float* G, int ldg, int b, const float* diag0, float* R,
                                                   int ldr, float* T, int ldt, int* flag, bool report,
                                                   unsigned long long* badmask, int bit0 = 0) {
  __shared__ __align__(16) float Rs[32][36];   // Rs[j][s] = R[j][j + 1 + s], zero past column b
  __shared__ float Tt[32][33];                 // Tt[j][l] = T[l][j]
  const unsigned full = 0xffffffffu;
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 32; ++q) Rs[q][l] = 0.f;
  if (l < 4) {
#pragma unroll
    for (int q = 0; q < 32; ++q) Rs[q][32 + l] = 0.f;
  }
  float a[32];                            // a[s] = G[j + s][l] at step j (rows <= l)
  float v[32];                            // v[s] = V[l][j + s] at step j
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    a[i] = (i <= l && l < b) ? G[i * ldg + l] : 0.f;
    v[i] = (i == l && l < b) ? 1.f : 0.f;
  }
  const float d0 = (l < b) ? diag0[l] : 1.f;
  bool bad = false;
  unsigned long long badbits = 0ull;
  __syncwarp();
#pragma unroll 1
  for (int j = 0; j < b; ++j) {
    float djj = __shfl_sync(full, a[0], j);
    const float dref = __shfl_sync(full, d0, j);
    if (!(djj > 1e-6f * dref)) {
      bad = true;
      badbits |= 1ull << j;
      djj = 1.f;
    }
    const float inv = rsqrtf(djj);
    const float rjl = (l == j) ? djj * inv : ((l > j) ? a[0] * inv : 0.f);   // R[j][l]
    const float tlj = v[0] * inv;                                            // T[l][j]
    if (l < b) R[j * ldr + l] = rjl;
    if (l > j) Rs[j][l - j - 1] = rjl;
    Tt[j][l] = tlj;
    __syncwarp();
    // G[j + s][l] -= R[j][j + s] R[j][l] and V[l][j + s] -= R[j][j + s] T[l][j],
    // then slide both windows down a row
    const float4* rv = reinterpret_cast<const float4*>(Rs[j]);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 r4 = rv[q];
      const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int s = 4 * q + e + 1;
        if (s < 32) {
          a[s - 1] = fmaf(-rr[e], rjl, a[s]);
          v[s - 1] = fmaf(-rr[e], tlj, v[s]);
        }
      }
    }
    a[31] = 0.f;
    v[31] = 0.f;
  }
  if (report && bad && l == 0 && flag) atomicExch(flag, 1);
  if (badmask && badbits && l == 0) atomicOr(badmask, badbits << bit0);
  __syncwarp();
  // row r of T: lane l writes T[r][l] = Tt[l][r] (zero below the diagonal)
  for (int r = 0; r < b; ++r)
    if (l < b) T[r * ldt + l] = (l >= r) ? Tt[l][r] : 0.f;
  __syncwarp();
}

// Out-of-line copy (one per kernel, its own register allocation).
static __device__ __noinline__ void chol_inv_warp_ool(const float* G, int ldg, int b, const float* diag0, float* R,
                                                       int ldr, float* T, int ldt, int* flag, bool report,
                                                       unsigned long long* badmask, int bit0) {
  chol_inv_warp(G, ldg, b, diag0, R, ldr, T, ldt, flag, report, badmask, bit0);
}

// chol_inv_cta's contract for b <= 32: the CTA synchronises, warp 0 alone
// factors (the other warps do not enter the call), the CTA synchronises.
__device__ __forceinline__ void chol_inv_warp32_call(const float* G, int ldg, int b, const float* diag0, float* R,
                                                     int ldr, float* T, int ldt, int* flag, bool report,
                                                     unsigned long long* badmask = nullptr) {
  __syncthreads();
  if (threadIdx.x < 32) chol_inv_warp_ool(G, ldg, b, diag0, R, ldr, T, ldt, flag, report, badmask, 0);
  __syncthreads();
}

// 32 < b <= 64 in two column blocks (first 32, then b2 = b - 32), the two
// diagonal blocks by the one-warp routine and the coupling products by the
// whole CTA:  R11 = chol(G11), T11 = R11^-1;  R12 = T11^T G12;
// G22 <- G22 - R12^T R12;  R22 = chol(G22), T22 = R22^-1;
// T12 = -(T11 R12) T22.  G (upper triangle used) is destroyed.
static __device__ __noinline__ void chol_inv_blocked64(float* G, int ldg, int b, const float* diag0, float* R, int ldr, float* T,
                                          int ldt, int* flag, bool report, unsigned long long* badmask) {
  const int tid = threadIdx.x, nt = blockDim.x, b2 = b - 32;
  __syncthreads();
  if (tid < 32) chol_inv_warp_ool(G, ldg, 32, diag0, R, ldr, T, ldt, flag, report, badmask, 0);
  __syncthreads();
  // R12[i][c] = sum_{k <= i} T11[k][i] G[k][32 + c]; zero R21 and T21
  for (int x = tid; x < 32 * b2; x += nt) {
    const int i = x / b2, c = x % b2;
    float acc = 0.f;
    for (int k = 0; k <= i; ++k) acc = fmaf(T[k * ldt + i], G[k * ldg + 32 + c], acc);
    R[i * ldr + 32 + c] = acc;
    R[(32 + c) * ldr + i] = 0.f;
    T[(32 + c) * ldt + i] = 0.f;
  }
  __syncthreads();
  // Schur complement, upper triangle, in place
  for (int x = tid; x < b2 * b2; x += nt) {
    const int i = x / b2, c = x % b2;
    if (c < i) continue;
    float acc = G[(32 + i) * ldg + 32 + c];
    for (int k = 0; k < 32; ++k) acc = fmaf(-R[k * ldr + 32 + i], R[k * ldr + 32 + c], acc);
    G[(32 + i) * ldg + 32 + c] = acc;
  }
  __syncthreads();
  if (tid < 32)
    chol_inv_warp_ool(G + 32 * ldg + 32, ldg, b2, diag0 + 32, R + 32 * ldr + 32, ldr, T + 32 * ldt + 32, ldt, flag,
                      report, badmask, 32);
  __syncthreads();
  // X = T11 R12 (T11 upper: k >= i) into the place of G12, which is no
  // longer needed, then T12 = -X T22 (T22 upper: k <= c)
  for (int x = tid; x < 32 * b2; x += nt) {
    const int i = x / b2, c = x % b2;
    float acc = 0.f;
    for (int k = i; k < 32; ++k) acc = fmaf(T[i * ldt + k], R[k * ldr + 32 + c], acc);
    G[i * ldg + 32 + c] = acc;
  }
  __syncthreads();
  for (int x = tid; x < 32 * b2; x += nt) {
    const int i = x / b2, c = x % b2;
    float acc = 0.f;
    for (int k = 0; k <= c; ++k) acc = fmaf(G[i * ldg + 32 + k], T[(32 + k) * ldt + 32 + c], acc);
    T[i * ldt + 32 + c] = -acc;
  }
  __syncthreads();
}

// The fastest routine for the CTA at hand (same contract as chol_inv_cta):
// one warp for b <= 32, two warp-factored column blocks for b <= 64.
__device__ inline void chol_inv_fast(float* G, int ldg, int b, const float* diag0, float* R, int ldr, float* T,
                                     int ldt, int* flag, bool report, unsigned long long* badmask = nullptr) {
  if (b <= 32) chol_inv_warp32_call(G, ldg, b, diag0, R, ldr, T, ldt, flag, report, badmask);
  else if (b <= 64) chol_inv_blocked64(G, ldg, b, diag0, R, ldr, T, ldt, flag, report, badmask);
  else chol_inv_cta(G, ldg, b, diag0, R, ldr, T, ldt, flag, report, badmask);
}

// Pivoted variant for a block that keeps only c <= b columns (the Krylov
// dimension cap): greedy symmetric pivoting on the largest remaining
// diagonal of G (b x b, full symmetric storage, row stride ldg) selects c
// columns; R (c x c, row stride ldr) is the Cholesky factor of the selected
// columns' Gram and Tf (b x bt, row stride ldt, zeroed here) maps the b
// columns to the c kept ones: Tf[perm[i]][j] = (R^{-1})[i][j] for i, j < c.
// perm (b ints of shared memory) receives the pivot order.  A pivot below
// 1e-6 of its original diagonal (or non-positive) raises *flag when report.
__device__ inline void pchol_select_cta(float* G, int ldg, int b, int c, const float* diag0, float* R, int ldr,
                                        float* Tf, int ldt, int bt, int* perm, float* dsw, int* flag,
                                        bool report, unsigned long long* badmask = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  __shared__ int s_piv;
  for (int i = tid; i < b; i += blockDim.x) {
    perm[i] = i;
    dsw[i] = diag0[i];
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    if (wid == 0) {
      float best = -1.f;
      int bi = j;
      for (int i = j + lane; i < b; i += 32) {
        const float v = G[i * ldg + i];
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) s_piv = bi;
    }
    __syncthreads();
    const int pv = s_piv;
    if (pv != j) {
      // symmetric swap of rows and columns j <-> pv
      for (int l = tid; l < b; l += blockDim.x) {
        const float t = G[j * ldg + l]; G[j * ldg + l] = G[pv * ldg + l]; G[pv * ldg + l] = t;
      }
      __syncthreads();
      for (int l = tid; l < b; l += blockDim.x) {
        const float t = G[l * ldg + j]; G[l * ldg + j] = G[l * ldg + pv]; G[l * ldg + pv] = t;
      }
      if (tid == 0) {
        const int t = perm[j]; perm[j] = perm[pv]; perm[pv] = t;
        const float d = dsw[j]; dsw[j] = dsw[pv]; dsw[pv] = d;
      }
      __syncthreads();
    }
    float dj = G[j * ldg + j];
    if (!(dj > 1e-6f * dsw[j])) {
      if (report && tid == 0 && flag) atomicExch(flag, 1);
      if (badmask && tid == 0) atomicOr(badmask, 1ull << j);
      dj = 1.f;
    }
    const float rj = sqrtf(dj), inv = 1.f / rj, inv2 = inv * inv;
    for (int l = j + tid; l < c; l += blockDim.x) R[j * ldr + l] = (l == j) ? rj : G[j * ldg + l] * inv;
    for (int l = tid; l < j; l += blockDim.x) R[j * ldr + l] = 0.f;
    // full trailing update (later swaps need whole rows and columns)
    for (int i = j + 1 + wid; i < b; i += nw) {
      const float gi = G[j * ldg + i] * inv2;
      for (int l = j + 1 + lane; l < b; l += 32) G[i * ldg + l] -= gi * G[j * ldg + l];
    }
    __syncthreads();
  }
  for (int x = tid; x < b * ldt; x += blockDim.x) Tf[x] = 0.f;
  __syncthreads();
  // (R^{-1}) column by column; row i of it lands on row perm[i] of Tf
  for (int col = tid; col < c; col += blockDim.x) {
    float t[64];
    for (int i = col; i >= 0; --i) {
      float s0 = (i == col) ? 1.f : 0.f;
      for (int l = i + 1; l <= col; ++l) s0 -= R[i * ldr + l] * t[l];
      t[i] = s0 / R[i * ldr + i];
    }
    for (int i = 0; i <= col; ++i) Tf[perm[i] * ldt + col] = t[i];
  }
  (void)bt;
  __syncthreads();
}

}  // namespace ttr
