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
                                    int ldt, int* flag, bool report) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    float dj = G[j * ldg + j];
    if (!(dj > 1e-6f * diag0[j])) {
      if (report && tid == 0) atomicExch(flag, 1);
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

}  // namespace ttr
