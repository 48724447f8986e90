// Small dense algebra of one mode: basis orthonormalisation (Alg. 3 step 5),
// Rayleigh-Ritz on the Krylov basis (Alg. 3 steps 6-8) and core emission.
//
// All of it runs on the GPU in FP32.  The matrices are tall-skinny
// (m x b, b <= 64) or small square (k x k, k = basis size).  Each kernel is
// one CTA: the work is latency-bound, and keeping it on one SM avoids
// cross-CTA synchronisation.
#include "common.cuh"
#include "kernels.h"

namespace ttr {

constexpr int SMALL_THREADS = 1024;

// ------------------------------------------------------------ helpers

// coef[t] = sum_i B[i*ldb + t] v[i] for t < nb; one warp per basis column.
__device__ void dots_cols(const float* B, int64_t ldb, int nb, const float* v, int64_t m,
                          float* coef) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = wid; t < nb; t += nw) {
    float s = 0.f;
    for (int64_t i = lane; i < m; i += 32) s = fmaf(B[i * ldb + t], v[i], s);
    s = warp_sum(s);
    if (lane == 0) coef[t] = s;
  }
}

// v[i] -= sum_t B[i*ldb + t] coef[t]
__device__ void sub_cols(const float* B, int64_t ldb, int nb, const float* coef, float* v, int64_t m) {
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    float s = 0.f;
    const float* row = B + i * ldb;
    for (int t = 0; t < nb; ++t) s = fmaf(row[t], coef[t], s);
    v[i] -= s;
  }
}

// Two-sided cyclic Jacobi on a symmetric k x k matrix H (row stride ldh),
// with V (row stride ldv) accumulating the rotations.  Disjoint pairs of a
// round-robin tournament are rotated simultaneously.  On return diag(H)
// holds the eigenvalues and V the eigenvectors (columns).
__device__ void jacobi_eig(float* H, int ldh, float* V, int ldv, int k, float* cs, float* red) {
  const int K = (k + 1) & ~1;            // pad to even; index k (if odd) is a dummy
  const int half = K / 2;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) V[(e / k) * ldv + e % k] = (e / k == e % k) ? 1.f : 0.f;
  __syncthreads();
  if (k <= 1) return;
  for (int sweep = 0; sweep < 16; ++sweep) {
    // convergence: off-diagonal energy vs diagonal energy
    float off = 0.f, dia = 0.f;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      int i = e / k, j = e % k;
      float h = H[i * ldh + j];
      if (i == j) dia += h * h; else off += h * h;
    }
    off = block_sum(off, red);
    __syncthreads();
    dia = block_sum(dia, red);
    // FP32 cannot push the off-diagonal energy much below k u^2 of the
    // diagonal; stop there
    if (off <= 1e-11f * dia || dia == 0.f) break;
    for (int r = 0; r < K - 1; ++r) {
      for (int j = threadIdx.x; j < half; j += blockDim.x) {
        int p = (j == 0) ? 0 : 1 + (r + j) % (K - 1);
        int q = (j == 0) ? 1 + r % (K - 1) : 1 + (r - j + (K - 1)) % (K - 1);
        if (p > q) { int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < k) {
          float a = H[p * ldh + p], d = H[q * ldh + q], e2 = H[p * ldh + q];
          if (fabsf(e2) > 1e-30f && fabsf(e2) > 1e-9f * sqrtf(fabsf(a * d))) {
            float th = (d - a) / (2.f * e2);
            float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = rsqrtf(t * t + 1.f);
            s = t * c;
          }
        }
        cs[4 * j] = c; cs[4 * j + 1] = s;
        reinterpret_cast<int*>(cs)[4 * j + 2] = p;
        reinterpret_cast<int*>(cs)[4 * j + 3] = q;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * k; e += blockDim.x) {      // rows p, q
        int j = e / k, col = e % k;
        int q = reinterpret_cast<int*>(cs)[4 * j + 3];
        if (q >= k) continue;
        int p = reinterpret_cast<int*>(cs)[4 * j + 2];
        float c = cs[4 * j], s = cs[4 * j + 1];
        if (s == 0.f) continue;
        float hp = H[p * ldh + col], hq = H[q * ldh + col];
        H[p * ldh + col] = c * hp - s * hq;
        H[q * ldh + col] = s * hp + c * hq;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * k; e += blockDim.x) {      // cols p, q of H and V
        int j = e / k, row = e % k;
        int q = reinterpret_cast<int*>(cs)[4 * j + 3];
        if (q >= k) continue;
        int p = reinterpret_cast<int*>(cs)[4 * j + 2];
        float c = cs[4 * j], s = cs[4 * j + 1];
        if (s == 0.f) continue;
        float hp = H[row * ldh + p], hq = H[row * ldh + q];
        H[row * ldh + p] = c * hp - s * hq;
        H[row * ldh + q] = s * hp + c * hq;
        float vp = V[row * ldv + p], vq = V[row * ldv + q];
        V[row * ldv + p] = c * vp - s * vq;
        V[row * ldv + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// order[j] = index of the j-th largest diagonal entry of H (ties: lower index).
__device__ void sort_desc(const float* H, int ldh, int k, int* order) {
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    float lt = H[t * ldh + t];
    int rank = 0;
    for (int s = 0; s < k; ++s) {
      float ls = H[s * ldh + s];
      rank += (ls > lt) || (ls == lt && s < t);
    }
    order[rank] = t;
  }
  __syncthreads();
}

// ------------------------------------------------------------ orth_block
// Appends c orthonormal columns to the basis Q (m x kq, row stride ldq),
// spanning the top-c directions of Z after projecting out span(Q):
//   Z <- Z - Q (Q^T Z) twice (block Gram-Schmidt);
//   if c < zc: keep the top-c left singular directions (eigenvectors of
//   Z^T Z), the Krylov dimension cap;
//   then column by column: project against [Q, new columns] until the norm
//   stops dropping by more than half (Daniel-Gragg-Kaufman-Stewart), and
//   normalise.  A column left with less than 1e-5 of its raw norm carries
//   no information above FP32 rounding; it is replaced by a deterministic
//   pseudo-random vector orthogonalised the same way, which keeps Q
//   orthonormal (such directions get no weight in Rayleigh-Ritz).
// Scratch (global): Zw m x zc, Zt m x zc, P kq x zc, G/Vg zc x zc.
__global__ void __launch_bounds__(SMALL_THREADS)
k_orth_block(const float* __restrict__ Z, int64_t ldz, int64_t m, int zc, float* Q, int64_t ldq, int kq,
             int c, float* scratch, uint64_t seed, int* status, const int* only_if) {
  if (only_if && *only_if == 0) return;   // the fast path succeeded
  extern __shared__ float sm[];
  float* coef = sm;                 // [kq + c]
  float* red = coef + kq + c + 32;  // [64]
  float* cs = red + 64;             // [4 * 32]
  int* order = reinterpret_cast<int*>(cs + 4 * 32);   // [64]
  float* v = reinterpret_cast<float*>(order + 64);     // [m]
  float* G = v + m + zc + 8;                           // [zc][zc + 1]
  float* Vg = G + zc * (zc + 1);                       // [zc][zc + 1]
  const int ldg = zc + 1;
  float* Zw = scratch;
  float* Zt = Zw + m * zc;
  float* P = Zt + m * zc;
  const int tid = threadIdx.x;

  // working copy and raw column norms (the reference scale for breakdown)
  float* rawn = v + m;  // [zc]
  for (int64_t e = tid; e < m * zc; e += blockDim.x) Zw[e] = Z[(e / zc) * ldz + e % zc];
  __syncthreads();
  for (int j = 0; j < zc; ++j) {
    float s = 0.f;
    for (int64_t i = tid; i < m; i += blockDim.x) s = fmaf(Zw[i * zc + j], Zw[i * zc + j], s);
    s = block_sum(s, red);
    if (tid == 0) rawn[j] = sqrtf(s);
    __syncthreads();
  }

  // block Gram-Schmidt twice
  if (kq > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int e = tid; e < kq * zc; e += blockDim.x) {
        int t = e / zc, j = e % zc;
        float s = 0.f;
        for (int64_t i = 0; i < m; ++i) s = fmaf(Q[i * ldq + t], Zw[i * zc + j], s);
        P[e] = s;
      }
      __syncthreads();
      for (int64_t e = tid; e < m * zc; e += blockDim.x) {
        int64_t i = e / zc;
        int j = (int)(e % zc);
        float s = 0.f;
        for (int t = 0; t < kq; ++t) s = fmaf(Q[i * ldq + t], P[t * zc + j], s);
        Zw[e] -= s;
      }
      __syncthreads();
    }
  }

  // dimension cap: top-c directions of the projected block
  const float* src = Zw;
  if (c < zc) {
    for (int e = tid; e < zc * zc; e += blockDim.x) {
      int s1 = e / zc, s2 = e % zc;
      float s = 0.f;
      for (int64_t i = 0; i < m; ++i) s = fmaf(Zw[i * zc + s1], Zw[i * zc + s2], s);
      G[s1 * ldg + s2] = s;
    }
    __syncthreads();
    jacobi_eig(G, ldg, Vg, ldg, zc, cs, red);
    sort_desc(G, ldg, zc, order);
    for (int64_t e = tid; e < m * c; e += blockDim.x) {
      int64_t i = e / c;
      int j = (int)(e % c);
      int col = order[j];
      float s = 0.f;
      for (int t = 0; t < zc; ++t) s = fmaf(Zw[i * zc + t], Vg[t * ldg + col], s);
      Zt[i * zc + j] = s;
    }
    // raw scale of a truncated column: the largest raw norm of the block
    __syncthreads();
    if (tid == 0) {
      float mx = 0.f;
      for (int j = 0; j < zc; ++j) mx = fmaxf(mx, rawn[j]);
      for (int j = 0; j < c; ++j) rawn[j] = mx;
    }
    __syncthreads();
    src = Zt;
  }

  // column-wise orthonormalisation against [Q, earlier new columns]
  for (int j = 0; j < c; ++j) {
    for (int64_t i = tid; i < m; i += blockDim.x) v[i] = src[i * zc + j];
    __syncthreads();
    float nrm;
    {
      float s = 0.f;
      for (int64_t i = tid; i < m; i += blockDim.x) s = fmaf(v[i], v[i], s);
      nrm = sqrtf(block_sum(s, red));
    }
    float scale = rawn[j];
    for (int attempt = 0; attempt < 3; ++attempt) {
      const int nb = kq + j;
      for (int it = 0; it < 4 && nb > 0; ++it) {
        __syncthreads();
        dots_cols(Q, ldq, nb, v, m, coef);
        __syncthreads();
        sub_cols(Q, ldq, nb, coef, v, m);
        __syncthreads();
        float s = 0.f;
        for (int64_t i = tid; i < m; i += blockDim.x) s = fmaf(v[i], v[i], s);
        float nn = sqrtf(block_sum(s, red));
        bool done = (it >= 1) && (nn > 0.5f * nrm);
        nrm = nn;
        if (done) break;
      }
      if (nrm > 1e-5f * scale && nrm > 0.f) break;
      // breakdown: replace by a pseudo-random vector and orthogonalise again
      __syncthreads();
      for (int64_t i = tid; i < m; i += blockDim.x)
        v[i] = hash_uniform(seed ^ ((uint64_t)(kq + j) << 40) ^ ((uint64_t)attempt << 56), (uint64_t)i);
      __syncthreads();
      float s = 0.f;
      for (int64_t i = tid; i < m; i += blockDim.x) s = fmaf(v[i], v[i], s);
      nrm = sqrtf(block_sum(s, red));
      scale = nrm;
      if (attempt == 2) set_status(tid == 0 ? status : nullptr, DEV_BREAKDOWN);
    }
    __syncthreads();
    const float inv = (nrm > 0.f) ? 1.f / nrm : 0.f;
    for (int64_t i = tid; i < m; i += blockDim.x) Q[i * ldq + kq + j] = v[i] * inv;
    __syncthreads();
  }
}

// ------------------------------------------------------------ rayleigh-ritz
// H = Q^T W (k x k, symmetrised), eigen-decomposed; U = Q V[:, top r]
// written to U (m x r, row stride r) and to the core (same layout, FP32).
// With identity_q, H = W (the Gram C C^T of the exhaustion route) and U = V.
__global__ void __launch_bounds__(SMALL_THREADS)
k_rayleigh_ritz(const float* __restrict__ Q, const float* __restrict__ W, int64_t ld, int64_t m, int k,
                int r, int identity_q, float* Hg, float* Vg, int use_global, float* U, float* core) {
  extern __shared__ float sm[];
  float* red = sm;               // [64]
  float* cs = red + 64;          // [4 * 128]
  int* order = reinterpret_cast<int*>(cs + 4 * 128);   // [k]
  float* H;
  float* V;
  const int ldh = k + 1;
  if (use_global) {
    H = Hg; V = Vg;
  } else {
    H = reinterpret_cast<float*>(order + ((k + 3) & ~3));
    V = H + k * ldh;
  }
  const int tid = threadIdx.x;
  for (int e = tid; e < k * k; e += blockDim.x) {
    int s1 = e / k, s2 = e % k;
    if (s2 < s1) continue;
    float h;
    if (identity_q) {
      h = 0.5f * (W[(int64_t)s1 * ld + s2] + W[(int64_t)s2 * ld + s1]);
    } else {
      float a = 0.f, bsum = 0.f;
      for (int64_t i = 0; i < m; ++i) {
        a = fmaf(Q[i * ld + s1], W[i * ld + s2], a);
        bsum = fmaf(Q[i * ld + s2], W[i * ld + s1], bsum);
      }
      h = 0.5f * (a + bsum);
    }
    H[s1 * ldh + s2] = h;
    H[s2 * ldh + s1] = h;
  }
  __syncthreads();
  jacobi_eig(H, ldh, V, ldh, k, cs, red);
  sort_desc(H, ldh, k, order);
  for (int64_t e = tid; e < m * r; e += blockDim.x) {
    int64_t i = e / r;
    int j = (int)(e % r);
    int col = order[j];
    float s;
    if (identity_q) {
      s = V[i * ldh + col];
    } else {
      s = 0.f;
      for (int t = 0; t < k; ++t) s = fmaf(Q[i * ld + t], V[t * ldh + col], s);
    }
    U[e] = s;
    if (core) core[e] = s;
  }
}

// ------------------------------------------------------------ last core and checks
// Alg. 3 step 12 and the final check in one launch.  Row y = 0 of the grid
// writes the last core (the last remainder converted to FP32) and checks the
// values it writes; row y = k + 1 checks core k.  A non-finite core entry is
// only possible from non-finite input, since every intermediate is a bounded
// combination of input values.
struct FinaliseArgs {
  float* last_core;
  int64_t last_count;
  int* status;
  const float* core[kFinaliseMaxCores];
  int64_t count[kFinaliseMaxCores];
};

template <typename T>
__global__ void k_finalise(const T* __restrict__ R, const FinaliseArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  if (blockIdx.y == 0) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.last_count; e += stride) {
      const float v = ld_elem(R, e);
      a.last_core[e] = v;
      bad |= !isfinite(v);
    }
  } else {
    const float* __restrict__ p = a.core[blockIdx.y - 1];
    const int64_t cnt = a.count[blockIdx.y - 1];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += stride) bad |= !isfinite(p[e]);
  }
  if (bad) set_status(a.status, DEV_NONFINITE);
}

// ------------------------------------------------------------ launchers
size_t orth_scratch_floats(int64_t m, int zc, int kq) {
  return (size_t)(2 * m * zc + (int64_t)kq * zc);
}

cudaError_t launch_orth_block(const float* Z, int64_t ldz, int64_t m, int zc, float* Q, int64_t ldq, int kq,
                              int c, float* scratch, uint64_t seed, int* status, const int* only_if,
                              cudaStream_t st) {
  if (zc > 64 || c > zc) return cudaErrorInvalidValue;
  size_t smem = sizeof(float) * ((size_t)kq + c + 32 + 64 + 4 * 32 + 64 + m + zc + 8 + 2 * (size_t)zc * (zc + 1));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  raise_smem_limit(k_orth_block);
  ProfScope prof("orth_block", st, 0, 0);
  note_launch("orth_block");
  k_orth_block<<<1, SMALL_THREADS, smem, st>>>(Z, ldz, m, zc, Q, ldq, kq, c, scratch, seed, status, only_if);
  return cudaGetLastError();
}

size_t rr_scratch_floats(int k) { return (size_t)2 * k * (k + 1); }

cudaError_t launch_rayleigh_ritz(const float* Q, const float* W, int64_t ld, int64_t m, int k, int r,
                                 int identity_q, float* scratch, float* U, float* core, cudaStream_t st) {
  size_t base = sizeof(float) * (64 + 4 * 128) + sizeof(int) * ((k + 3) & ~3);
  size_t mats = sizeof(float) * 2 * (size_t)k * (k + 1);
  int use_global = (base + mats > 220 * 1024) ? 1 : 0;
  if (k > 256) return cudaErrorInvalidValue;   // cs scratch holds 128 pairs
  size_t smem = base + (use_global ? 0 : mats);
  raise_smem_limit(k_rayleigh_ritz);
  ProfScope prof("rayleigh_ritz", st, 0, 0);
  note_launch("rayleigh_ritz");
  k_rayleigh_ritz<<<1, SMALL_THREADS, smem, st>>>(Q, W, ld, m, k, r, identity_q, scratch,
                                                  scratch + (size_t)k * (k + 1), use_global, U, core);
  return cudaGetLastError();
}

cudaError_t launch_finalise(const void* R, int dtype, int64_t last_count, float* last_core,
                            const float* const* cores, const int64_t* counts, int ncores, int* status,
                            cudaStream_t st) {
  if (ncores < 0 || ncores > kFinaliseMaxCores || last_count < 0) return cudaErrorInvalidValue;
  FinaliseArgs a;
  a.last_core = last_core;
  a.last_count = last_count;
  a.status = status;
  int64_t most = last_count;
  for (int k = 0; k < kFinaliseMaxCores; ++k) {
    a.core[k] = k < ncores ? cores[k] : nullptr;
    a.count[k] = k < ncores ? counts[k] : 0;
    most = imax(most, a.count[k]);
  }
  const dim3 grid((unsigned)imax(1, imin(ceil_div(most, 256), 1024)), (unsigned)(ncores + 1));
  note_launch("finalise");
  if (dtype == TT_BF16)
    k_finalise<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)R, a);
  else
    k_finalise<float><<<grid, 256, 0, st>>>((const float*)R, a);
  return cudaGetLastError();
}

}  // namespace ttr
