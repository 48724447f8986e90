// Top-r eigenpairs of the small symmetric Rayleigh-Ritz matrix (Alg. 3
// steps 6-8), k <= 160, in two one-CTA kernels.  The first holds H in
// registers: 8 warps, thread (warp w, lane l) owning the entries
// (l + 32 a, w + 8 c), a < KT = ceil(k / 32), c < 4 KT.  The second (16
// warps, so that the register-resident Cholesky of step 4 fits) does steps
// 2-5.
//
//  1. Householder tridiagonalisation.  Per column two barriers: the warp
//     owning column j forms the reflector v from its registers; each warp
//     forms p = tau H v for its own columns by a lane reduction; then every
//     thread applies H -= v w^T + w v^T to its entries, w = p - (tau/2)
//     (v^T p) v.  The reflectors go to global scratch.
//  2. Bisection by Sturm counts: one round with a count at each of 512
//     points over the Gershgorin interval, then each warp refines the
//     brackets of two wanted eigenvalues at once by three rounds of 33-point
//     multisection.
//  3. Inverse iteration on the tridiagonal T (pivoted LU), one thread per
//     wanted eigenvalue, two rounds of one solve each, and
//  4. after each round an orthonormalisation of the r vectors by Cholesky
//     QR twice (columns in descending eigenvalue order, so the result is
//     the Gram-Schmidt basis), or Gram-Schmidt twice when a Cholesky pivot
//     is too small.
//  5. Back-transformation by the stored reflectors, four at a time, a warp
//     per two vectors held in registers.
#include <float.h>

#include <utility>

#include "chol.cuh"
#include "cluster_la.cuh"
#include "common.cuh"
#include "kernels.h"

namespace ttr {

namespace {

constexpr int ER_KTMAX = 5;
constexpr int ER_TRI_WARPS = 8;          // warps of the tridiagonalisation CTA (16 measured slower)

// Compile-time loop: f(integral_constant<int, 0>) ... f(<N - 1>), so that
// register-tile indices are constants however large the unrolled body.
template <int I>
struct CIdx {
  static constexpr int value = I;
  __host__ __device__ constexpr operator int() const { return I; }
};
template <typename F, int... I>
__device__ __forceinline__ void sfor_impl(F& f, std::integer_sequence<int, I...>) {
  (f(CIdx<I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}

__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Number of eigenvalues of T = (d, e) below x (Sturm sequence of the LDL^T
// pivots); e2 holds the squared off-diagonal.
__device__ __forceinline__ int sturm(const float* d, const float* e2, int k, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
#pragma unroll 4
  for (int i = 1; i < k; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// Two Sturm counts (at x0 and x1) in one pass, so that the two dependent
// chains overlap.
__device__ __forceinline__ void sturm2(const float* d, const float* e2, int k, float x0, float x1, float pivmin,
                                       int& c0, int& c1) {
  float q0 = d[0] - x0, q1 = d[0] - x1;
  if (fabsf(q0) < pivmin) q0 = -pivmin;
  if (fabsf(q1) < pivmin) q1 = -pivmin;
  c0 = q0 < 0.f;
  c1 = q1 < 0.f;
#pragma unroll 4
  for (int i = 1; i < k; ++i) {
    const float di = d[i], ei = e2[i - 1];
    q0 = (di - x0) - __fdividef(ei, q0);
    q1 = (di - x1) - __fdividef(ei, q1);
    if (fabsf(q0) < pivmin) q0 = -pivmin;
    if (fabsf(q1) < pivmin) q1 = -pivmin;
    c0 += q0 < 0.f;
    c1 += q1 < 0.f;
  }
}

// Pivoted LU of T - lam I into w[0..5k) (reciprocal pivots, two upper
// diagonals, multipliers, exchange flags); tiny pivots replaced by +-tiny.
__device__ void tri_lu(const float* d, const float* e, int k, float lam, float tiny, float* w) {
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
      const float rp = __fdividef(1.f, piv);
      const float li = sub * rp;
      r0[i] = rp; u1[i] = beta; u2[i] = 0.f; l[i] = li; sw[i] = 0.f;
      alpha = fmaf(-li, beta, a1);
      beta = c1;
    } else {
      const float rs = __fdividef(1.f, (fabsf(sub) < tiny) ? copysignf(tiny, sub) : sub);
      const float li = alpha * rs;
      r0[i] = rs; u1[i] = a1; u2[i] = c1; l[i] = li; sw[i] = 1.f;
      alpha = fmaf(-li, a1, beta);
      beta = -li * c1;
    }
  }
  r0[k - 1] = __fdividef(1.f, (fabsf(alpha) < tiny) ? copysignf(tiny, alpha) : alpha);
  u1[k - 1] = 0.f; u2[k - 1] = 0.f; l[k - 1] = 0.f; sw[k - 1] = 0.f;
}

__device__ void tri_lu_solve(const float* w, int k, float* x) {
  const float* r0 = w;
  const float* u1 = w + k;
  const float* u2 = w + 2 * k;
  const float* l = w + 3 * k;
  const float* sw = w + 4 * k;
  float xi = x[0];
  for (int i = 0; i + 1 < k; ++i) {
    float xn = x[i + 1];
    if (sw[i] != 0.f) { const float t = xi; xi = xn; xn = t; }
    x[i] = xi;
    xi = fmaf(-l[i], xi, xn);
  }
  x[k - 1] = xi;
  float x1 = 0.f, x2 = 0.f;
  for (int i = k - 1; i >= 0; --i) {
    const float v = (x[i] - u1[i] * x1 - u2[i] * x2) * r0[i];
    x[i] = v;
    x2 = x1;
    x1 = v;
  }
}

}  // namespace

// Shared-memory floats of k_eig_vectors for k (padded to KM = 32 KT) and r.
// Odd row strides for the vectors (k + 1 or k + 2) and the per-vector
// inverse-iteration factors (5 k or 5 k + 1): one thread per vector walks
// its row, so an odd stride keeps the 32 threads on 32 banks.
__host__ __device__ inline int er_ldx(int k) { return (k + 1) | 1; }
__host__ __device__ inline int er_ldw(int k) { return (5 * k) | 1; }
__host__ __device__ inline size_t er_union_floats(int k, int r) {
  const size_t a = (size_t)k * k, b = (size_t)r * er_ldw(k);
  return a > b ? a : b;
}
__host__ __device__ inline size_t er_smem_floats(int KM, int k, int r) {
  return er_union_floats(k, r) + 4 * (size_t)KM + 32 + 64 + 1024 + 2 * (size_t)r * er_ldx(k) + 3 * 33 * 32 + 8;
}

// Sum over the 32 lanes of NV values x[0..NV) (NV a power of two <= 32) with
// the transposing butterfly: at each level a lane keeps half of its values
// and sends the other half, so after log2(NV) levels every lane holds one
// partial sum; the remaining levels are plain butterflies.  Lane l ends with
// the total of value (l >> (5 - log2 NV)).
template <int NV>
__device__ __forceinline__ float lane_transpose_sum(float (&x)[NV]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  float cur[NV];
  sfor<NV>([&](auto i) { cur[i] = x[i]; });
  int n = NV, o = 16;
  // levels that halve the value count (compile-time sizes via sfor)
  sfor<5>([&](auto lvl) {
    constexpr int L = decltype(lvl)::value;
    constexpr int N = NV >> L;          // values held before this level
    if constexpr (N >= 2) {
      constexpr int H = N / 2;
      const int off = 16 >> L;
      const bool up = lane & off;
      sfor<H>([&](auto i) {
        const float send = up ? cur[i] : cur[i + H];
        const float keep = up ? cur[i + H] : cur[i];
        cur[i] = keep + __shfl_xor_sync(full, send, off);
      });
    } else {
      const int off = 16 >> L;
      cur[0] += __shfl_xor_sync(full, cur[0], off);
    }
  });
  (void)n;
  (void)o;
  return cur[0];
}

// Step 1 in one CTA of 8 warps: T = (d, e) and the reflectors (row j of
// Vg = v_j, tau[j]) to global scratch.  Thread (warp w, lane l) holds the
// entries (l + 32 a, w + 8 c), a < KR, c < 4 KR, so every column lives in one
// warp and each thread carries 20 KR entries (the per-column reductions,
// broadcasts and barriers are spread over many multiply-adds).  Per column
// two barriers:
//   R  the warp owning column j forms the reflector v (and tau) from its
//      registers and publishes it;
//   M  every warp forms tau (H v)_c for its columns c (H is symmetric, so the
//      column dot is the row product) and its share of v^T H v, reduced over
//      the lanes by one transposing butterfly;
//   U  every thread applies H -= v w^T + w v^T, w = p - (tau/2)(v^T p) v,
//      to its entries of the trailing block.
// Tiles of finished rows (32-row blocks) and columns (8-column slots) are
// skipped at compile time: the column loop is split into 32-column segments.
template <int KR, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_eig_tridiag8(const float* __restrict__ Hin, int64_t ldh, int k,
                                                        float* __restrict__ Vg, float* __restrict__ tau_g,
                                                        float* __restrict__ d_g, float* __restrict__ e_g) {
  constexpr int SPS = 32 / NW;            // column slots per warp in a 32-column segment
  constexpr int KC = SPS * KR;
  constexpr int KM = 32 * KR;
  constexpr int NV = (KC + 1 <= 8) ? 8 : (KC + 1 <= 16) ? 16 : 32;
  __shared__ __align__(16) float vs[KM];
  __shared__ __align__(16) float ps[KM];
  __shared__ float wsum[NW];
  __shared__ float scal[2];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  float A[KR][KC];   // A[a][c] = H[lane + 32 a][w + NW c]
  sfor<KR>([&](auto a) {
    sfor<KC>([&](auto c) {
      const int i = lane + 32 * a, j = w + NW * c;
      A[a][c] = (i < k && j < k) ? 0.5f * (Hin[(int64_t)i * ldh + j] + Hin[(int64_t)j * ldh + i]) : 0.f;
    });
  });
  const int z0 = (k >= 2) ? (k - 2) * k : 0;
  for (int x = z0 + tid; x < k * k; x += NW * 32) Vg[x] = 0.f;
  sfor<KR>([&](auto seg) {
    constexpr int S = decltype(seg)::value;
    const int jend = min(32 * S + 32, k - 2);
    for (int j = 32 * S; j < jend; ++j) {
      // R: the reflector of column j (slot j / NW in warp j % NW)
      if (w == (j % NW)) {
        const int t = (j / NW) - SPS * S;   // 0 .. SPS - 1
        float colv[KR];
        sfor<KR>([&](auto a) {
          float x = 0.f;
          if constexpr (a >= S) {
            sfor<SPS>([&](auto u) {
              if constexpr (SPS * S + u < KC)
                if (t == u) x = A[a][SPS * S + u];
            });
          }
          colv[a] = x;
        });
        float part = 0.f, sel = 0.f;
        const int a1 = (j + 1) >> 5;
        sfor<KR>([&](auto a) {
          if constexpr (a >= S) {
            const float x = colv[a];
            const int i = lane + 32 * a;
            if (i >= j + 2 && i < k) part = fmaf(x, x, part);
            if (a == a1) sel = x;
            if (i == j) d_g[j] = x;
          }
        });
        const float sigma = warp_sum(part);
        const float x0 = __shfl_sync(0xffffffffu, sel, (j + 1) & 31);
        float tt = 0.f, iv = 0.f, beta = x0;
        if (sigma > 0.f) {
          const float mu = sqrtf(fmaf(x0, x0, sigma));
          const float v0 = (x0 <= 0.f) ? x0 - mu : __fdividef(-sigma, x0 + mu);
          tt = __fdividef(2.f * v0 * v0, fmaf(v0, v0, sigma));
          beta = mu;
          iv = __fdividef(1.f, v0);
        }
        sfor<KR>([&](auto a) {
          const int i = lane + 32 * a;
          const float v = (a < S) ? 0.f : ((i == j + 1) ? 1.f : ((i > j + 1 && i < k) ? colv[a] * iv : 0.f));
          vs[i] = v;
          if (i < k) Vg[(size_t)j * k + i] = (tt != 0.f) ? v : 0.f;
        });
        if (lane == 0) {
          scal[j & 1] = tt;
          tau_g[j] = tt;
          e_g[j] = beta;
        }
      }
      __syncthreads();
      const float tau = scal[j & 1];
      if (tau == 0.f) continue;              // the same decision in every thread
      // M: (H v)_c for this thread's live columns, its share of v^T H v
      float vr[KR], vc[KC];
      sfor<KR>([&](auto a) { vr[a] = (a >= S) ? vs[lane + 32 * a] : 0.f; });
      sfor<KC>([&](auto c) { vc[c] = (c >= SPS * S) ? vs[w + NW * c] : 0.f; });
      float xv[NV];
      sfor<NV>([&](auto c) { xv[c] = 0.f; });
      sfor<KC>([&](auto c) {
        if constexpr (c >= SPS * S) {
          float acc = 0.f;
          sfor<KR>([&](auto a) {
            if constexpr (a >= S) acc = fmaf(A[a][c], vr[a], acc);
          });
          xv[c] = acc;
          xv[KC] = fmaf(vc[c], acc, xv[KC]);
        }
      });
      const float tot = lane_transpose_sum<NV>(xv);
      {
        constexpr int shift = (NV == 32) ? 0 : (NV == 16) ? 1 : 2;
        const int vi = lane >> shift;
        if ((lane & ((1 << shift) - 1)) == 0) {
          if (vi < KC) {
            const int col = w + NW * vi;
            if (col < KM) ps[col] = (col > j && col < k) ? tau * tot : 0.f;
          } else if (vi == KC) {
            wsum[w] = tot;
          }
        }
      }
      __syncthreads();
      // U: rank-2 update of the live tiles
      float vhv = 0.f;
#pragma unroll
      for (int q = 0; q < NW; ++q) vhv += wsum[q];
      const float K = 0.5f * tau * tau * vhv;
      float wr[KR], wc[KC];
      sfor<KR>([&](auto a) { wr[a] = (a >= S) ? fmaf(-K, vr[a], ps[lane + 32 * a]) : 0.f; });
      sfor<KC>([&](auto c) { wc[c] = (c >= SPS * S) ? fmaf(-K, vc[c], ps[w + NW * c]) : 0.f; });
      sfor<KR>([&](auto a) {
        if constexpr (a >= S) {
          sfor<KC>([&](auto c) {
            if constexpr (c >= SPS * S) A[a][c] -= fmaf(vr[a], wc[c], wr[a] * vc[c]);
          });
        }
      });
    }
  });
  // trailing 2 x 2 (or 1 x 1) block, written by the owners of its entries
  sfor<KR>([&](auto a) {
    sfor<KC>([&](auto c) {
      const int i = lane + 32 * a, jj = w + NW * c;
      if (k >= 2 && i == k - 2 && jj == k - 2) d_g[k - 2] = A[a][c];
      if (k >= 2 && i == k - 1 && jj == k - 2) e_g[k - 2] = A[a][c];
      if (i == k - 1 && jj == k - 1) d_g[k - 1] = A[a][c];
    });
  });
  if (tid == 0) {
    if (k >= 2) tau_g[k - 2] = 0.f;
    e_g[k - 1] = 0.f;
    tau_g[k - 1] = 0.f;
  }
}

// Step 5 for NV vectors held by one warp: x <- P_0 P_1 ... P_{k-3} x, the
// reflectors taken four at a time from the last (gg holds each group's six
// inner products), each vector's entries i = lane + 32 c in registers.
template <int KT, int NV>
__device__ __forceinline__ void back_transform_warp(const float* Vs, const float* tau, const float* gg, int k,
                                                    const float* cur, int ldx, const int (&js)[NV], float* V,
                                                    int ldv) {
  const int lane = threadIdx.x & 31;
  const int ng = (k - 2 + 3) / 4;
  float x[NV][KT];
#pragma unroll
  for (int u = 0; u < NV; ++u)
#pragma unroll
    for (int c = 0; c < KT; ++c) {
      const int i = lane + 32 * c;
      x[u][c] = (i < k) ? cur[(size_t)js[u] * ldx + i] : 0.f;
    }
  for (int g = 0; g < ng; ++g) {
    const int ht = k - 3 - 4 * g;
    const int c0 = (max(ht - 3, 0) + 1) >> 5;   // first chunk with a nonzero entry
    float v[4][KT];
    float dd[4 * NV];
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) dd[q] = 0.f;
#pragma unroll
    for (int c = 0; c < KT; ++c) {
      if (c >= c0) {                     // warp-uniform: chunks below c0 are zero
        const int i = lane + 32 * c;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          v[a][c] = (ht - a >= 0 && i < k) ? Vs[(size_t)(ht - a) * k + i] : 0.f;
#pragma unroll
          for (int u = 0; u < NV; ++u) dd[4 * u + a] = fmaf(v[a][c], x[u][c], dd[4 * u + a]);
        }
      }
    }
    // lane (32 / (4 NV)) q ends with the total of dd[q]
    const float tot = lane_transpose_sum<4 * NV>(dd);
    float d[4 * NV];
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) d[q] = __shfl_sync(0xffffffffu, tot, (32 / (4 * NV)) * q);
    const float* gq = gg + g * 8;
    const float g01 = gq[0], g02 = gq[1], g03 = gq[2], g12 = gq[3], g13 = gq[4], g23 = gq[5];
    float t[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) t[a] = (ht - a >= 0) ? tau[ht - a] : 0.f;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const float* du = d + 4 * u;
      const float c0v = t[0] * du[0];
      const float c1v = t[1] * fmaf(-g01, c0v, du[1]);
      const float c2v = t[2] * fmaf(-g12, c1v, fmaf(-g02, c0v, du[2]));
      const float c3v = t[3] * fmaf(-g23, c2v, fmaf(-g13, c1v, fmaf(-g03, c0v, du[3])));
#pragma unroll
      for (int c = 0; c < KT; ++c) {
        if (c >= c0) {
          float s = x[u][c];
          s = fmaf(-c0v, v[0][c], s);
          s = fmaf(-c1v, v[1][c], s);
          s = fmaf(-c2v, v[2][c], s);
          s = fmaf(-c3v, v[3][c], s);
          x[u][c] = s;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < KT; ++c) {
    const int i = lane + 32 * c;
    if (i < k)
#pragma unroll
      for (int u = 0; u < NV; ++u) V[(size_t)i * ldv + js[u]] = x[u][c];
  }
}

// Steps 2-5 in one CTA of 16 warps, from T and the reflectors in global
// scratch (the reflectors are staged in shared memory).
template <int KT>
__global__ void __launch_bounds__(512, 1) k_eig_vectors(const float* __restrict__ Vg, const float* __restrict__ tau_g,
                                                       const float* __restrict__ d_g, const float* __restrict__ e_g,
                                                       int k, int r, float* __restrict__ V, int ldv,
                                                       float* __restrict__ evals) {
  constexpr int NW = 16;
  constexpr int KM = 32 * KT;
  constexpr int NT = 32 * NW;
  extern __shared__ __align__(16) float sm[];
  // the reflectors (step 5) and the inverse-iteration factors (step 3) are
  // never live together: one region holds both
  float* Vs = sm;                         // [k][k], row j = reflector v_j
  float* Wk = sm;                         // [r][ldw] inverse-iteration factors
  float* tau = sm + er_union_floats(k, r);   // [KM]
  float* d = tau + KM;                    // [KM]
  float* e = d + KM;                      // [KM]
  float* e2 = e + KM;                     // [KM]
  float* lam = e2 + KM;                   // [32]
  float* red = lam + 32;                  // [64]
  int* cnt = reinterpret_cast<int*>(red + 64);   // [1024]
  float* X = reinterpret_cast<float*>(cnt + 1024);   // [r][ldx]
  float* X2 = X + (size_t)r * er_ldx(k);   // [r][ldx]
  float* G = X2 + (size_t)r * er_ldx(k);  // [32][33]
  float* Rm = G + 33 * 32;                // [32][32]
  float* Tm = Rm + 33 * 32;               // [32][32]
  int* sflag = reinterpret_cast<int*>(Tm + 33 * 32);
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  const int ldx = er_ldx(k);
  for (int i = tid; i < k; i += NT) {
    tau[i] = tau_g[i];
    d[i] = d_g[i];
    e[i] = e_g[i];
  }
  if (tid == 0) *sflag = 0;
  __syncthreads();

  // ---------------------------------------------------------------- 2
  float glo = FLT_MAX, ghi = -FLT_MAX, amax = 0.f;
  for (int i = tid; i < k; i += NT) {
    const float off = (i > 0 ? fabsf(e[i - 1]) : 0.f) + fabsf(e[i]);
    glo = fminf(glo, d[i] - off);
    ghi = fmaxf(ghi, d[i] + off);
    amax = fmaxf(amax, fmaxf(fabsf(d[i]), fabsf(e[i])));
    e2[i] = e[i] * e[i];
  }
  glo = warp_min_f(glo);
  ghi = warp_max_f(ghi);
  amax = warp_max_f(amax);
  if (lane == 0) {
    red[ty] = glo;
    red[32 + ty] = ghi;
    cnt[ty] = __float_as_int(amax);
  }
  __syncthreads();
  glo = warp_min_f(lane < NW ? red[lane] : FLT_MAX);
  ghi = warp_max_f(lane < NW ? red[32 + lane] : -FLT_MAX);
  amax = warp_max_f(lane < NW ? __int_as_float(cnt[lane]) : 0.f);
  __syncthreads();
  const float tnorm = fmaxf(amax, FLT_MIN);
  const float pivmin = FLT_MIN * fmaxf(1.f, tnorm * tnorm);
  const float pad = 2.f * FLT_EPSILON * tnorm + pivmin;
  const float lo0 = glo - pad, hi0 = ghi + pad;
  const float step = (hi0 - lo0) * (1.f / (float)(NT + 1));
  cnt[tid] = sturm(d, e2, k, fmaf((float)(tid + 1), step, lo0), pivmin);
  __syncthreads();
  // a warp refines the brackets of eigenvalues ty and ty + NW together
  // (two independent Sturm chains in flight)
  {
    const int j0 = ty, j1 = ty + NW;
    const bool has0 = j0 < r, has1 = j1 < r;
    auto bracket = [&](int jj, float& lo, float& hi) {
      const int want = k - jj;             // count reaching k - j brackets the j-th largest
      int first = NT;
      for (int u = 0; u < NW; ++u) {
        const int tt = lane * NW + u;
        if (cnt[tt] >= want) {
          first = tt;
          break;
        }
      }
      first = warp_min_i(first);
      lo = (first == 0) ? lo0 : fmaf((float)first, step, lo0);
      hi = (first == NT) ? hi0 : fmaf((float)(first + 1), step, lo0);
    };
    auto narrow = [&](int c, int want, float x, float& lo, float& hi) {
      const unsigned ge = __ballot_sync(0xffffffffu, c >= want);
      const int sidx = ge ? (__ffs(ge) - 1) : 32;
      const float xs = __shfl_sync(0xffffffffu, x, sidx < 32 ? sidx : 31);
      const float xp = __shfl_sync(0xffffffffu, x, sidx > 0 ? sidx - 1 : 0);
      if (sidx == 32) lo = xs;
      else {
        hi = xs;
        if (sidx > 0) lo = xp;
      }
    };
    float lo_0 = 0.f, hi_0 = 0.f, lo_1 = 0.f, hi_1 = 0.f;
    if (has0) bracket(j0, lo_0, hi_0);
    if (has1) bracket(j1, lo_1, hi_1);
    // three rounds: the bracket is then (span / 513) / 33^3 ~ 5e-8 of the
    // Gershgorin span, the resolution of FP32 itself
    for (int it = 0; it < 3 && has0; ++it) {
      const float x0 = lo_0 + (hi_0 - lo_0) * (float)(lane + 1) * (1.f / 33.f);
      if (has1) {
        const float x1 = lo_1 + (hi_1 - lo_1) * (float)(lane + 1) * (1.f / 33.f);
        int c0, c1;
        sturm2(d, e2, k, x0, x1, pivmin, c0, c1);
        narrow(c0, k - j0, x0, lo_0, hi_0);
        narrow(c1, k - j1, x1, lo_1, hi_1);
      } else {
        narrow(sturm(d, e2, k, x0, pivmin), k - j0, x0, lo_0, hi_0);
      }
    }
    if (lane == 0 && has0) lam[j0] = 0.5f * (lo_0 + hi_0);
    if (lane == 0 && has1) lam[j1] = 0.5f * (lo_1 + hi_1);
  }
  __syncthreads();

  // ---------------------------------------------------------------- 3
  // Two rounds of one inverse-iteration solve per vector followed by an
  // orthonormalisation of all r vectors (a subspace iteration): for nearly
  // equal eigenvalues the solves pull every vector towards the same
  // eigenvector, and orthonormalising after each single solve keeps the
  // remainders inside the cluster's invariant subspace.
  const float tiny = FLT_EPSILON * tnorm + pivmin;
  float* cur = X;
  float* nxt = X2;
  for (int round = 0; round < 2; ++round) {
    if (tid < r) {
      float* x = cur + (size_t)tid * ldx;
      float* w = Wk + (size_t)tid * er_ldw(k);
      if (round == 0) {
        tri_lu(d, e, k, lam[tid], tiny, w);
        // start vector 1 + 0.01 h(tid, i), h pseudo-random in [-1, 1) and
        // different for every vector: equal shifts (a cluster below FP32
        // resolution) must not produce equal vectors
        for (int i = 0; i < k; ++i) x[i] = fmaf(0.01f, hash_uniform(0xE16ull + (uint64_t)tid, (uint64_t)i), 1.f);
      }
      tri_lu_solve(w, k, x);
      float mx = 0.f;
      for (int i = 0; i < k; ++i) mx = fmaxf(mx, fabsf(x[i]));
      const float sc = mx > 0.f ? 1.f / mx : 0.f;
      for (int i = 0; i < k; ++i) x[i] *= sc;
    }
    __syncthreads();
    // the factors are dead after the last solve: stage the reflectors for
    // step 5 in their place while step 4 runs
    if (round == 1)
      for (int x = tid; x < k * k; x += NT) cp_async4(Vs + x, Vg + x, true);

  // ---------------------------------------------------------------- 4
    // one Cholesky QR pass keeps the vectors apart before the second solve;
    // two make the final ones orthonormal to working accuracy
    if (tid == 0) *sflag = 0;
    for (int pass = 0; pass < (round == 0 ? 1 : 2); ++pass) {
      for (int x = tid; x < r * r; x += NT) {
        const int a = x / r, b = x % r;
        if (b >= a) {
          float s0 = 0.f, s1 = 0.f;
          const float* xa = cur + (size_t)a * ldx;
          const float* xb = cur + (size_t)b * ldx;
          int i = 0;
          for (; i + 1 < k; i += 2) {
            s0 = fmaf(xa[i], xb[i], s0);
            s1 = fmaf(xa[i + 1], xb[i + 1], s1);
          }
          if (i < k) s0 = fmaf(xa[i], xb[i], s0);
          G[a * 33 + b] = s0 + s1;
        }
      }
      __syncthreads();
      if (round == 1 && pass == 1) {
        // after one Cholesky QR the Gram is usually within rounding of the
        // identity: then X (1.5 I - 0.5 G) (first-order polar correction,
        // orthogonality error O(|G - I|^2), same span) replaces the second
        float dev = 0.f;
        for (int x = tid; x < r * r; x += NT) {
          const int a = x / r, b = x % r;
          if (b >= a) dev = fmaxf(dev, fabsf(G[a * 33 + b] - (a == b ? 1.f : 0.f)));
        }
        dev = warp_max_f(dev);
        if (lane == 0) red[32 + ty] = dev;
        __syncthreads();
        dev = warp_max_f(lane < NW ? red[32 + lane] : 0.f);
        if (dev < 1e-4f) {                // the same decision in every thread
          for (int x = tid; x < r * r; x += NT) {
            const int a = x / r, b = x % r;
            const float g = (b >= a) ? G[a * 33 + b] : G[b * 33 + a];
            Tm[a * 33 + b] = (a == b ? 1.5f : 0.f) - 0.5f * g;
          }
          __syncthreads();
          for (int x = tid; x < r * k; x += NT) {
            const int j = x / k, i = x % k;
            float s = 0.f;
            for (int a = 0; a < r; ++a) s = fmaf(cur[(size_t)a * ldx + i], Tm[a * 33 + j], s);
            nxt[(size_t)j * ldx + i] = s;
          }
          __syncthreads();
          float* tmp = cur; cur = nxt; nxt = tmp;
          continue;
        }
        __syncthreads();
      }
      if (tid < r) red[tid] = G[tid * 33 + tid];
      chol_inv_warp32_call(G, 33, r, red, Rm, 33, Tm, 33, sflag, true);
      if (*sflag) break;                  // uniform: fall back below
      // nxt[j][i] = sum_{a <= j} cur[a][i] T[a][j]
      for (int x = tid; x < r * k; x += NT) {
        const int j = x / k, i = x % k;
        float s = 0.f;
        for (int a = 0; a <= j; ++a) s = fmaf(cur[(size_t)a * ldx + i], Tm[a * 33 + j], s);
        nxt[(size_t)j * ldx + i] = s;
      }
      __syncthreads();
      float* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (*sflag) {
      // Gram-Schmidt twice in descending eigenvalue order (a Cholesky pass
      // that was applied leaves the span of each leading set unchanged)
      for (int j = 0, attempt = 0; j < r;) {
        float* xj = cur + (size_t)j * ldx;
        float p0 = 0.f;
        for (int i = tid; i < k; i += NT) p0 = fmaf(xj[i], xj[i], p0);
        const float n0 = sqrtf(block_sum(p0, red));
        __syncthreads();
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
          for (int i2 = ty; i2 < j; i2 += NW) {
            const float* xi = cur + (size_t)i2 * ldx;
            float pp = 0.f;
            for (int i = lane; i < k; i += 32) pp = fmaf(xi[i], xj[i], pp);
            pp = warp_sum(pp);
            if (lane == 0) G[i2] = pp;
          }
          __syncthreads();
          for (int i = tid; i < k; i += NT) {
            float s0 = xj[i];
            for (int i2 = 0; i2 < j; ++i2) s0 = fmaf(-G[i2], cur[(size_t)i2 * ldx + i], s0);
            xj[i] = s0;
          }
          __syncthreads();
        }
        float pp = 0.f;
        for (int i = tid; i < k; i += NT) pp = fmaf(xj[i], xj[i], pp);
        const float nrm = sqrtf(block_sum(pp, red));
        __syncthreads();
        if (!(nrm > 1e-4f * n0) && attempt < 3) {
          // numerically inside the span of the earlier vectors (a cluster
          // below FP32 resolution): any direction orthogonal to them serves,
          // take a pseudo-random one through the same projections
          for (int i = tid; i < k; i += NT)
            xj[i] = hash_uniform(0x65A0ull + 64ull * (uint64_t)attempt + (uint64_t)j, (uint64_t)i);
          __syncthreads();
          ++attempt;
          continue;
        }
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        for (int i = tid; i < k; i += NT) xj[i] *= inv;
        __syncthreads();
        ++j;
        attempt = 0;
      }
    }
    __syncthreads();
  }

  // ---------------------------------------------------------------- 5
  cp_async_wait_all();
  __syncthreads();
  // x <- P_0 P_1 ... P_{k-3} x for the r vectors, reflectors taken four at a
  // time from the last.  For the group {h, h-1, h-2, h-3}, applied in that
  // order, the coefficients follow from the dots d_a = v_{h-a}^T x of the
  // group's incoming x and the group's inner products g_ab = v_{h-a}^T v_{h-b}:
  //   c_a = tau_{h-a} (d_a - sum_{b < a} g_ba c_b),   x -= sum_a c_a v_{h-a},
  // so a group costs one lane reduction where single reflectors cost four.
  // v_h is zero at indices <= h (and entirely where tau_h = 0), so a group
  // skips the 32-entry chunks below its lowest reflector.
  {
    const int ng = (k - 2 + 3) / 4;       // groups over reflectors 0 .. k-3
    float* gg = Tm;                       // [ng][8]: g01 g02 g03 g12 g13 g23
    for (int g = ty; g < ng; g += NW) {
      const int ht = k - 3 - 4 * g;
      float p6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < KT; ++c) {
        const int i = lane + 32 * c;
        float v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = (ht - a >= 0 && i < k) ? Vs[(size_t)(ht - a) * k + i] : 0.f;
        p6[0] = fmaf(v[0], v[1], p6[0]);
        p6[1] = fmaf(v[0], v[2], p6[1]);
        p6[2] = fmaf(v[0], v[3], p6[2]);
        p6[3] = fmaf(v[1], v[2], p6[3]);
        p6[4] = fmaf(v[1], v[3], p6[4]);
        p6[5] = fmaf(v[2], v[3], p6[5]);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) p6[q] = warp_sum(p6[q]);
      if (lane < 6) {
        float o = p6[0];
#pragma unroll
        for (int q = 1; q < 6; ++q) o = (lane == q) ? p6[q] : o;
        gg[g * 8 + lane] = o;
      }
    }
    __syncthreads();
    // warps ty < r - NW take vectors ty and ty + NW (each reflector read
    // once for both, their lane reductions merged), the others vector ty
    if (ty + NW < r) {
      const int js[2] = {ty, ty + NW};
      back_transform_warp<KT, 2>(Vs, tau, gg, k, cur, ldx, js, V, ldv);
    } else if (ty < r) {
      const int js[1] = {ty};
      back_transform_warp<KT, 1>(Vs, tau, gg, k, cur, ldx, js, V, ldv);
    }
    if (evals)
      for (int j = tid; j < r; j += NT) evals[j] = lam[j];
  }
}

// ------------------------------------------------------------ launcher
static int er_kt(int k) { return (k + 31) / 32; }

bool eig_reg_ok(int k, int r) {
  if (k < 1 || r < 1 || r > 32 || r > k || k > 32 * ER_KTMAX) return false;
  // dynamic shared memory plus the kernel's static arrays (the Cholesky's
  // 4.5 KB of R rows) within the 227 KB a CTA may use
  return er_smem_floats(32 * er_kt(k), k, r) * 4 + 6 * 1024 <= 227 * 1024;
}

template <int KT>
static cudaError_t launch_kt(const float* H, int64_t ldh, int k, int r, float* V, int ldv, float* evals,
                             float* scratch, cudaStream_t st) {
  float* Vg = scratch;
  float* tau = Vg + (size_t)k * k;
  float* d = tau + k;
  float* e = d + k;
  k_eig_tridiag8<KT, ER_TRI_WARPS><<<1, ER_TRI_WARPS * 32, 0, st>>>(H, ldh, k, Vg, tau, d, e);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const size_t smem = er_smem_floats(32 * KT, k, r) * 4;
  err = raise_smem_limit(k_eig_vectors<KT>);
  if (err != cudaSuccess) return err;
  k_eig_vectors<KT><<<1, 512, smem, st>>>(Vg, tau, d, e, k, r, V, ldv, evals);
  return cudaGetLastError();
}

// scratch: k * k + 3 k floats (device)
cudaError_t launch_eig_reg(const float* H, int64_t ldh, int k, int r, float* V, int ldv, float* evals,
                           float* scratch, cudaStream_t st) {
  if (!eig_reg_ok(k, r)) return cudaErrorInvalidValue;
  ProfScope prof("eig_top", st, 0, 0);
  note_launch("eig_top", 2);
  switch (er_kt(k)) {
    case 1: return launch_kt<1>(H, ldh, k, r, V, ldv, evals, scratch, st);
    case 2: return launch_kt<2>(H, ldh, k, r, V, ldv, evals, scratch, st);
    case 3: return launch_kt<3>(H, ldh, k, r, V, ldv, evals, scratch, st);
    case 4: return launch_kt<4>(H, ldh, k, r, V, ldv, evals, scratch, st);
    default: return launch_kt<5>(H, ldh, k, r, V, ldv, evals, scratch, st);
  }
}

}  // namespace ttr
