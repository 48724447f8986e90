// Block orthonormalisation of one Krylov block (Alg. 3 step 5) across many
// CTAs.  The m x b block Z and the basis Q (m x kq) are split by rows; each
// launch ("phase") transforms the CTA's rows, computes its rows' share of
// Q^T Z and/or Z^T Z, and the CTA that finishes last (atomic ticket, no
// waiting) sums the shares in CTA order and factors the b x b Gram.
//
// Sequence for a block with an existing basis (kq > 0):
//   A: Z = W;                share Q^T Z  -> P1
//   B: Z -= Q P1;            share Q^T Z  -> P2          (block Gram-Schmidt, twice)
//   C: Z -= Q P2;            share Z^T Z  -> R1 = chol(G + s I)   (shifted CholeskyQR)
//   D: Z = Z R1^-1;          shares Q^T Z, Z^T Z -> P3, R2 = chol(G - P3^T P3)
//   E: Z = (Z - Q P3) R2^-1; share Z^T Z  -> R3 = chol(G)
//   F: X = Z R3^-1 -> Q[:, kq:kq+b]
// For the first block (kq = 0) the sequence is C, D, E, F without Q terms.
// The shift s = 11 (m b + b (b + 1)) u tr(G) follows Fukaya et al. (2020),
// with tr(G) bounding ||Z||_2^2.  A Cholesky pivot below 1e-6 of its
// diagonal raises a flag; the one-CTA robust path then redoes the block.
#include "chol.cuh"
#include "common.cuh"
#include "kernels.h"

namespace ttr {

constexpr int ORTH_THREADS = 512;

enum : int { IN_COPY = 0, IN_SUBQ = 1, IN_TRI = 2, IN_SUBQ_TRI = 3 };
enum : int { PROD_QZ = 1, PROD_ZZ = 2 };
enum : int { FIN_P = 0, FIN_SHIFTED = 1, FIN_PROJ_CHOL = 2, FIN_CHOL = 3, FIN_NONE = 4 };

struct OrthArgs {
  const float* W;
  int64_t ldw;
  float* Z;          // m x b, row stride b
  float* Q;
  int64_t ldq;
  int kq;
  int64_t m;
  int b;
  int64_t rows;      // rows per CTA
  float* parts;      // nctas x (kq + b) x b
  float* P;          // kq x b (finisher output / next input)
  float* T;          // b x b upper-triangular inverse of the last Cholesky factor
  unsigned* ticket;
  int* flag;
};

// Finisher of the last CTA: sums the shares and factors.
__device__ void orth_finish(const OrthArgs& a, int nctas, int prod, int fin, float* sm) {
  const int kq = a.kq, b = a.b, tid = threadIdx.x;
  const int E = (kq + b) * b;
  const int rows_qz = (prod & PROD_QZ) ? kq : 0;
  float* G = sm;                       // [b][b+1]
  float* red = G + b * (b + 1);        // [64]
  // sum shares in CTA order
  for (int e = tid; e < E; e += blockDim.x) {
    const int row = e / b;
    const bool need = (row < kq) ? (prod & PROD_QZ) : (prod & PROD_ZZ);
    if (!need) continue;
    // four independent chains keep several loads in flight; fixed order
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int c = 0;
    for (; c + 4 <= nctas; c += 4) {
      s0 += __ldcg(a.parts + (int64_t)c * E + e);
      s1 += __ldcg(a.parts + (int64_t)(c + 1) * E + e);
      s2 += __ldcg(a.parts + (int64_t)(c + 2) * E + e);
      s3 += __ldcg(a.parts + (int64_t)(c + 3) * E + e);
    }
    for (; c < nctas; ++c) s0 += __ldcg(a.parts + (int64_t)c * E + e);
    const float s = (s0 + s1) + (s2 + s3);
    if (row < kq) a.P[e] = s;
    else G[(row - kq) * (b + 1) + e % b] = s;
  }
  __syncthreads();
  (void)rows_qz;
  if (fin == FIN_P || fin == FIN_NONE) return;
  float* diag0 = red + 64;             // [64]
  for (int i = tid; i < b; i += blockDim.x) diag0[i] = G[i * (b + 1) + i];
  __syncthreads();
  if (fin == FIN_PROJ_CHOL) {
    // Gram of the projected block: G - P3^T P3 (Q has orthonormal columns)
    for (int e = tid; e < b * b; e += blockDim.x) {
      const int i = e / b, j = e % b;
      float s = 0.f;
      for (int t = 0; t < kq; ++t) s = fmaf(a.P[t * b + i], a.P[t * b + j], s);
      G[i * (b + 1) + j] -= s;
    }
    __syncthreads();
  }
  if (fin == FIN_SHIFTED) {
    float tr = 0.f;
    for (int i = tid; i < b; i += blockDim.x) tr += G[i * (b + 1) + i];
    tr = block_sum(tr, red);
    const float shift = 11.f * ((float)a.m * b + (float)b * (b + 1)) * 5.9604645e-08f * tr;
    for (int i = tid; i < b; i += blockDim.x) G[i * (b + 1) + i] += shift;
    __syncthreads();
  }
  // Cholesky and triangular inverse in shared memory, then T to global
  float* Rs = diag0 + 64;              // [b][b]
  float* Ts = Rs + b * b;              // [b][b]
  chol_inv_fast(G, b + 1, b, diag0, Rs, b, Ts, b, a.flag, true);
  for (int e = tid; e < b * b; e += blockDim.x) a.T[e] = Ts[e];
}

__global__ void __launch_bounds__(ORTH_THREADS) k_orth_phase(OrthArgs a, int in_op, int prod, int fin, int out) {
  extern __shared__ float sm[];
  const int kq = a.kq, b = a.b, tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * a.rows;
  const int rc = (int)imin(a.rows, a.m - r0);
  const bool use_q = (in_op == IN_SUBQ || in_op == IN_SUBQ_TRI || (prod & PROD_QZ)) && kq > 0;
  float* Qs = sm;                                     // [rows][kq]
  float* Zs = Qs + (use_q ? a.rows * kq : 0);         // [rows][b]
  float* Ps = Zs + a.rows * b;                        // [kq][b]
  float* Ts = Ps + ((in_op == IN_SUBQ || in_op == IN_SUBQ_TRI) ? kq * b : 0);   // [b][b]
  if (use_q)
    for (int x = tid; x < rc * kq; x += blockDim.x) Qs[x] = a.Q[(r0 + x / kq) * a.ldq + x % kq];
  if (in_op == IN_COPY) {
    for (int x = tid; x < rc * b; x += blockDim.x) Zs[x] = a.W[(r0 + x / b) * a.ldw + x % b];
  } else {
    for (int x = tid; x < rc * b; x += blockDim.x) Zs[x] = a.Z[(r0 + x / b) * b + x % b];
  }
  if (in_op == IN_SUBQ || in_op == IN_SUBQ_TRI)
    for (int x = tid; x < kq * b; x += blockDim.x) Ps[x] = a.P[x];
  if (in_op == IN_TRI || in_op == IN_SUBQ_TRI)
    for (int x = tid; x < b * b; x += blockDim.x) Ts[x] = a.T[x];
  __syncthreads();
  // row transform
  if (in_op == IN_SUBQ || in_op == IN_SUBQ_TRI) {
    float vals[8];
    int n = 0;
    for (int x = tid; x < rc * b; x += blockDim.x, ++n) {
      const int i = x / b, j = x % b;
      float s = Zs[x];
      for (int t = 0; t < kq; ++t) s = fmaf(-Qs[i * kq + t], Ps[t * b + j], s);
      if (n < 8) vals[n] = s;
    }
    __syncthreads();
    n = 0;
    for (int x = tid; x < rc * b; x += blockDim.x, ++n)
      if (n < 8) Zs[x] = vals[n];
    __syncthreads();
  }
  if (in_op == IN_TRI || in_op == IN_SUBQ_TRI) {
    float vals[8];
    int n = 0;
    for (int x = tid; x < rc * b; x += blockDim.x, ++n) {
      const int i = x / b, j = x % b;
      float s = 0.f;
      for (int t = 0; t <= j; ++t) s = fmaf(Zs[i * b + t], Ts[t * b + j], s);
      if (n < 8) vals[n] = s;
    }
    __syncthreads();
    n = 0;
    for (int x = tid; x < rc * b; x += blockDim.x, ++n)
      if (n < 8) Zs[x] = vals[n];
    __syncthreads();
  }
  if (out) {
    for (int x = tid; x < rc * b; x += blockDim.x) a.Q[(r0 + x / b) * a.ldq + a.kq + x % b] = Zs[x];
    return;
  }
  for (int x = tid; x < rc * b; x += blockDim.x) a.Z[(r0 + x / b) * b + x % b] = Zs[x];
  // shares of Q^T Z and Z^T Z for these rows
  const int E = (kq + b) * b;
  float* share = a.parts + (int64_t)blockIdx.x * E;
  for (int e = tid; e < E; e += blockDim.x) {
    const int row = e / b, j = e % b;
    float s = 0.f;
    if (row < kq) {
      if (!(prod & PROD_QZ)) continue;
      for (int i = 0; i < rc; ++i) s = fmaf(Qs[i * kq + row], Zs[i * b + j], s);
    } else {
      if (!(prod & PROD_ZZ)) continue;
      const int c = row - kq;
      for (int i = 0; i < rc; ++i) s = fmaf(Zs[i * b + c], Zs[i * b + j], s);
    }
    share[e] = s;
  }
  // last CTA to arrive sums the shares and factors
  __threadfence();
  __syncthreads();
  __shared__ unsigned last;
  if (tid == 0) last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  orth_finish(a, gridDim.x, prod, fin, sm);
  if (tid == 0) *a.ticket = 0u;
}

// ------------------------------------------------------------ launchers
static int64_t orth_rows(int64_t m, int kq, int b) {
  int64_t rows = imax(32, ceil_div(m, 16));
  const int64_t budget = 180 * 1024 / 4 - (int64_t)kq * b - (int64_t)b * b;
  const int64_t per_row = kq + b;
  rows = imin(rows, imax(1, budget / per_row));
  // the row transform keeps at most 8 values per thread
  rows = imin(rows, (int64_t)8 * ORTH_THREADS / b);
  return imax(rows, 1);
}

size_t orth_fast_scratch_floats(int64_t m, int kq, int b) {
  const int64_t rows = orth_rows(m, kq, b);
  const int64_t nctas = ceil_div(m, rows);
  return (size_t)(m * b + nctas * (kq + b) * b + (int64_t)kq * b + (int64_t)b * b + 64);
}

bool orth_fast_ok(int64_t m, int kq, int b) { return b <= 64 && kq <= 256 && m >= 1; }

cudaError_t launch_orth_fast(const float* W, int64_t ldw, int64_t m, int b, float* Q, int64_t ldq, int kq,
                             float* scratch, unsigned* ticket, int* flag, cudaStream_t st) {
  OrthArgs a;
  a.W = W; a.ldw = ldw; a.Q = Q; a.ldq = ldq; a.kq = kq; a.m = m; a.b = b;
  a.rows = orth_rows(m, kq, b);
  const int nctas = (int)ceil_div(m, a.rows);
  a.Z = scratch;
  a.parts = a.Z + m * b;
  a.P = a.parts + (int64_t)nctas * (kq + b) * b;
  a.T = a.P + (int64_t)kq * b;
  a.ticket = ticket;
  a.flag = flag;
  const size_t smem_main = sizeof(float) * ((size_t)a.rows * (kq + b) + (size_t)kq * b + (size_t)b * b);
  const size_t smem_fin = sizeof(float) * ((size_t)b * (b + 1) + 128 + 2 * (size_t)b * b);
  const size_t smem = smem_main > smem_fin ? smem_main : smem_fin;
  raise_smem_limit(k_orth_phase);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  ProfScope prof("orth_fast", st, 0, 0);
  struct Ph { int in, prod, fin, out; };
  const Ph seq_q[6] = {{IN_COPY, PROD_QZ, FIN_P, 0}, {IN_SUBQ, PROD_QZ, FIN_P, 0},
                       {IN_SUBQ, PROD_ZZ, FIN_SHIFTED, 0}, {IN_TRI, PROD_QZ | PROD_ZZ, FIN_PROJ_CHOL, 0},
                       {IN_SUBQ_TRI, PROD_ZZ, FIN_CHOL, 0}, {IN_TRI, 0, FIN_NONE, 1}};
  const Ph seq_0[4] = {{IN_COPY, PROD_ZZ, FIN_SHIFTED, 0}, {IN_TRI, PROD_ZZ, FIN_CHOL, 0},
                       {IN_TRI, PROD_ZZ, FIN_CHOL, 0}, {IN_TRI, 0, FIN_NONE, 1}};
  const Ph* seq = kq > 0 ? seq_q : seq_0;
  const int nph = kq > 0 ? 6 : 4;
  for (int i = 0; i < nph; ++i) {
    note_launch("orth_fast");
    k_orth_phase<<<nctas, ORTH_THREADS, smem, st>>>(a, seq[i].in, seq[i].prod, seq[i].fin, seq[i].out);
  }
  return cudaGetLastError();
}

}  // namespace ttr
