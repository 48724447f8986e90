// Block orthonormalisation of one Krylov block (Alg. 3 step 5) in a single
// launch on one thread-block cluster.
//
// The NC CTAs of the cluster split the m rows of the block Z (and of the
// basis Q).  Each phase transforms the CTA's rows, forms the CTA's share of
// Q^T Z and/or Z^T Z in its own shared memory, and after one cluster barrier
// every CTA sums all NC shares in rank order through distributed shared
// memory (so all CTAs hold identical sums and repeat the small b x b
// factorisations themselves).  Shares are double-buffered by phase parity,
// so one barrier per phase suffices.  The sequence is that of orth.cu:
//   A: Z = W;                 P1 = Q^T Z
//   B: Z -= Q P1;             P2 = Q^T Z                 (block Gram-Schmidt twice)
//   C: Z -= Q P2;             R1 = chol(Z^T Z + s I)     (shifted CholeskyQR)
//   D: Z = Z R1^-1;           P3 = Q^T Z, R2 = chol(Z^T Z)
//   E: Z = (Z - Q P3) R2^-1;  R3 = chol(Z^T Z)
//   F: X = Z R3^-1 -> Q[:, kq:kq+b]  (X = Z (1.5 I - 0.5 Z^T Z) when Z^T Z
//      is within 1e-4 of the identity in every entry)
// (C, D, E, F without Q terms for the first block).  The Krylov power
// blocks are typically far from orthogonal (their columns lean towards the
// dominant directions), so the shift is always applied.  A pivot below 1e-6 of
// its diagonal sets the breakdown flag for the one-CTA robust path.
// When the Krylov dimension cap keeps only c < b columns, the projected Z
// has (with probability one) rank c: its range is the part of range(C), or
// of R^m, not yet in span(Q).  Phase C then selects c columns by greedy
// diagonal pivoting of the shifted Cholesky, which spans that range, and
// D-F carry c columns.
// All products use 4 x 4 register tiles over shared arrays whose row
// strides are padded to multiples of 4 with zeros.
#include "chol.cuh"
#include "cluster_la.cuh"
#include "kernels.h"

namespace ttr {

constexpr int OC_THREADS = 512;

struct ClusterOrthArgs {
  const float* W;
  int64_t ldw;
  float* Q;
  int64_t ldq;
  int kq;
  int64_t m;
  int b;
  int64_t rows;     // rows per CTA
  int c;            // columns kept (c <= b; c < b under the dimension cap)
  int* flag;
};

// Shared-memory layout (floats), kp = pad4(kq), bp = pad4(b), rp = pad4(rows):
//   share[2][(kp + bp) * bp] | P[kp * bp] | G[b * (b + 1)] | T[bp * bp] | R[b * b] (sizes padded to 4)
//   | diag0[64] | red[64] | perm[64] | dsw[64] | Z[rp * bp] | Z2[rp * bp] | Qc[rp * kp]
__host__ __device__ inline size_t oc_smem_floats(int kq, int b, int64_t rows) {
  const size_t kp = pad4(kq), bp = pad4(b), rp = pad4((int)rows);
  return 2 * (kp + bp) * bp + kp * bp + pad4(b * (b + 1)) + bp * bp + pad4(b * b) + 256 + 2 * rp * bp + rp * kp;
}

__global__ void __launch_bounds__(OC_THREADS, 1) k_orth_cluster(ClusterOrthArgs a) {
  extern __shared__ __align__(16) float sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int kq = a.kq, b = a.b, tid = threadIdx.x;
  const int kp = pad4(kq), bp = pad4(b), rp = pad4((int)a.rows);
  const unsigned rank = cl.block_rank();
  const int64_t r0 = (int64_t)rank * a.rows;
  const int rc = (int)imax(0, imin(a.rows, a.m - r0));
  const int E = (kp + bp) * bp;
  float* share0 = sm;
  float* share1 = share0 + E;
  float* P = share1 + E;
  float* G = P + kp * bp;
  float* T = G + pad4(b * (b + 1));      // every region starts 16-byte aligned
  float* R = T + bp * bp;
  float* diag0 = R + pad4(b * b);
  float* red = diag0 + 64;
  int* perm = reinterpret_cast<int*>(red + 64);
  float* dsw = red + 128;
  float* Zc = red + 192;       // current rows
  float* Zn = Zc + rp * bp;    // scratch rows
  float* Qc = Zn + rp * bp;
  const bool report = rank == 0;

  // zero-padded copies of the CTA's rows of Q and W by asynchronous copies
  // (a warp per row, lanes along the row; padding entries are zero-filled
  // copies that read nothing), all in flight together; zero T and P
  {
    const int lane = tid & 31, nw = blockDim.x >> 5;
    for (int i = tid >> 5; i < rp; i += nw) {
      const bool row_ok = i < rc;
      const float* qrow = row_ok ? a.Q + (r0 + i) * a.ldq : a.Q;
      const float* wrow = row_ok ? a.W + (r0 + i) * a.ldw : a.W;
      for (int t = lane; t < kp; t += 32) {
        const bool ok = row_ok && t < kq;
        cp_async4(&Qc[i * kp + t], ok ? qrow + t : a.Q, ok);
      }
      for (int j = lane; j < bp; j += 32) {
        const bool ok = row_ok && j < b;
        cp_async4(&Zc[i * bp + j], ok ? wrow + j : a.W, ok);
        Zn[i * bp + j] = 0.f;
      }
    }
    cp_async_wait_all();
  }
  for (int x = tid; x < bp * bp; x += blockDim.x) T[x] = 0.f;
  for (int x = tid; x < kp * bp; x += blockDim.x) P[x] = 0.f;
  __syncthreads();

  int phase = 0;
  // shares of Q^T Z (rows < kp) and/or Z^T Z (rows kp..kp+bp) over this
  // CTA's rows, then the rank-ordered sum into P and G
  auto reduce = [&](bool qz, bool zz) {
    float* mine = (phase & 1) ? share1 : share0;
    if (qz) tn_tile(Qc, kp, kp, Zc, bp, bp, rp, mine, bp);
    if (zz) tn_tile(Zc, bp, bp, Zc, bp, bp, rp, mine + kp * bp, bp);
    cl.sync();
    const int e0 = qz ? 0 : kp * bp, e1 = zz ? E : kp * bp;
    auto put = [&](int e, float s) {
      const int row = e / bp, j = e % bp;
      if (row < kp) P[e] = s;
      else if (row - kp < b && j < b) G[(row - kp) * (b + 1) + j] = s;
    };
    switch (cl.num_blocks()) {
      case 8: sum_ranks<8>(cl, mine, e0, e1, put); break;
      case 4: sum_ranks<4>(cl, mine, e0, e1, put); break;
      default: sum_ranks<1>(cl, mine, e0, e1, put); break;
    }
    __syncthreads();
    ++phase;
  };
  auto swap = [&]() { float* t = Zc; Zc = Zn; Zn = t; };
  auto sub_q = [&]() {     // Z = Z - Q P
    nn_tile(Qc, kp, kp, P, bp, rp, bp, Zn, bp, Zc, -1.f);
    __syncthreads();
    swap();
  };
  auto mul_t = [&]() {     // Z = Z T
    nn_tile(Zc, bp, bp, T, bp, rp, bp, Zn, bp, nullptr, 1.f);
    __syncthreads();
    swap();
  };
  auto set_diag0 = [&]() {
    for (int i = tid; i < b; i += blockDim.x) diag0[i] = G[i * (b + 1) + i];
    __syncthreads();
  };
  const int c = a.c;
  auto factor = [&](int bc, int* fl, bool rep) {
    if (bc < b) {
      for (int x = tid; x < bp * bp; x += blockDim.x) T[x] = 0.f;
      __syncthreads();
    }
    chol_inv_fast(G, b + 1, bc, diag0, R, b, T, bp, fl, rep);
  };
  auto write_q = [&](int cols) {
    for (int x = tid; x < rc * cols; x += blockDim.x) {
      const int i = x / cols, j = x % cols;
      a.Q[(r0 + i) * a.ldq + kq + j] = Zc[i * bp + j];
    }
  };

  if (kq > 0) {
    reduce(true, false);                       // A
    sub_q();
    reduce(true, false);                       // B
    sub_q();
  }
  // C, D, E: three Cholesky QR passes
  for (int pass = 0; pass < 3; ++pass) {
    reduce(pass == 1 && kq > 0, true);
    set_diag0();
    if (pass == 0) {
      // shifted Cholesky QR first: Krylov power blocks lean towards the
      // dominant directions, so their Gram is far from the identity
      float tr = 0.f;
      for (int i = tid; i < b; i += blockDim.x) tr += G[i * (b + 1) + i];
      tr = block_sum(tr, red);
      const float shift = 11.f * ((float)a.m * b + (float)b * (b + 1)) * 5.9604645e-08f * tr;
      __syncthreads();
      for (int i = tid; i < b; i += blockDim.x) G[i * (b + 1) + i] += shift;
    }
    // pass 1: Z^T Z stands in for the Gram of Z - Q P3 (after the block
    // Gram-Schmidt passes P3 = Q^T Z is at rounding level relative to Z, so
    // P3^T P3 is second order, and pass 2 restores orthonormality anyway)
    bool polar = false;
    if (pass == 2) {
      // the last pass usually finds the Gram within rounding of the
      // identity: then Z (1.5 I - 0.5 G) (first-order polar correction,
      // orthogonality error O(|G - I|^2), same span) replaces the Cholesky
      float e = 0.f;
      for (int x = tid; x < c * c; x += blockDim.x) {
        const int i = x / c, j = x % c;
        e = fmaxf(e, fabsf(G[i * (b + 1) + j] - (i == j ? 1.f : 0.f)));
      }
      e = warp_max(e);
      __syncthreads();
      if ((tid & 31) == 0) red[tid >> 5] = e;
      __syncthreads();
      e = warp_max((tid & 31) < (int)(blockDim.x >> 5) ? red[tid & 31] : 0.f);
      polar = e < 1e-4f;                     // the same in every thread
      if (polar) {
        for (int x = tid; x < bp * bp; x += blockDim.x) {
          const int i = x / bp, j = x % bp;
          T[x] = (i < c && j < c) ? (i == j ? 1.5f : 0.f) - 0.5f * G[i * (b + 1) + j] : 0.f;
        }
        __syncthreads();
      }
    }
    if (pass == 0 && c < b)
      pchol_select_cta(G, b + 1, b, c, diag0, R, b, T, bp, bp, perm, dsw, a.flag, report);
    else if (!polar)
      factor(pass == 0 ? b : c, a.flag, report);
    if (pass == 1 && kq > 0) sub_q();
    mul_t();
  }
  write_q(c);
  cl.sync();   // no CTA leaves while others may still read its shares
}

// ------------------------------------------------------------ launcher
constexpr int kOcSmemMax = 200 * 1024;

static int oc_cluster_size(int64_t m) {
  if (m <= 64) return 1;
  if (m <= 256) return 4;
  return 8;
}

bool orth_cluster_ok(int64_t m, int kq, int b) {
  if (b > 64 || kq > 256) return false;
  const int64_t rows = ceil_div(m, oc_cluster_size(m));
  return oc_smem_floats(kq, b, rows) * 4 <= kOcSmemMax;
}

cudaError_t launch_orth_cluster(const float* W, int64_t ldw, int64_t m, int b, int c, float* Q, int64_t ldq, int kq,
                                int* flag, cudaStream_t st) {
  if (!orth_cluster_ok(m, kq, b) || c < 1 || c > b) return cudaErrorInvalidValue;
  ClusterOrthArgs a;
  a.W = W; a.ldw = ldw; a.Q = Q; a.ldq = ldq; a.kq = kq; a.m = m; a.b = b; a.c = c; a.flag = flag;
  const int nc = oc_cluster_size(m);
  a.rows = ceil_div(m, nc);
  const size_t smem = oc_smem_floats(kq, b, a.rows) * 4;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = raise_smem_limit(k_orth_cluster);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(OC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope prof("orth_cluster", st, 0, 0);
  note_launch("orth_cluster");
  e = cudaLaunchKernelEx(&cfg, k_orth_cluster, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ttr
