// Host side of the C ABI: argument checks, the per-mode plan, the workspace
// layout and the mode loop of Alg. 3.  Everything is enqueued on the
// caller's stream without a host round trip.
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace {

thread_local std::string g_last_error;

tt_status fail(tt_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define TTR_CUDA(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(TT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));        \
  } while (0)

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }
size_t esize(int dt) { return dt == TT_BF16 ? 2 : 4; }

struct ModePlan {
  int64_t m = 0, n = 0, D = 0;
  int r_in = 1, r_out = 1, b = 0, kq = 0;
  std::vector<int> blocks;   // columns of X_0, X_1, ... (Krylov dimension cap applied)
  int iters = 0;             // subspace iteration: powers applied to the single block
  bool gram_route = false;   // exhaustion with D == m: one Gram pass
  bool gram_cols = false;    // exhaustion with D == n < m: the n x n Gram C^T C
  bool gram_power = false;   // short unfolding: G = C C^T formed once, each power W = G X
  bool fused_ga = false;     // Gram-apply fused in one pass over C
  bool literal = false;      // the paper's steps taken literally (first-r truncation)
  int64_t n_global = 0;      // columns of the whole unfolding (n: this rank's slab of them)
  int allreduces = 0;        // sums over the ranks this mode needs (sharded form)
  int64_t allreduce_floats = 0;
};

struct Plan {
  int d = 0, p = 0, q = 0;
  std::vector<int64_t> dims, rr;
  tt_options o{};
  int storage = TT_F32, remainder = TT_F32;
  std::vector<ModePlan> modes;
  // sharded form: this rank's slab [slab_lo, slab_lo + slab_w) of the last
  // mode (of size nd) and the callback that sums a device buffer over ranks
  int world = 1, rank = 0;
  int64_t slab_lo = 0, slab_w = 0, nd = 0;
  tt_allreduce_fn allreduce = nullptr;
  void* comm = nullptr;
  // workspace offsets in bytes
  size_t off_status = 0, off_R0 = 0, off_R1 = 0, off_S = 0, off_T = 0, off_part = 0, off_Y = 0,
         off_Q = 0, off_W = 0, off_U = 0, off_G = 0, off_small = 0, off_X = 0, off_Xg = 0, off_B = 0, off_Hd = 0,
         off_dfp = 0, off_part2 = 0, total = 0;
};

tt_status resolve_options(const tt_options* in, tt_options* out) {
  tt_rbki_default_options(out);
  if (in) *out = *in;
  if (out->storage != TT_F32 && out->storage != TT_BF16) return fail(TT_EINVAL, "options.storage must be TT_F32 or TT_BF16");
  if (out->remainder < 0) out->remainder = out->storage;
  if (out->remainder != TT_F32 && out->remainder != TT_BF16) return fail(TT_EINVAL, "options.remainder must be TT_F32 or TT_BF16");
  if (out->method != TT_METHOD_RBKI && out->method != TT_METHOD_RSI)
    return fail(TT_EINVAL, "options.method must be TT_METHOD_RBKI or TT_METHOD_RSI");
  if (out->gram_power != 0 && out->gram_power != 1) return fail(TT_EINVAL, "options.gram_power must be 0 or 1");
  if (out->paper_literal != 0 && out->paper_literal != 1) return fail(TT_EINVAL, "options.paper_literal must be 0 or 1");
  if (out->accurate_rr != 0 && out->accurate_rr != 1) return fail(TT_EINVAL, "options.accurate_rr must be 0 or 1");
  if (out->accurate_rr && out->paper_literal)
    return fail(TT_EINVAL, "options.accurate_rr and options.paper_literal exclude each other");
  if (out->reserved != 0) return fail(TT_EINVAL, "options.reserved must be zero");
  return TT_OK;
}

tt_status clamp(const int64_t* dims, int d, const int64_t* ranks, std::vector<int64_t>& rr) {
  if (!dims || !ranks) return fail(TT_EINVAL, "dims and ranks must not be NULL");
  if (d < 2 || d > 64) return fail(TT_EINVAL, "order d must be in [2, 64]");
  for (int k = 0; k < d; ++k)
    if (dims[k] < 1) return fail(TT_EINVAL, "mode sizes must be >= 1");
  for (int k = 0; k < d - 1; ++k)
    if (ranks[k] < 1) return fail(TT_EINVAL, "ranks must be >= 1");
  int64_t total = 1;
  for (int k = 0; k < d; ++k) {
    if (total > (int64_t(1) << 46) / dims[k]) return fail(TT_EINVAL, "tensor too large");
    total *= dims[k];
  }
  rr.assign(d + 1, 1);
  int64_t n = total;
  for (int k = 0; k < d - 1; ++k) {
    n /= dims[k];
    const int64_t m = rr[k] * dims[k];
    rr[k + 1] = std::min(ranks[k], std::min(m, n));
  }
  rr[d] = 1;
  return TT_OK;
}

tt_status build_plan(const int64_t* dims, int d, const int64_t* ranks, int p, int q, const tt_options* opts,
                     Plan& P, int world = 1, int rank = 0) {
  tt_status s = resolve_options(opts, &P.o);
  if (s != TT_OK) return s;
  if (p < 0 || q < 0) return fail(TT_EINVAL, "oversample and q must be >= 0");
  s = clamp(dims, d, ranks, P.rr);
  if (s != TT_OK) return s;
  if (world < 1 || rank < 0 || rank >= world) return fail(TT_EINVAL, "need 0 <= rank < world");
  if (world > dims[d - 1]) return fail(TT_EINVAL, "the last mode must have at least one index per rank");
  if (world > 1 && (P.o.paper_literal || P.o.accurate_rr))
    return fail(TT_EUNSUPPORTED, "the sharded form takes neither paper_literal nor accurate_rr");
  P.world = world;
  P.rank = rank;
  P.nd = dims[d - 1];
  {
    // contiguous slabs, the first ones one larger when I_d is not a multiple
    // of the world size: slab g = [ceil(g I_d / W), ceil((g + 1) I_d / W))
    const int64_t lo = ((int64_t)rank * P.nd + world - 1) / world;
    const int64_t hi = ((int64_t)(rank + 1) * P.nd + world - 1) / world;
    P.slab_lo = lo;
    P.slab_w = hi - lo;
  }
  P.d = d;
  P.p = p;
  P.q = q;
  P.dims.assign(dims, dims + d);
  P.storage = P.o.storage;
  P.remainder = P.o.remainder;
  P.modes.resize(d - 1);
  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= dims[k];
  int64_t n = total;
  size_t maxR = 0, maxS = 0, maxT = 0, maxPart = 0, maxY = 0, maxQ = 0, maxU = 0, maxG = 0, maxSmall = 0,
         maxX = 0, maxXg = 0, maxB = 0, maxHd = 0, maxDf = 0, maxPart2 = 0;
  for (int k = 0; k < d - 1; ++k) {
    ModePlan& M = P.modes[k];
    n /= dims[k];
    M.m = P.rr[k] * dims[k];
    M.n = n;
    M.r_in = (int)P.rr[k];
    M.r_out = (int)P.rr[k + 1];
    M.D = std::min(M.m, M.n);
    const int64_t b64 = (int64_t)M.r_out + p;
    if (b64 > 64) return fail(TT_EUNSUPPORTED, "r_k + p must be <= 64");
    M.b = (int)b64;
    int64_t cols = ttr::imin(M.b, M.D);
    M.blocks.assign(1, (int)cols);
    if (P.o.method == TT_METHOD_RSI) {
      // Alg. 4: one block, q powers (none once it spans all D directions)
      M.iters = (cols >= M.D) ? 0 : q;
    } else {
      for (int j = 1; j <= q; ++j) {
        if (cols >= M.D) break;
        const int64_t c = ttr::imin(M.b, M.D - cols);
        M.blocks.push_back((int)c);
        cols += c;
      }
    }
    M.kq = (int)cols;
    M.gram_route = P.o.exhaust_gram && cols == M.D && M.D == M.m && M.m <= 128;
    M.gram_cols = P.o.exhaust_gram && !M.gram_route && cols == M.D && M.D == M.n && M.n < M.m &&
                  ttr::eig_top_ok((int)M.n) && !P.o.accurate_rr && world == 1;
    if (P.o.accurate_rr && !M.gram_route && M.kq > ttr::RR_SVD_KMAX)
      return fail(TT_EUNSUPPORTED, "options.accurate_rr needs Krylov bases of at most 160 columns");
    if (P.o.paper_literal) {
      // Alg. 3 steps 4-8 (Alg. 4 steps 4-12, Alg. 2 for q = 0) taken
      // literally: the kept r columns span (C C^T)^s C W(:, 1:r), s = min(q, 1)
      // for Alg. 3 (only the first block of its right-side Krylov matrix
      // reaches the first r columns of qr(Y)) and s = q for Alg. 4
      M.literal = true;
      M.blocks.assign(1, M.r_out);
      M.kq = M.r_out;
      M.iters = (P.o.method == TT_METHOD_RSI) ? q : std::min(q, 1);
      M.gram_route = M.gram_cols = false;
    }
    M.fused_ga = ttr::simt_ga_fused_ok(M.m, M.b);
    // Krylov powers over a short unfolding (n <= 8192) are latency-bound
    // passes over few column tiles; when there are at least two, one Gram
    // G = C C^T (m^2 n flops, gram.cu) and small products W = G X replace
    // them.  For a BF16 unfolding of at most 1024 rows the tensor-core Gram
    // (2 m n flops per entry of C) also beats three or more streaming
    // passes (4 b flops per entry each, HBM-bound) at any n.  G stays below
    // 16 MB.
    {
      const size_t powers = M.literal ? (size_t)M.iters
                          : (P.o.method == TT_METHOD_RSI) ? (size_t)M.iters + 1 : M.blocks.size();
      const int cdt_k = (k == 0) ? P.storage : P.remainder;
      M.gram_power = P.o.gram_power && !M.gram_route && !M.gram_cols && ttr::gram_power_ok(M.m, M.b) &&
                     ((powers >= 2 && M.m <= 2048 && M.n <= 8192) ||
                      (cdt_k == TT_BF16 && powers >= 3 && M.m <= 1024 && M.n < (int64_t(1) << 31)));
    }
    if (!M.gram_route && !M.gram_cols && M.kq > 256)
      return fail(TT_EUNSUPPORTED, "Krylov basis larger than 256 columns");
    // sharded form (the routes are decided on the whole unfolding above):
    // this rank's columns, and the sums over ranks — the sketch and every
    // streamed power (m x b blocks), or the Gram once (m x m) on the Gram
    // routes; the column-Gram route needs every rank's columns and is off
    M.n_global = M.n;
    if (world > 1) {
      if (M.gram_cols) return fail(TT_EUNSUPPORTED, "internal: column Gram in the sharded form");
      M.n = M.n / P.nd * P.slab_w;
      const int powers = (P.o.method == TT_METHOD_RSI) ? M.iters + 1 : (int)M.blocks.size();
      if (M.gram_route) {
        M.allreduces = 1;
        M.allreduce_floats = M.m * M.m;
      } else if (M.gram_power) {
        M.allreduces = 2;
        M.allreduce_floats = M.m * M.b + M.m * M.m;
      } else {
        M.allreduces = 1 + powers;
        M.allreduce_floats = M.m * M.b * (1 + powers);
      }
    }
    // sizes
    maxR = std::max(maxR, (size_t)(M.r_out * M.n) * esize(P.remainder));
    if (M.gram_route) {
      maxPart = std::max(maxPart, (size_t)ttr::simt_gram_partials(M.m, M.n));
      maxG = std::max(maxG, (size_t)(M.m * M.m));
      maxSmall = std::max(maxSmall, ttr::rr_scratch_floats((int)M.m));
      maxSmall = std::max(maxSmall, ttr::rr_fast_scratch_floats(M.m, (int)M.m, M.r_out));
    } else if (M.gram_cols) {
      maxY = std::max(maxY, (size_t)(M.m * M.r_out));
      maxSmall = std::max(maxSmall, ttr::colgram_scratch_floats(M.m, (int)M.n, M.r_out));
      maxSmall = std::max(maxSmall, ttr::orth_scratch_floats(M.m, M.r_out, M.r_out));
      maxSmall = std::max(maxSmall, ttr::orth_fast_scratch_floats(M.m, 0, M.r_out));
    } else {
      maxS = std::max(maxS, (size_t)(M.b * M.n));
      maxPart = std::max(maxPart, (size_t)ttr::simt_cs_partials(M.m, M.n, M.b));
      if (M.fused_ga)
        maxPart = std::max(maxPart, (size_t)ttr::simt_ga_partials(M.m, M.n, M.b));
      else
        maxT = std::max(maxT, (size_t)(M.b * M.n));
      maxY = std::max(maxY, (size_t)(M.m * M.b));
      maxQ = std::max(maxQ, (size_t)(M.m * M.kq));
      maxSmall = std::max(maxSmall, ttr::orth_scratch_floats(M.m, M.b, M.kq));
      maxSmall = std::max(maxSmall, ttr::rr_scratch_floats(M.kq));
      maxSmall = std::max(maxSmall, ttr::orth_fast_scratch_floats(M.m, M.kq, M.b));
      // the last block's call has the largest basis: kq0 + c <= kq
      maxSmall = std::max(maxSmall, ttr::orth_grid_rs_scratch_floats(M.m, std::max(0, M.kq - M.b), M.b));
      maxSmall = std::max(maxSmall, ttr::rr_fast_scratch_floats(M.m, M.kq, M.r_out));
    }
    maxU = std::max(maxU, (size_t)(M.m * M.r_out));
    maxPart = std::max(maxPart, (size_t)(ttr::simt_proj_splits(M.m, M.n) * M.b * M.n));
    // tensor-core passes (BF16 unfoldings)
    const int cdt = (k == 0) ? P.storage : P.remainder;
    if (cdt == TT_BF16 && ttr::tc_shape_ok(M.m, M.n)) {
      maxPart = std::max(maxPart, (size_t)ttr::tc_cs_partials(M.m, M.n, M.b));
      maxPart = std::max(maxPart, (size_t)ttr::tc_ga_partials(M.m, M.n, M.b));
      if (M.m <= 128) maxPart = std::max(maxPart, (size_t)ttr::tc_gram_partials(M.m, M.n));
      maxX = std::max(maxX, ttr::tc_proj_scratch_bytes(M.m, M.b, 0));
      maxX = std::max(maxX, ttr::tc_proj_scratch_bytes(M.m, M.r_out, 1));
      maxX = std::max(maxX, ttr::tc_ga_scratch_bytes(M.m, M.b));
      if (!M.gram_route && !M.gram_cols) maxT = std::max(maxT, (size_t)(M.b * M.n));
    }
    if (M.gram_power) {
      maxG = std::max(maxG, (size_t)(M.m * M.m));
      maxPart = std::max(maxPart, ttr::gram_tiled_partials(M.m, M.n, cdt == TT_BF16 ? 1 : 0));
      // the Gram's own partials when it runs beside the sketch
      maxPart2 = std::max(maxPart2, (cdt == TT_BF16 && ttr::tc_shape_ok(M.m, M.n) && M.m <= 128)
                                        ? (size_t)ttr::tc_gram_partials(M.m, M.n)
                                        : ttr::gram_tiled_partials(M.m, M.n, cdt == TT_BF16 ? 1 : 0));
      // padded copy of the current block for the power
      maxXg = std::max(maxXg, (size_t)M.m * (size_t)((M.b + 3) & ~3));
    }
    if (P.o.accurate_rr && !M.gram_cols) {
      // B = Q^T C (kq x n; the row-exhaustion route takes B = C), the FP64
      // Gram B B^T and its per-CTA partials
      const int kk = M.gram_route ? (int)M.m : M.kq;
      if (!ttr::rr_svd_ok(kk, M.r_out)) return fail(TT_EUNSUPPORTED, "options.accurate_rr: basis too large");
      if (!M.gram_route) maxB = std::max(maxB, (size_t)M.kq * (size_t)M.n);
      maxHd = std::max(maxHd, (size_t)kk * kk);
      maxDf = std::max(maxDf, ttr::gram_df_partial_doubles(kk, M.n));
    }
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1)); return o; };
  P.off_status = take(256);
  P.off_R0 = take(maxR);
  P.off_R1 = take(maxR);
  P.off_S = take(maxS * 4);
  P.off_T = take(maxT * 4);
  P.off_part = take(maxPart * 4);
  P.off_Y = take(maxY * 4);
  P.off_Q = take(maxQ * 4);
  P.off_W = take(maxQ * 4);
  P.off_U = take(maxU * 4);
  P.off_G = take(maxG * 4);
  P.off_small = take(maxSmall * 4);
  P.off_X = take(maxX);
  P.off_Xg = take(maxXg * 4);
  P.off_B = take(maxB * 4);
  P.off_Hd = take(maxHd * 8);
  P.off_dfp = take(maxDf * 8);
  P.off_part2 = take(maxPart2 * 4);
  P.total = off;
  return TT_OK;
}

// A second stream (and its fork/join events) per host thread and device,
// created on first use and kept: work forked onto it is always joined back
// into the caller's stream before the call returns, so a capture in progress
// stays well formed.
struct AuxStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
AuxStream* aux_stream() {
  thread_local std::map<int, AuxStream> per_device;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  AuxStream& a = per_device[dev];
  if (!a.s) {
    if (cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess) {
      a = AuxStream{};
      return nullptr;
    }
  }
  return &a;
}

template <typename TIn>
tt_status run_mode(const Plan& P, int k, const TIn* C, char* ws, int* status, const float* omega_explicit,
                   uint64_t seed, float* core, cudaStream_t st, bool fork_ok) {
  const ModePlan& M = P.modes[k];
  constexpr bool kBf16 = std::is_same<TIn, __nv_bfloat16>::value;
  const bool use_tc = kBf16 && ttr::tc_shape_ok(M.m, M.n);
  const __nv_bfloat16* Cb = reinterpret_cast<const __nv_bfloat16*>(C);
  void* xs = ws + P.off_X;
  float* part = (float*)(ws + P.off_part);
  float* U = (float*)(ws + P.off_U);
  float* small = (float*)(ws + P.off_small);
  const int r = M.r_out;
  // sharded form: the sum of a partial block over the ranks (a no-op alone)
  auto sum_ranks = [&](float* buf, int64_t count) -> tt_status {
    if (P.world <= 1) return TT_OK;
    if (P.allreduce(buf, count, (void*)st, P.comm) != 0) return fail(TT_ECUDA, "allreduce callback failed");
    return TT_OK;
  };
  if (M.gram_route && P.o.accurate_rr) {
    // Alg. 3 steps 6-8 at exhaustion with B = C: the compensated Gram, FP64
    // Cholesky, one-sided Jacobi (rr_svd.cu)
    double* Hd = (double*)(ws + P.off_Hd);
    double* dfp = (double*)(ws + P.off_dfp);
    TTR_CUDA(ttr::gram_df<TIn>(C, (int)M.m, M.n, M.n, dfp, Hd, st));
    TTR_CUDA(ttr::launch_rr_svd(Hd, (int)M.m, r, nullptr, M.m, 0, U, core, status, st));
  } else if (M.gram_route) {
    float* G = (float*)(ws + P.off_G);
    if (use_tc && M.m <= 128)
      TTR_CUDA(ttr::tc_gram(Cb, M.m, M.n, part, G, status, st));
    else
      TTR_CUDA(ttr::simt_gram<TIn>(C, M.m, M.n, part, G, st));
    {
      const tt_status rs = sum_ranks(G, M.m * M.m);
      if (rs != TT_OK) return rs;
    }
    if (ttr::eig_top_ok((int)M.m))
      TTR_CUDA(ttr::launch_rr_fast(nullptr, G, M.m, M.m, (int)M.m, r, 1, small, U, core, st));
    else
      TTR_CUDA(ttr::launch_rayleigh_ritz(nullptr, G, M.m, M.m, (int)M.m, r, 1, small, U, core, st));
  } else if (M.gram_cols) {
    // exhaustion with D = n < m: the Krylov basis would span range(C), so
    // Rayleigh-Ritz would return the exact top-r left singular vectors;
    // they are orth(C V'), V' the top-r eigenvectors of the n x n Gram
    // C^T C (orthonormalising C v'_1, C v'_2, ... in order recovers
    // u_1, u_2, ... since C v'_j = sigma_j u_j)
    float* Y = (float*)(ws + P.off_Y);
    int* flag = status + 1;
    unsigned* ticket = reinterpret_cast<unsigned*>(status + 2);
    const uint64_t rseed = 0x5EEDull * (uint64_t)(k + 1);
    TTR_CUDA(ttr::launch_colgram<TIn>(C, M.m, (int)M.n, r, small, Y, st));
    if (ttr::orth_cluster_ok(M.m, 0, r)) {
      TTR_CUDA(ttr::launch_orth_cluster(Y, r, M.m, r, r, U, r, 0, flag, st));
      TTR_CUDA(ttr::launch_orth_block(Y, r, M.m, r, U, r, 0, r, small, rseed, status, flag, st));
    } else if (ttr::orth_fast_ok(M.m, 0, r)) {
      TTR_CUDA(ttr::launch_orth_fast(Y, r, M.m, r, U, r, 0, small, ticket, flag, st));
      TTR_CUDA(ttr::launch_orth_block(Y, r, M.m, r, U, r, 0, r, small, rseed, status, flag, st));
    } else {
      TTR_CUDA(ttr::launch_orth_block(Y, r, M.m, r, U, r, 0, r, small, rseed, status, nullptr, st));
    }
    TTR_CUDA(cudaMemcpyAsync(core, U, sizeof(float) * (size_t)M.m * r, cudaMemcpyDeviceToDevice, st));
  } else {
    float* S = (float*)(ws + P.off_S);
    float* T = (float*)(ws + P.off_T);
    float* Y = (float*)(ws + P.off_Y);
    float* Q = (float*)(ws + P.off_Q);
    float* W = (float*)(ws + P.off_W);
    const int kq = M.kq;
    // Alg. 3 step 3: Omega_k, stored transposed (b x n); BF16 for the tensor cores
    const int om_dt = use_tc ? TT_BF16 : TT_F32;
    if (omega_explicit)
      TTR_CUDA(ttr::launch_omega_transpose_any(omega_explicit, M.n, M.b, S, om_dt, st));
    else
      TTR_CUDA(ttr::launch_omega(seed, k, M.n, M.b, S, om_dt, 1, M.n, st, P.world > 1 ? P.slab_w : 0, P.nd,
                                 P.slab_lo));
    // Gram-power route: G = C C^T does not depend on the sketch, so on the
    // single-problem path it runs on a second stream beside the sketch and
    // the first block's orthonormalisation (tensor-bound Gram next to the
    // HBM-bound sketch), joined before the first power
    float* Gp = (float*)(ws + P.off_G);
    const bool fork = M.gram_power && fork_ok && P.world == 1;
    AuxStream* ax = fork ? aux_stream() : nullptr;
    if (fork && !ax) return fail(TT_ECUDA, "could not create the auxiliary stream");
    if (M.gram_power) {
      cudaStream_t gst = st;
      float* gpart = part;
      if (fork) {
        TTR_CUDA(cudaEventRecord(ax->fork, st));
        TTR_CUDA(cudaStreamWaitEvent(ax->s, ax->fork, 0));
        gst = ax->s;
        gpart = (float*)(ws + P.off_part2);
      }
      // short BF16 unfoldings (m <= 128): the one-tile tcgen05 Gram pass;
      // taller ones: the tiled Gram (tensor cores for BF16, SIMT for FP32)
      if (use_tc && M.m <= 128)
        TTR_CUDA(ttr::tc_gram(Cb, M.m, M.n, gpart, Gp, status, gst));
      else
        TTR_CUDA(ttr::gram_tiled(C, kBf16 ? 1 : 0, M.m, M.n, gpart, Gp, status, gst));
      if (fork) TTR_CUDA(cudaEventRecord(ax->join, ax->s));
      const tt_status rs = sum_ranks(Gp, M.m * M.m);
      if (rs != TT_OK) return rs;
    }
    auto join_gram = [&]() -> tt_status {
      if (fork) TTR_CUDA(cudaStreamWaitEvent(st, ax->join, 0));
      return TT_OK;
    };
    // sketch Y = C Omega, first basis block (the literal form sketches with
    // the first r columns of Omega: the first r rows of its transpose S)
    const int bw = M.literal ? r : M.b;
    if (use_tc)
      TTR_CUDA(ttr::tc_cs(Cb, M.m, M.n, reinterpret_cast<const __nv_bfloat16*>(S), M.n, bw, part, Y, bw, status,
                          st));
    else
      TTR_CUDA(ttr::simt_cs<TIn>(C, M.m, M.n, S, M.n, bw, part, Y, bw, st));
    {
      const tt_status rs = sum_ranks(Y, M.m * bw);
      if (rs != TT_OK) return rs;
    }
    const uint64_t rseed = 0x5EEDull * (uint64_t)(k + 1);
    int* flag = status + 1;
    unsigned* ticket = reinterpret_cast<unsigned*>(status + 2);
    // orthonormalise a block: cluster (or multi-CTA) CholeskyQR path with
    // the one-CTA robust path as fallback, run only if the fast path flagged
    // a breakdown; the one-CTA path alone for shapes neither fast path takes
    // the block just appended, padded and 16-byte aligned, for the power
    float* Xg = (float*)(ws + P.off_Xg);
    const int xld = (M.b + 3) & ~3;
    bool xg_written = false;
    auto orth = [&](const float* Z, int64_t ldz, int zc, int kq0, int c, uint64_t sd) -> tt_status {
      xg_written = false;
      if (ttr::orth_cluster_rs_ok(M.m, kq0, zc, c)) {
        // one cluster launch, rank-deficient columns repaired inside
        const cudaError_t e = ttr::launch_orth_cluster_rs(Z, ldz, zc, M.m, c, kq0, Q, kq, M.gram_power ? Xg : nullptr,
                                                          xld, sd, status, st);
        if (e == cudaSuccess) {
          xg_written = M.gram_power;
          return TT_OK;
        }
        if (e != cudaErrorNotSupported) TTR_CUDA(e);
      }
      if (ttr::orth_grid_rs_ok(M.m, kq0, zc, c)) {
        // blocks taller than a cluster holds: one cooperative launch
        TTR_CUDA(ttr::launch_orth_grid_rs(Z, ldz, zc, M.m, c, kq0, Q, kq, M.gram_power ? Xg : nullptr, xld, sd,
                                          small, status, st));
        xg_written = M.gram_power;
        return TT_OK;
      }
      if (ttr::orth_cluster_ok(M.m, kq0, zc)) {
        TTR_CUDA(ttr::launch_orth_cluster(Z, ldz, M.m, zc, c, Q, kq, kq0, flag, st));
        TTR_CUDA(ttr::launch_orth_block(Z, ldz, M.m, zc, Q, kq, kq0, c, small, sd, status, flag, st));
      } else if (c == zc && ttr::orth_fast_ok(M.m, kq0, zc)) {
        TTR_CUDA(ttr::launch_orth_fast(Z, ldz, M.m, zc, Q, kq, kq0, small, ticket, flag, st));
        TTR_CUDA(ttr::launch_orth_block(Z, ldz, M.m, zc, Q, kq, kq0, c, small, sd, status, flag, st));
      } else {
        TTR_CUDA(ttr::launch_orth_block(Z, ldz, M.m, zc, Q, kq, kq0, c, small, sd, status, nullptr, st));
      }
      return TT_OK;
    };
    // one power: Wj = C C^T Xj (cj columns; row stride kq for both)
    auto power = [&](const float* Xj, float* Wj, int cj) -> tt_status {
      if (M.gram_power) {
        if (!xg_written)   // the block lives only in Q: pack it
          TTR_CUDA(cudaMemcpy2DAsync(Xg, sizeof(float) * xld, Xj, sizeof(float) * kq, sizeof(float) * cj, M.m,
                                     cudaMemcpyDeviceToDevice, st));
        TTR_CUDA(ttr::gram_power(Gp, M.m, Xg, xld, cj, Wj, kq, st));
      } else if (use_tc) {
        if (ttr::tc_ga_ok(M.m, M.n, cj)) {
          TTR_CUDA(ttr::tc_ga(Cb, M.m, M.n, Xj, kq, cj, part, Wj, kq, xs, status, st));
        } else {
          __nv_bfloat16* Tb = reinterpret_cast<__nv_bfloat16*>(T);
          TTR_CUDA(ttr::tc_proj(Cb, M.m, M.n, Xj, kq, cj, 0, Tb, 1, M.n, xs, status, st));
          TTR_CUDA(ttr::tc_cs(Cb, M.m, M.n, Tb, M.n, cj, part, Wj, kq, status, st));
        }
      } else if (M.fused_ga) {
        TTR_CUDA(ttr::simt_ga<TIn>(C, M.m, M.n, Xj, kq, cj, part, Wj, kq, st));
      } else {
        TTR_CUDA((ttr::simt_proj<TIn, float>(C, M.m, M.n, Xj, kq, cj, T, M.n, st, part)));
        TTR_CUDA(ttr::simt_cs<TIn>(C, M.m, M.n, T, M.n, cj, part, Wj, kq, st));
      }
      if (P.world > 1 && !M.gram_power) {
        // the streamed power is a partial sum: add the ranks' blocks (packed
        // into the sketch buffer, free once the first block is orthonormal)
        TTR_CUDA(cudaMemcpy2DAsync(Y, sizeof(float) * cj, Wj, sizeof(float) * kq, sizeof(float) * cj, M.m,
                                   cudaMemcpyDeviceToDevice, st));
        const tt_status rs = sum_ranks(Y, M.m * cj);
        if (rs != TT_OK) return rs;
        TTR_CUDA(cudaMemcpy2DAsync(Wj, sizeof(float) * kq, Y, sizeof(float) * cj, sizeof(float) * cj, M.m,
                                   cudaMemcpyDeviceToDevice, st));
      }
      return TT_OK;
    };
    if (M.literal) {
      // Q = orth((C C^T)^s C W(:, 1:r)): orthonormalise after every power
      // (the same leading-column spans as the literal QRs); Q is the core
      tt_status os = orth(Y, r, r, 0, r, rseed);
      if (os == TT_OK) os = join_gram();
      if (os != TT_OK) return os;
      for (int it = 0; it < M.iters; ++it) {
        os = power(Q, W, r);
        if (os != TT_OK) return os;
        os = orth(W, kq, r, 0, r, rseed + 7919ull * (it + 1));
        if (os != TT_OK) return os;
      }
      TTR_CUDA(cudaMemcpyAsync(U, Q, sizeof(float) * (size_t)M.m * r, cudaMemcpyDeviceToDevice, st));
      TTR_CUDA(cudaMemcpyAsync(core, Q, sizeof(float) * (size_t)M.m * r, cudaMemcpyDeviceToDevice, st));
    } else {
    tt_status os = orth(Y, M.b, M.b, 0, M.blocks[0], rseed);
    if (os == TT_OK) os = join_gram();
    if (os != TT_OK) return os;
    if (P.o.method == TT_METHOD_RSI) {
      // Alg. 4 steps 6-11: Q <- orth(C C^T Q), q times; then one more power
      // gives the Rayleigh-Ritz data W = C C^T Q
      const int c0 = M.blocks[0];
      for (int it = 0; it <= M.iters; ++it) {
        os = power(Q, W, c0);
        if (os != TT_OK) return os;
        if (it < M.iters) {
          os = orth(W, kq, c0, 0, c0, rseed + 7919ull * (it + 1));
          if (os != TT_OK) return os;
        }
      }
    } else {
      int col = 0;
      for (size_t j = 0; j < M.blocks.size(); ++j) {
        const int cj = M.blocks[j];
        // one Krylov power: W_j = C C^T X_j (also the Rayleigh-Ritz data)
        os = power(Q + col, W + col, cj);
        if (os != TT_OK) return os;
        if (j + 1 < M.blocks.size()) {
          os = orth(W + col, kq, cj, col + cj, M.blocks[j + 1], rseed + 7919ull * (j + 1));
          if (os != TT_OK) return os;
        }
        col += cj;
      }
    }
    if (P.o.accurate_rr) {
      // Alg. 3 steps 6-8 without squaring in FP32: B = Q^T C by FP32
      // projections, then rr_svd.cu
      float* Bm = (float*)(ws + P.off_B);
      double* Hd = (double*)(ws + P.off_Hd);
      double* dfp = (double*)(ws + P.off_dfp);
      for (int c0 = 0; c0 < kq; c0 += 64) {   // one pass per 64 basis columns
        const int cw = std::min(64, kq - c0);
        TTR_CUDA((ttr::simt_proj<TIn, float>(C, M.m, M.n, Q + c0, kq, cw, Bm + (size_t)c0 * M.n, M.n, st, nullptr)));
      }
      TTR_CUDA(ttr::gram_df<float>(Bm, kq, M.n, M.n, dfp, Hd, st));
      TTR_CUDA(ttr::launch_rr_svd(Hd, kq, r, Q, M.m, kq, U, core, status, st));
    } else if (ttr::eig_top_ok(kq)) {
      TTR_CUDA(ttr::launch_rr_fast(Q, W, kq, M.m, kq, r, 0, small, U, core, st));
    } else {
      TTR_CUDA(ttr::launch_rayleigh_ritz(Q, W, kq, M.m, kq, r, 0, small, U, core, st));
    }
    }
  }
  // Alg. 3 step 10: next remainder R = U^T C (r x n)
  char* Rout = ws + ((k % 2 == 0) ? P.off_R0 : P.off_R1);
  if (use_tc && r <= 32)
    TTR_CUDA(ttr::tc_proj(Cb, M.m, M.n, U, r, r, 1, Rout, P.remainder == TT_BF16 ? 1 : 0, M.n, xs, status, st));
  else if (P.remainder == TT_BF16)
    TTR_CUDA((ttr::simt_proj<TIn, __nv_bfloat16>(C, M.m, M.n, U, r, r, (__nv_bfloat16*)Rout, M.n, st, part)));
  else
    TTR_CUDA((ttr::simt_proj<TIn, float>(C, M.m, M.n, U, r, r, (float*)Rout, M.n, st, part)));
  return TT_OK;
}

// Argument checks of one problem that need no workspace (Alg. 3 inputs).
tt_status check_problem(const Plan& P, const void* tensor, const float* const* omegas, float* const* cores_out) {
  if (!tensor) return fail(TT_EINVAL, "tensor is NULL");
  if (!cores_out) return fail(TT_EINVAL, "cores_out is NULL");
  for (int k = 0; k < P.d; ++k)
    if (!cores_out[k]) return fail(TT_EINVAL, "cores_out[k] is NULL");
  if (omegas)
    for (int k = 0; k < P.d - 1; ++k)
      if (!omegas[k] && !P.modes[k].gram_route && !P.modes[k].gram_cols)
        return fail(TT_EINVAL, "omegas[k] is NULL");
  return TT_OK;
}

// Enqueues the whole mode loop of Alg. 3 for one problem on `st`.  `ws`
// holds P.total bytes (its own status area unused); `status` points to the
// problem's 256-byte status area, cleared by the caller.
tt_status enqueue_problem(const Plan& P, const void* tensor, const float* const* omegas, uint64_t seed,
                          float* const* cores_out, char* ws, int* status, cudaStream_t st, bool fork_ok = true) {
  tt_status s = TT_OK;
  const int d = P.d;
  for (int k = 0; k < d - 1; ++k) {
    const void* C;
    int dt;
    if (k == 0) {
      C = tensor;
      dt = P.storage;
    } else {
      C = ws + (((k - 1) % 2 == 0) ? P.off_R0 : P.off_R1);
      dt = P.remainder;
    }
    const float* om = omegas ? omegas[k] : nullptr;
    if (dt == TT_BF16)
      s = run_mode<__nv_bfloat16>(P, k, (const __nv_bfloat16*)C, ws, status, om, seed, cores_out[k], st, fork_ok);
    else
      s = run_mode<float>(P, k, (const float*)C, ws, status, om, seed, cores_out[k], st, fork_ok);
    if (s != TT_OK) return s;
  }
  // Alg. 3 step 12: last core = last remainder
  const char* Rlast = ws + (((d - 2) % 2 == 0) ? P.off_R0 : P.off_R1);
  const int64_t wd = (P.world > 1) ? P.slab_w : P.dims[d - 1];   // this rank's slab of the last mode
  const int64_t last = P.rr[d - 1] * wd;
  const float* first[ttr::kFinaliseMaxCores];
  int64_t counts[ttr::kFinaliseMaxCores];
  for (int k = 0; k < d - 1; ++k) {
    first[k] = cores_out[k];
    counts[k] = P.rr[k] * P.dims[k] * P.rr[k + 1];
  }
  TTR_CUDA(ttr::launch_finalise(Rlast, P.remainder, last, cores_out[d - 1], first, counts, d - 1, status, st));
  return TT_OK;
}

tt_status decompose_impl(const void* tensor, const int64_t* dims, int d, const int64_t* ranks, int oversample,
                         int q, const float* const* omegas, uint64_t seed, float* const* cores_out,
                         int64_t* ranks_out, void* workspace, size_t ws_bytes, void* stream,
                         const tt_options* opts) {
  Plan P;
  tt_status s = build_plan(dims, d, ranks, oversample, q, opts, P);
  if (s != TT_OK) return s;
  s = check_problem(P, tensor, omegas, cores_out);
  if (s != TT_OK) return s;
  if (!workspace) return fail(TT_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(TT_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < P.total) return fail(TT_ENOMEM, "workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  int* status = (int*)(ws + P.off_status);
  TTR_CUDA(cudaMemsetAsync(status, 0, 256, st));   // status, breakdown flag, orth ticket
  s = enqueue_problem(P, tensor, omegas, seed, cores_out, ws, status, st);
  if (s != TT_OK) return s;
  if (ranks_out)
    for (int k = 0; k <= d; ++k) ranks_out[k] = P.rr[k];
  return TT_OK;
}

// ---------------------------------------------------------------------------
// Batched form: independent problems spread over concurrent worker streams
// (one fork/join on the caller's stream), so that the small-problem kernels,
// which each occupy a few SMs, run side by side.  Problems are assigned to
// workers by longest-processing-time-first on an estimated cost; problems
// that share a worker run one after another and share its workspace region.

constexpr int kMaxWorkers = 64;
constexpr int kDefaultWorkers = 16;

struct BatchLayout {
  std::vector<Plan> plans;
  std::vector<std::vector<int>> order;   // problem indices per worker, in run order
  std::vector<size_t> worker_off;        // byte offset of each worker's region
  size_t status_bytes = 0, total = 0;
  int workers = 0;
};

// Estimated microseconds of one problem on one worker: bytes streamed at a
// per-worker share of HBM plus a fixed latency per small-algebra launch.
double plan_cost(const Plan& P) {
  double us = 0;
  for (int k = 0; k < P.d - 1; ++k) {
    const ModePlan& M = P.modes[k];
    const double e = (double)esize(k == 0 ? P.storage : P.remainder);
    const bool gram = M.gram_route || M.gram_cols || M.gram_power;
    const double passes = gram ? 2.0 : 2.0 + 2.0 * (double)M.blocks.size();
    us += passes * (double)M.m * (double)M.n * e / 1.0e6;
    us += M.gram_route ? 60.0 : M.gram_cols ? 110.0 : 50.0 * (double)M.blocks.size() + 30.0 + 0.02 * (double)M.kq * M.kq;
  }
  return us + 10.0;
}

tt_status batch_layout(int count, const tt_problem* pr, const tt_options* opts, tt_status* per_problem,
                       BatchLayout& L) {
  if (count < 0) return fail(TT_EINVAL, "count must be >= 0");
  if (count > 0 && !pr) return fail(TT_EINVAL, "problems is NULL");
  tt_options o;
  tt_status s = resolve_options(opts, &o);
  if (s != TT_OK) return s;
  if (o.batch_streams < 0 || o.batch_streams > kMaxWorkers)
    return fail(TT_EINVAL, "options.batch_streams must be in [0, 64]");
  L.plans.assign(count, Plan());
  tt_status first = TT_OK;
  std::string first_msg;
  for (int i = 0; i < count; ++i) {
    s = (pr[i].reserved != 0) ? fail(TT_EINVAL, "problem.reserved must be zero")
                              : build_plan(pr[i].dims, pr[i].d, pr[i].ranks, pr[i].oversample, pr[i].q, &o,
                                           L.plans[i]);
    if (s == TT_OK) s = check_problem(L.plans[i], pr[i].tensor, nullptr, pr[i].cores_out);
    if (per_problem) per_problem[i] = s;
    if (s != TT_OK && first == TT_OK) {
      first = s;
      first_msg = "problem " + std::to_string(i) + ": " + g_last_error;
    }
  }
  if (first != TT_OK) return fail(first, first_msg);
  const int want = o.batch_streams > 0 ? o.batch_streams : kDefaultWorkers;
  L.workers = std::max(1, std::min(want, count));
  std::vector<std::pair<double, int>> cost(count);
  for (int i = 0; i < count; ++i) cost[i] = {plan_cost(L.plans[i]), i};
  std::stable_sort(cost.begin(), cost.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first;
  });
  std::vector<double> load(L.workers, 0.0);
  std::vector<size_t> need(L.workers, 0);
  L.order.assign(L.workers, {});
  for (const auto& c : cost) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += c.first;
    L.order[w].push_back(c.second);
    need[w] = std::max(need[w], L.plans[c.second].total);
  }
  L.status_bytes = align_up((size_t)count * 256);
  size_t off = L.status_bytes;
  L.worker_off.assign(L.workers, 0);
  for (int w = 0; w < L.workers; ++w) {
    L.worker_off[w] = off;
    off += align_up(need[w]);
  }
  L.total = std::max<size_t>(off, 256);
  return TT_OK;
}

struct WorkerPool {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
};
std::mutex g_pool_mu;
std::map<int, WorkerPool> g_pools;

// Worker streams of the current device (created once, kept for the process).
tt_status worker_pool(int workers, WorkerPool** out) {
  int dev = 0;
  TTR_CUDA(cudaGetDevice(&dev));
  WorkerPool& W = g_pools[dev];
  if (!W.fork) TTR_CUDA(cudaEventCreateWithFlags(&W.fork, cudaEventDisableTiming));
  while ((int)W.streams.size() < workers) {
    cudaStream_t s;
    cudaEvent_t e;
    TTR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    TTR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    W.streams.push_back(s);
    W.joins.push_back(e);
  }
  *out = &W;
  return TT_OK;
}

// Enqueues the batch: clear the status areas, fork, run every worker's
// problems, join back onto `st`.  Caller holds g_pool_mu.
tt_status enqueue_batch(const BatchLayout& L, const tt_problem* pr, char* ws, cudaStream_t st) {
  const int count = (int)L.plans.size();
  if (count == 0) return TT_OK;
  WorkerPool* W = nullptr;
  tt_status s = worker_pool(L.workers, &W);
  if (s != TT_OK) return s;
  TTR_CUDA(cudaMemsetAsync(ws, 0, L.status_bytes, st));
  TTR_CUDA(cudaEventRecord(W->fork, st));
  for (int w = 0; w < L.workers; ++w) TTR_CUDA(cudaStreamWaitEvent(W->streams[w], W->fork, 0));
  // issue round-robin over workers so that every worker has work queued early
  size_t most = 0;
  for (const auto& o : L.order) most = std::max(most, o.size());
  tt_status err = TT_OK;
  for (size_t j = 0; j < most && err == TT_OK; ++j)
    for (int w = 0; w < L.workers && err == TT_OK; ++w) {
      if (j >= L.order[w].size()) continue;
      const int i = L.order[w][j];
      int* status = (int*)(ws + (size_t)i * 256);
      // a side stream per problem only when one worker runs them all (it
      // would order the workers' Grams after one another otherwise)
      err = enqueue_problem(L.plans[i], pr[i].tensor, nullptr, pr[i].omega_seed, pr[i].cores_out,
                            ws + L.worker_off[w], status, W->streams[w], L.workers == 1);
    }
  // always join, so that a capture in progress stays well formed
  for (int w = 0; w < L.workers; ++w) {
    TTR_CUDA(cudaEventRecord(W->joins[w], W->streams[w]));
    TTR_CUDA(cudaStreamWaitEvent(st, W->joins[w], 0));
  }
  return err;
}

tt_status check_batch_ws(const BatchLayout& L, void* workspace, size_t ws_bytes) {
  if (!workspace) return fail(TT_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(TT_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < L.total) return fail(TT_ENOMEM, "workspace too small");
  return TT_OK;
}

void fill_ranks_out(const BatchLayout& L, const tt_problem* pr) {
  for (size_t i = 0; i < L.plans.size(); ++i)
    if (pr[i].ranks_out)
      for (int k = 0; k <= L.plans[i].d; ++k) pr[i].ranks_out[k] = L.plans[i].rr[k];
}

}  // namespace

namespace ttr {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace ttr

extern "C" {

tt_status tt_rbki_default_options(tt_options* o) {
  if (!o) return fail(TT_EINVAL, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->storage = TT_F32;
  o->remainder = -1;
  o->exhaust_gram = 1;
  o->gram_power = 1;
  return TT_OK;
}

tt_status tt_rbki_core_sizes(const int64_t* dims, int d, const int64_t* ranks, int64_t* ranks_out,
                             int64_t* core_elems) {
  std::vector<int64_t> rr;
  tt_status s = clamp(dims, d, ranks, rr);
  if (s != TT_OK) return s;
  if (!ranks_out) return fail(TT_EINVAL, "ranks_out is NULL");
  for (int k = 0; k <= d; ++k) ranks_out[k] = rr[k];
  if (core_elems)
    for (int k = 0; k < d; ++k) core_elems[k] = rr[k] * dims[k] * rr[k + 1];
  return TT_OK;
}

tt_status tt_rbki_workspace_size(const int64_t* dims, int d, const int64_t* ranks, int oversample, int q,
                                 const tt_options* opts, size_t* bytes) {
  if (!bytes) return fail(TT_EINVAL, "bytes is NULL");
  Plan P;
  tt_status s = build_plan(dims, d, ranks, oversample, q, opts, P);
  if (s != TT_OK) return s;
  *bytes = P.total;
  return TT_OK;
}

tt_status tt_rbki_plan_modes(const int64_t* dims, int d, const int64_t* ranks, int oversample, int q,
                             const tt_options* opts, tt_mode_plan* modes, int max_modes) {
  if (!modes) return fail(TT_EINVAL, "modes is NULL");
  Plan P;
  tt_status s = build_plan(dims, d, ranks, oversample, q, opts, P);
  if (s != TT_OK) return s;
  if (max_modes < d - 1) return fail(TT_EINVAL, "max_modes must be >= d - 1");
  for (int k = 0; k < d - 1; ++k) {
    const ModePlan& M = P.modes[k];
    tt_mode_plan& o = modes[k];
    std::memset(&o, 0, sizeof(o));
    o.m = M.m;
    o.n = M.n;
    o.r_in = M.r_in;
    o.r_out = M.r_out;
    o.b = M.b;
    o.basis_cols = M.kq;
    o.blocks = (int32_t)M.blocks.size();
    const bool exhaustion = M.gram_route || M.gram_cols;
    o.powers = exhaustion ? 0
             : M.literal ? M.iters
             : (P.o.method == TT_METHOD_RSI ? M.iters + 1 : (int32_t)M.blocks.size());
    o.route = M.gram_route ? TT_ROUTE_GRAM_ROWS
            : M.gram_cols  ? TT_ROUTE_GRAM_COLS
            : M.gram_power ? TT_ROUTE_GRAM_POWER
                           : TT_ROUTE_KRYLOV;
    const int cdt = (k == 0) ? P.storage : P.remainder;
    const bool tc = cdt == TT_BF16 && ttr::tc_shape_ok(M.m, M.n);
    o.tensor_cores = tc ? 1 : 0;
    if (!exhaustion && !M.gram_power) o.fused_power = (tc ? ttr::tc_ga_ok(M.m, M.n, M.b) : M.fused_ga) ? 1 : 0;
  }
  return TT_OK;
}

tt_status tt_rbki_decompose(const void* tensor, const int64_t* dims, int d, const int64_t* ranks, int oversample,
                            int q, uint64_t omega_seed, float* const* cores_out, int64_t* ranks_out,
                            void* workspace, size_t ws_bytes, void* stream, const tt_options* opts) {
  return decompose_impl(tensor, dims, d, ranks, oversample, q, nullptr, omega_seed, cores_out, ranks_out,
                        workspace, ws_bytes, stream, opts);
}

tt_status tt_rbki_decompose_omega(const void* tensor, const int64_t* dims, int d, const int64_t* ranks,
                                  int oversample, int q, const float* const* omegas, float* const* cores_out,
                                  int64_t* ranks_out, void* workspace, size_t ws_bytes, void* stream,
                                  const tt_options* opts) {
  if (!omegas) return fail(TT_EINVAL, "omegas is NULL");
  return decompose_impl(tensor, dims, d, ranks, oversample, q, omegas, 0, cores_out, ranks_out, workspace,
                        ws_bytes, stream, opts);
}

tt_status tt_rbki_device_status(const void* workspace, void* stream, int* device_status) {
  if (!workspace || !device_status) return fail(TT_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  TTR_CUDA(cudaMemcpyAsync(&h, workspace, sizeof(int), cudaMemcpyDeviceToHost, st));
  TTR_CUDA(cudaStreamSynchronize(st));
  *device_status = h;
  return TT_OK;
}

const char* tt_rbki_last_error(void) { return g_last_error.c_str(); }

tt_status tt_permute_convert(const void* src, int src_dtype, const int64_t* dims, const int64_t* src_strides,
                             const int* perm, int d, void* dst, int dst_dtype, void* stream) {
  if (!src || !dst || !dims || !src_strides) return fail(TT_EINVAL, "NULL argument");
  if (d < 1 || d > 8) return fail(TT_EINVAL, "d must be in [1, 8]");
  if ((src_dtype != TT_F32 && src_dtype != TT_BF16) || (dst_dtype != TT_F32 && dst_dtype != TT_BF16))
    return fail(TT_EINVAL, "dtype must be TT_F32 or TT_BF16");
  bool seen[8] = {false};
  for (int j = 0; j < d; ++j) {
    if (dims[j] < 0 || src_strides[j] < 0) return fail(TT_EINVAL, "negative size or stride");
    const int s = perm ? perm[j] : j;
    if (s < 0 || s >= d || seen[s]) return fail(TT_EINVAL, "perm is not a permutation");
    seen[s] = true;
  }
  TTR_CUDA(ttr::launch_permute(src, src_dtype, dst, dst_dtype, dims, src_strides, perm, d, (cudaStream_t)stream));
  return TT_OK;
}

tt_status tt_omega_generate(uint64_t seed, int mode, int64_t n, int b, void* out, int out_dtype, int64_t ld,
                            void* stream) {
  if (!out) return fail(TT_EINVAL, "out is NULL");
  if (n < 0 || b < 0 || ld < b || mode < 0) return fail(TT_EINVAL, "bad shape");
  if (out_dtype != TT_F32 && out_dtype != TT_BF16) return fail(TT_EINVAL, "bad dtype");
  if (n == 0 || b == 0) return TT_OK;
  TTR_CUDA(ttr::launch_omega(seed, mode, n, b, out, out_dtype, ld, 1, (cudaStream_t)stream));
  return TT_OK;
}

struct PassLayout {
  size_t part = 0, sbuf = 0, xt = 0, status = 0, total = 0;
  bool tc = false, fused = false;
};

static tt_status pass_layout(int op, int64_t m, int64_t n, int b, int c_dtype, PassLayout* L) {
  if (m < 1 || n < 1) return fail(TT_EINVAL, "bad shape");
  if (c_dtype != TT_F32 && c_dtype != TT_BF16) return fail(TT_EINVAL, "bad dtype");
  if (op != TT_PASS_GRAM && (b < 1 || b > 64)) return fail(TT_EUNSUPPORTED, "b must be in [1, 64]");
  size_t part = 0, sbuf = 0, xt = 0;
  const bool tc = c_dtype == TT_BF16 && ttr::tc_shape_ok(m, n);
  L->tc = tc;
  switch (op) {
    case TT_PASS_SKETCH:
      part = tc ? ttr::tc_cs_partials(m, n, b) : ttr::simt_cs_partials(m, n, b);
      sbuf = (size_t)b * n;
      break;
    case TT_PASS_GRAMAPPLY:
      if (tc) {
        L->fused = ttr::tc_ga_ok(m, n, b);
        part = L->fused ? ttr::tc_ga_partials(m, n, b) : ttr::tc_cs_partials(m, n, b);
        if (!L->fused) sbuf = (size_t)b * n;
        xt = std::max(ttr::tc_ga_scratch_bytes(m, b), ttr::tc_proj_scratch_bytes(m, b, 0));
      } else {
        L->fused = ttr::simt_ga_fused_ok(m, b);
        part = L->fused ? ttr::simt_ga_partials(m, n, b) : ttr::simt_cs_partials(m, n, b);
        if (!L->fused) sbuf = (size_t)b * n;
      }
      break;
    case TT_PASS_PROJECT:
      if (tc) xt = ttr::tc_proj_scratch_bytes(m, b, b <= 32 ? 1 : 0);
      break;
    case TT_PASS_GRAM:
      if (m > 2048) return fail(TT_EUNSUPPORTED, "Gram pass needs m <= 2048");
      if (m > 128) part = ttr::gram_tiled_partials(m, n, c_dtype == TT_BF16 ? 1 : 0);
      else part = tc ? ttr::tc_gram_partials(m, n) : ttr::simt_gram_partials(m, n);
      break;
    default:
      return fail(TT_EINVAL, "unknown op");
  }
  L->part = 0;
  L->sbuf = align_up(part * 4);
  L->xt = L->sbuf + align_up(sbuf * 4);
  L->status = L->xt + align_up(xt);
  L->total = L->status + 256;
  return TT_OK;
}

tt_status tt_pass_workspace_size(int op, int64_t m, int64_t n, int b, int c_dtype, size_t* bytes) {
  if (!bytes) return fail(TT_EINVAL, "bytes is NULL");
  PassLayout L;
  tt_status s = pass_layout(op, m, n, b, c_dtype, &L);
  if (s != TT_OK) return s;
  *bytes = L.total;
  return TT_OK;
}

tt_status tt_pass(int op, const void* C, int c_dtype, int64_t m, int64_t n, int b, const float* x, void* y,
                  int y_dtype, void* workspace, size_t ws_bytes, void* stream) {
  PassLayout L;
  tt_status s = pass_layout(op, m, n, b, c_dtype, &L);
  if (s != TT_OK) return s;
  if (!C || !y || (op != TT_PASS_GRAM && !x)) return fail(TT_EINVAL, "NULL argument");
  if (!workspace || ws_bytes < L.total) return fail(TT_ENOMEM, "workspace too small");
  if (((uintptr_t)workspace & 255) != 0) return fail(TT_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  float* part = (float*)(ws + L.part);
  float* sbuf = (float*)(ws + L.sbuf);
  void* xt = ws + L.xt;
  int* status = (int*)(ws + L.status);
  TTR_CUDA(cudaMemsetAsync(status, 0, 256, st));
  const bool bf = c_dtype == TT_BF16;
  const __nv_bfloat16* Cb = (const __nv_bfloat16*)C;
  __nv_bfloat16* Sb = (__nv_bfloat16*)sbuf;
  switch (op) {
    case TT_PASS_SKETCH:
      if (L.tc) {
        TTR_CUDA(ttr::launch_omega_transpose_any(x, n, b, Sb, TT_BF16, st));
        TTR_CUDA(ttr::tc_cs(Cb, m, n, Sb, n, b, part, (float*)y, b, status, st));
      } else {
        TTR_CUDA(ttr::launch_omega_transpose_any(x, n, b, sbuf, TT_F32, st));
        if (bf) TTR_CUDA(ttr::simt_cs<__nv_bfloat16>(Cb, m, n, sbuf, n, b, part, (float*)y, b, st));
        else TTR_CUDA(ttr::simt_cs<float>((const float*)C, m, n, sbuf, n, b, part, (float*)y, b, st));
      }
      break;
    case TT_PASS_GRAMAPPLY:
      if (L.tc) {
        if (L.fused) {
          TTR_CUDA(ttr::tc_ga(Cb, m, n, x, b, b, part, (float*)y, b, xt, status, st));
        } else {
          TTR_CUDA(ttr::tc_proj(Cb, m, n, x, b, b, 0, Sb, 1, n, xt, status, st));
          TTR_CUDA(ttr::tc_cs(Cb, m, n, Sb, n, b, part, (float*)y, b, status, st));
        }
      } else if (L.fused) {
        if (bf) TTR_CUDA(ttr::simt_ga<__nv_bfloat16>(Cb, m, n, x, b, b, part, (float*)y, b, st));
        else TTR_CUDA(ttr::simt_ga<float>((const float*)C, m, n, x, b, b, part, (float*)y, b, st));
      } else {
        if (bf) {
          TTR_CUDA((ttr::simt_proj<__nv_bfloat16, float>(Cb, m, n, x, b, b, sbuf, n, st)));
          TTR_CUDA(ttr::simt_cs<__nv_bfloat16>(Cb, m, n, sbuf, n, b, part, (float*)y, b, st));
        } else {
          TTR_CUDA((ttr::simt_proj<float, float>((const float*)C, m, n, x, b, b, sbuf, n, st)));
          TTR_CUDA(ttr::simt_cs<float>((const float*)C, m, n, sbuf, n, b, part, (float*)y, b, st));
        }
      }
      break;
    case TT_PASS_PROJECT:
      if (L.tc) {
        TTR_CUDA(ttr::tc_proj(Cb, m, n, x, b, b, b <= 32 ? 1 : 0, y, y_dtype == TT_BF16 ? 1 : 0, n, xt, status, st));
      } else if (y_dtype == TT_BF16) {
        if (bf) TTR_CUDA((ttr::simt_proj<__nv_bfloat16, __nv_bfloat16>(Cb, m, n, x, b, b, (__nv_bfloat16*)y, n, st)));
        else TTR_CUDA((ttr::simt_proj<float, __nv_bfloat16>((const float*)C, m, n, x, b, b, (__nv_bfloat16*)y, n, st)));
      } else {
        if (bf) TTR_CUDA((ttr::simt_proj<__nv_bfloat16, float>(Cb, m, n, x, b, b, (float*)y, n, st)));
        else TTR_CUDA((ttr::simt_proj<float, float>((const float*)C, m, n, x, b, b, (float*)y, n, st)));
      }
      break;
    case TT_PASS_GRAM:
      if (m > 128) TTR_CUDA(ttr::gram_tiled(C, bf ? 1 : 0, m, n, part, (float*)y, status, st));
      else if (L.tc) TTR_CUDA(ttr::tc_gram(Cb, m, n, part, (float*)y, status, st));
      else if (bf) TTR_CUDA(ttr::simt_gram<__nv_bfloat16>(Cb, m, n, part, (float*)y, st));
      else TTR_CUDA(ttr::simt_gram<float>((const float*)C, m, n, part, (float*)y, st));
      break;
  }
  return TT_OK;
}

tt_status tt_gram_power(const float* G, int64_t m, const float* X, int64_t ldx, int c, float* W, int64_t ldw,
                        void* stream) {
  if (!G || !X || !W) return fail(TT_EINVAL, "NULL argument");
  if (m < 1 || c < 1 || ldx < ((c + 3) & ~3) || ldw < c) return fail(TT_EINVAL, "bad shape");
  if (ldx % 4 != 0 || ((uintptr_t)X & 15) != 0) return fail(TT_EINVAL, "X must be 16-byte aligned with ldx % 4 == 0");
  if (!ttr::gram_power_ok(m, c)) return fail(TT_EUNSUPPORTED, "c must be <= 64");
  TTR_CUDA(ttr::gram_power(G, m, X, ldx, c, W, ldw, (cudaStream_t)stream));
  return TT_OK;
}

tt_status tt_rbki_batched_workspace_size(int count, const tt_problem* problems, const tt_options* opts,
                                         size_t* bytes) {
  if (!bytes) return fail(TT_EINVAL, "bytes is NULL");
  BatchLayout L;
  tt_status s = batch_layout(count, problems, opts, nullptr, L);
  if (s != TT_OK) return s;
  *bytes = L.total;
  return TT_OK;
}

tt_status tt_rbki_decompose_batched(int count, const tt_problem* problems, void* workspace, size_t ws_bytes,
                                    void* stream, const tt_options* opts, tt_status* per_problem) {
  BatchLayout L;
  tt_status s = batch_layout(count, problems, opts, per_problem, L);
  if (s != TT_OK) return s;
  s = check_batch_ws(L, workspace, ws_bytes);
  if (s != TT_OK) return s;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    s = enqueue_batch(L, problems, (char*)workspace, (cudaStream_t)stream);
  }
  if (s != TT_OK) return s;
  fill_ranks_out(L, problems);
  return TT_OK;
}

tt_status tt_rbki_batched_device_status(const void* workspace, int count, void* stream, int* device_status) {
  if (!workspace || (count > 0 && !device_status)) return fail(TT_EINVAL, "NULL argument");
  if (count <= 0) return TT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  TTR_CUDA(cudaMemcpy2DAsync(device_status, sizeof(int), workspace, 256, sizeof(int), (size_t)count,
                             cudaMemcpyDeviceToHost, st));
  TTR_CUDA(cudaStreamSynchronize(st));
  return TT_OK;
}

struct tt_graph_t {
  cudaGraphExec_t exec = nullptr;
};

tt_status tt_rbki_batched_graph_create(int count, const tt_problem* problems, void* workspace, size_t ws_bytes,
                                       const tt_options* opts, tt_status* per_problem, tt_graph* graph) {
  if (!graph) return fail(TT_EINVAL, "graph is NULL");
  *graph = nullptr;
  BatchLayout L;
  tt_status s = batch_layout(count, problems, opts, per_problem, L);
  if (s != TT_OK) return s;
  s = check_batch_ws(L, workspace, ws_bytes);
  if (s != TT_OK) return s;
  cudaStream_t cs;
  TTR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cs);
      return fail(TT_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    }
    s = enqueue_batch(L, problems, (char*)workspace, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (s == TT_OK && e != cudaSuccess) s = fail(TT_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  }
  cudaStreamDestroy(cs);
  if (s != TT_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  tt_graph out = new tt_graph_t;
  cudaError_t e = cudaGraphInstantiate(&out->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    delete out;
    return fail(TT_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  fill_ranks_out(L, problems);
  *graph = out;
  return TT_OK;
}

tt_status tt_rbki_graph_launch(tt_graph graph, void* stream) {
  if (!graph || !graph->exec) return fail(TT_EINVAL, "graph is NULL");
  TTR_CUDA(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
  return TT_OK;
}

tt_status tt_rbki_graph_destroy(tt_graph graph) {
  if (!graph) return TT_OK;
  cudaError_t e = graph->exec ? cudaGraphExecDestroy(graph->exec) : cudaSuccess;
  delete graph;
  if (e != cudaSuccess) return fail(TT_ECUDA, std::string("cudaGraphExecDestroy: ") + cudaGetErrorString(e));
  return TT_OK;
}

tt_status tt_sym_eig_workspace_size(int k, int r, size_t* bytes) {
  if (!bytes) return fail(TT_EINVAL, "bytes is NULL");
  if (k < 1 || r < 1 || r > k) return fail(TT_EINVAL, "need 1 <= r <= k");
  if (!ttr::eig_top_ok(k)) return fail(TT_EUNSUPPORTED, "k must be <= 224");
  *bytes = align_up(ttr::eig_scratch_floats(k, r) * 4);
  return TT_OK;
}

tt_status tt_sym_eig_top(const float* H, int64_t ldh, int k, int r, float* V, float* evals, void* workspace,
                         size_t ws_bytes, void* stream) {
  size_t need = 0;
  tt_status s = tt_sym_eig_workspace_size(k, r, &need);
  if (s != TT_OK) return s;
  if (!H || !V) return fail(TT_EINVAL, "NULL argument");
  if (ldh < k) return fail(TT_EINVAL, "ldh < k");
  if (!workspace || ws_bytes < need) return fail(TT_ENOMEM, "workspace too small");
  TTR_CUDA(ttr::launch_eig_top(H, ldh, k, r, V, (float*)workspace, evals, (cudaStream_t)stream));
  return TT_OK;
}

// Sharded form: this rank's slab of the last mode; the sums over ranks go
// through the caller's callback (see include/tt_rbki.h).
tt_status tt_rbki_shard_plan(const int64_t* dims, int d, const int64_t* ranks, int oversample, int q,
                             const tt_options* opts, int32_t world, int32_t rank, int64_t* slab_lo, int64_t* slab_w,
                             tt_shard_mode* modes, int max_modes) {
  if (!slab_lo || !slab_w || !modes) return fail(TT_EINVAL, "slab_lo, slab_w and modes must not be NULL");
  Plan P;
  tt_status s = build_plan(dims, d, ranks, oversample, q, opts, P, world, rank);
  if (s != TT_OK) return s;
  if (max_modes < d - 1) return fail(TT_EINVAL, "max_modes must be >= d - 1");
  *slab_lo = P.slab_lo;
  *slab_w = P.slab_w;
  for (int k = 0; k < d - 1; ++k) {
    const ModePlan& M = P.modes[k];
    tt_shard_mode& o = modes[k];
    std::memset(&o, 0, sizeof(o));
    o.m = M.m;
    o.n_global = M.n_global;
    o.n_local = M.n;
    o.route = M.gram_route ? TT_ROUTE_GRAM_ROWS : M.gram_power ? TT_ROUTE_GRAM_POWER : TT_ROUTE_KRYLOV;
    o.allreduces = M.allreduces;
    o.allreduce_floats = M.allreduce_floats;
  }
  return TT_OK;
}

tt_status tt_rbki_sharded_workspace_size(const int64_t* dims, int d, const int64_t* ranks, int oversample, int q,
                                         const tt_options* opts, int32_t world, int32_t rank, size_t* bytes) {
  if (!bytes) return fail(TT_EINVAL, "bytes is NULL");
  Plan P;
  tt_status s = build_plan(dims, d, ranks, oversample, q, opts, P, world, rank);
  if (s != TT_OK) return s;
  *bytes = P.total;
  return TT_OK;
}

tt_status tt_rbki_decompose_sharded(const void* local_tensor, const int64_t* dims, int d, const int64_t* ranks,
                                    int oversample, int q, uint64_t omega_seed, float* const* cores_out,
                                    int64_t* ranks_out, void* workspace, size_t ws_bytes, int32_t world, int32_t rank,
                                    tt_allreduce_fn allreduce, void* ctx, void* stream, const tt_options* opts) {
  Plan P;
  tt_status s = build_plan(dims, d, ranks, oversample, q, opts, P, world, rank);
  if (s != TT_OK) return s;
  if (world > 1 && !allreduce) return fail(TT_EINVAL, "allreduce is NULL");
  P.allreduce = allreduce;
  P.comm = ctx;
  s = check_problem(P, local_tensor, nullptr, cores_out);
  if (s != TT_OK) return s;
  if (!workspace) return fail(TT_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(TT_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < P.total) return fail(TT_ENOMEM, "workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  int* status = (int*)(ws + P.off_status);
  TTR_CUDA(cudaMemsetAsync(status, 0, 256, st));
  s = enqueue_problem(P, local_tensor, nullptr, omega_seed, cores_out, ws, status, st);
  if (s != TT_OK) return s;
  if (ranks_out)
    for (int k = 0; k <= d; ++k) ranks_out[k] = P.rr[k];
  return TT_OK;
}

}  // extern "C"
