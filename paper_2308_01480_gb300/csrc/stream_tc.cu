// Tensor-core (tcgen05 + TMA) streaming passes over a BF16 unfolding C
// (m x n, row-major), FP32 accumulation in Tensor Memory:
//   gram : G = C C^T                 (m <= 128; exhaustion route)
//   cs   : Y = C S^T, S is b x n      (sketch C W with S = W^T; second half
//                                       of a Krylov power for tall C)
//   proj : S = X^T C (b x n)          (projection U^T C of Alg. 3 step 10,
//                                       with U split in BF16 hi + lo parts;
//                                       first half of a power for tall C)
//   ga   : Y = C (C^T X)              (one Krylov power, each column tile
//                                       read from HBM once; for m > 256 the
//                                       tile's 128-row chunks stream twice,
//                                       the second time from L2)
// Column tiles of C arrive by TMA (128-byte swizzle) into a ring of shared
// memory stages.  Warp 0 issues TMA, warp 1 issues tcgen05.mma from one
// thread and owns the TMEM allocation, warps 2-5 read TMEM (each warp the
// 32 lanes of its quarter) for the epilogue.  Every wait is bounded: on a
// timeout the kernel records TT_ETIMEOUT in the status word, lets its own
// copies and MMAs drain, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace ttr {

using namespace tc;

constexpr int TC_THREADS = 192;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int SMEM_HALF = 113 * 1024;   // two CTAs per SM

enum : int { OPK_GRAM = 0, OPK_CS = 1, OPK_PROJ = 2, OPK_GA = 3 };

struct TcParams {
  int64_t m, n;
  int b;            // logical output columns (proj: rows of S written)
  int npad;         // MMA N (multiple of 16)
  int mb;           // M blocks of 128 rows handled by a CTA (cs, ga)
  int kb;           // 64-column boxes per tile (1 or 2)
  int stages;
  int64_t tiles;    // column tiles of width 64*kb
  int64_t row_groups;
  int nchunks;      // proj, ga: row chunks of C per tile (ga: > 1 for tall C)
  int split_hi_lo;  // proj: out = D[:, c] + D[:, c + lo_off]
  int lo_off;
  int out_bf16;     // proj: output dtype
  int64_t ld_out;   // proj: row stride of S
  void* out;        // proj: S (b x n); others: partials
  int* status;
  int stage_bytes;
  int c_box_bytes;  // bytes of one C box (64 cols x box rows)
  int c_box_rows;
  int x_box_bytes;  // proj/ga: one X^T box (64 of m x npad)
  int s_box_bytes;  // cs: one S box (64 cols x npad)
  int x_res_bytes;  // ga: resident X^T bytes
  int t_bytes;      // ga: one T buffer
  int mpad;         // ga: padded m (multiple of 64)
  int chunk_rows;   // proj: rows of C per chunk (multiple of 16)
  int x_resident;   // proj: X^T loaded once (single chunk)
  int slack_bytes;  // shared memory after the ring covering MMA reads past short boxes
  int o_bytes;      // proj: output staging buffer of one epilogue warp (b rows x 32
                    // columns); 0 = one scalar store per output element
};

struct TcShared {
  uint64_t full[8];
  uint64_t empty[8];
  uint64_t dfull[2];
  uint64_t dempty[2];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t zfull;
  uint64_t drain;
  uint64_t xfull;
  uint32_t tmem_base;
  int abort_flag;
};

__device__ __forceinline__ void tc_abort(TcShared* sh, int* status) {
  sh->abort_flag = 1;
  set_status(status, TT_ETIMEOUT);
}

// ---------------------------------------------------------------- kernel
template <int OP>
__global__ void __launch_bounds__(TC_THREADS, 2)
k_tc_stream(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ CUtensorMap mapB, TcParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ring = smem;
  uint8_t* xres = ring + (size_t)p.stages * p.stage_bytes + p.slack_bytes;   // resident X^T
  uint8_t* tbuf = xres + p.x_res_bytes;                         // ga: T buffers
  uint8_t* obuf = tbuf + 2 * p.t_bytes;                         // proj: output staging
  TcShared* sh = reinterpret_cast<TcShared*>(obuf + 4 * p.o_bytes);
  volatile int* abortp = &sh->abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  const int row_group = (OP == OPK_CS) ? (int)(blockIdx.x % p.row_groups) : 0;
  const int cta_in_group = (OP == OPK_CS) ? (int)(blockIdx.x / p.row_groups) : (int)blockIdx.x;
  const int ctas_in_group = (OP == OPK_CS) ? (int)(gridDim.x / p.row_groups) : (int)gridDim.x;
  const int64_t row0 = (int64_t)row_group * p.mb * 128;
  // tiles handled by this CTA: cta_in_group, + ctas_in_group, ...
  const int64_t my_tiles =
      (p.tiles > cta_in_group) ? (p.tiles - cta_in_group + ctas_in_group - 1) / ctas_in_group : 0;
  // gram: two accumulation buffers of npad columns (see the MMA issuer)
  const int acc_cols = (OP == OPK_GRAM) ? 2 * p.npad : p.mb * p.npad;
  const uint32_t tmem_cols = (OP == OPK_PROJ) ? 128u
                            : (OP == OPK_GA ? (128 + p.mb * p.npad <= 256 ? 256u : 512u)
                                            : (acc_cols <= 32 ? 32u : acc_cols <= 64 ? 64u
                                               : acc_cols <= 128 ? 128u : 256u));
  // gram: column tiles per TMEM accumulation chunk (16 or 32 MMAs)
  const int gram_ck = (p.kb >= 8) ? 1 : 2;
  const int64_t gram_chunks = (my_tiles + gram_ck - 1) / gram_ck;
  const bool ga_tall = (OP == OPK_GA) && p.nchunks > 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&sh->full[s], 1); mbar_init(&sh->empty[s], 1); }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh->dfull[i], 1); mbar_init(&sh->dempty[i], 4);
      mbar_init(&sh->tfull[i], 4); mbar_init(&sh->tempty[i], 1);
    }
    mbar_init(&sh->zfull, 1);
    mbar_init(&sh->drain, 1);
    mbar_init(&sh->xfull, 1);
    sh->abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&mapC);
    prefetch_tmap(&mapB);
  }
  if (warp == 1) {
    tmem_alloc(&sh->tmem_base, tmem_cols);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;

  // =========================================================== producer
  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      if (OP == OPK_GA || (OP == OPK_PROJ && p.x_resident)) {
        // resident X^T: mpad/64 boxes of (64 x npad)
        const int nbox = p.mpad / 64;
        mbar_arrive_expect_tx(&sh->xfull, (uint32_t)(nbox * p.x_box_bytes));
        for (int i = 0; i < nbox; ++i) tma_load_2d(xres + (size_t)i * p.x_box_bytes, &mapB, &sh->xfull, i * 64, 0);
      }
      int64_t fill = 0;
      // tall Gram-apply: the chunks of tile t for C^T X, then those of tile
      // t - 1 again for C T (by then its T is in shared memory)
      auto load_tile = [&](int64_t it) {
        const int64_t tile = cta_in_group + it * ctas_in_group;
        for (int r = 0; r < p.nchunks && ok; ++r, ++fill) {
          const int s = (int)(fill % S);
          if (!mbar_wait(&sh->empty[s], (uint32_t)(((fill / S) & 1) ^ 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
          uint8_t* st = ring + (size_t)s * p.stage_bytes;
          mbar_arrive_expect_tx(&sh->full[s], (uint32_t)(2 * p.c_box_bytes));
          for (int kb = 0; kb < 2; ++kb)
            tma_load_2d(st + (size_t)kb * p.c_box_bytes, &mapC, &sh->full[s], (int)(tile * 128 + 64 * kb), r * 128);
        }
      };
      if (ga_tall) {
        for (int64_t it = 0; it < my_tiles && ok; ++it) {
          load_tile(it);
          if (it > 0) load_tile(it - 1);
        }
        if (my_tiles > 0) load_tile(my_tiles - 1);
      }
      const int per_tile = (OP == OPK_PROJ) ? p.nchunks : 1;
      for (int64_t it = 0; it < my_tiles && ok && !ga_tall; ++it) {
        const int64_t tile = cta_in_group + it * ctas_in_group;
        for (int ch = 0; ch < per_tile && ok; ++ch, ++fill) {
          const int s = (int)(fill % S);
          const uint32_t round = (uint32_t)(fill / S);
          if (!mbar_wait(&sh->empty[s], (round & 1) ^ 1, abortp)) { tc_abort(sh, p.status); ok = false; break; }
          uint8_t* st = ring + (size_t)s * p.stage_bytes;
          const int x0 = (int)(tile * 64 * p.kb);
          if (OP == OPK_GRAM || OP == OPK_GA) {
            mbar_arrive_expect_tx(&sh->full[s], (uint32_t)(p.kb * p.c_box_bytes));
            for (int kb = 0; kb < p.kb; ++kb) tma_load_2d(st + (size_t)kb * p.c_box_bytes, &mapC, &sh->full[s], x0 + 64 * kb, 0);
          } else if (OP == OPK_CS) {
            mbar_arrive_expect_tx(&sh->full[s], (uint32_t)(p.mb * p.c_box_bytes + p.s_box_bytes));
            for (int b = 0; b < p.mb; ++b)
              tma_load_2d(st + (size_t)b * p.c_box_bytes, &mapC, &sh->full[s], x0, (int)(row0 + 128 * b));
            tma_load_2d(st + (size_t)p.mb * p.c_box_bytes, &mapB, &sh->full[s], x0, 0);
          } else {  // PROJ: C chunk (2 boxes of 64 cols x chunk_rows) [+ X^T chunk (2 boxes 64 x npad)]
            const int xb = p.x_resident ? 0 : 2;
            mbar_arrive_expect_tx(&sh->full[s], (uint32_t)(2 * p.c_box_bytes + xb * p.x_box_bytes));
            for (int kb = 0; kb < 2; ++kb)
              tma_load_2d(st + (size_t)kb * p.c_box_bytes, &mapC, &sh->full[s], x0 + 64 * kb, ch * p.chunk_rows);
            for (int kb = 0; kb < xb; ++kb)
              tma_load_2d(st + 2 * (size_t)p.c_box_bytes + (size_t)kb * p.x_box_bytes, &mapB, &sh->full[s],
                          ch * p.chunk_rows + 64 * kb, 0);
          }
        }
      }
      // drain: every issued copy must land before the CTA can exit (the
      // last fill of stage s is the largest f < fill with f = s mod S)
      for (int s = 0; s < S; ++s)
        if (s < fill) {
          const int64_t last = s + (int64_t)S * ((fill - 1 - s) / S);
          int zero = 0;
          mbar_wait(&sh->full[s], (uint32_t)((last / S) & 1), &zero);
        }
      if (OP == OPK_GA || (OP == OPK_PROJ && p.x_resident)) { int zero = 0; mbar_wait(&sh->xfull, 0, &zero); }
    }
  }
  // =========================================================== MMA issuer
  else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int64_t fill = 0;
      // descriptors relative to the ring base (offsets of xres and tbuf too):
      // K-major 128-byte-swizzled operands, the MN-major C tile (its two
      // 64-column atoms one box apart), and T (8 x 8 core matrices)
      const uint32_t ring_s = smem_u32(ring);
      const DescGen gK(ring_s, 16, 1024, SW_128B);
      const DescGen gM(ring_s, (uint32_t)p.c_box_bytes, 1024, SW_128B);
      const DescGen gT(ring_s, 128, 2048, SW_NONE);
      const uint32_t xres_off = (uint32_t)(xres - ring), tbuf_off = (uint32_t)(tbuf - ring);
      if (OP == OPK_GRAM) {
        // The tensor cores' FP32 accumulation does not round to nearest, so
        // its error grows with the MMAs added into one accumulator: the
        // tiles go in chunks of gram_ck into two alternating TMEM buffers
        // (dfull / dempty), and the epilogue adds each chunk into FP32
        // registers with round-to-nearest while the next chunk accumulates.
        const uint32_t idesc = idesc_bf16(128, p.npad, 0, 0);
        for (int64_t c = 0; c < gram_chunks && ok; ++c) {
          const int buf = (int)(c & 1);
          if (!mbar_wait(&sh->dempty[buf], (uint32_t)(((c >> 1) & 1) ^ 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * p.npad);
          const int64_t ite = imin(my_tiles, (c + 1) * gram_ck);
          for (int64_t it = c * gram_ck; it < ite; ++it, ++fill) {
            const int s = (int)(fill % S);
            if (!mbar_wait(&sh->full[s], (uint32_t)((fill / S) & 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
            tc_fence_after();
            const uint32_t soff = (uint32_t)s * (uint32_t)p.stage_bytes;
            const bool first = it == c * gram_ck;
            for (int kb = 0; kb < p.kb; ++kb) {
              const uint32_t boff = soff + (uint32_t)(kb * p.c_box_bytes);
#pragma unroll
              for (int k4 = 0; k4 < 4; ++k4) {
                const uint64_t da = gK.at(boff + k4 * 32);
                mma_bf16(d, da, da, idesc, (!first || kb > 0 || k4 > 0) ? 1u : 0u);
              }
            }
            mma_commit(&sh->empty[s]);
          }
          mma_commit(&sh->dfull[buf]);
        }
      } else if (OP == OPK_CS) {
        const uint32_t idesc = idesc_bf16(128, p.npad, 0, 0);
        for (int64_t it = 0; it < my_tiles && ok; ++it, ++fill) {
          const int s = (int)(fill % S);
          if (!mbar_wait(&sh->full[s], (uint32_t)((fill / S) & 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
          tc_fence_after();
          const uint32_t soff = (uint32_t)s * (uint32_t)p.stage_bytes;
          const uint32_t sboff = soff + (uint32_t)(p.mb * p.c_box_bytes);
          for (int b = 0; b < p.mb; ++b) {
            const uint32_t aoff = soff + (uint32_t)(b * p.c_box_bytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_bf16(tmem + (uint32_t)(b * p.npad), gK.at(aoff + ks * 32), gK.at(sboff + ks * 32), idesc,
                       (it > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(&sh->empty[s]);
        }
        mma_commit(&sh->zfull);
      } else if (OP == OPK_PROJ) {
        // D1 (128 x npad) = C_tile^T X: A is MN-major (tile columns contiguous)
        const uint32_t idesc = idesc_bf16(128, p.npad, 1, 0);
        if (p.x_resident) {
          if (!mbar_wait(&sh->xfull, 0, abortp)) { tc_abort(sh, p.status); ok = false; }
          tc_fence_after();
        }
        const int ksteps = p.chunk_rows / 16;
        for (int64_t it = 0; it < my_tiles && ok; ++it) {
          const int buf = (int)(it & 1);
          const uint32_t use = (uint32_t)(it >> 1);
          if (!mbar_wait(&sh->dempty[buf], (use & 1) ^ 1, abortp)) { tc_abort(sh, p.status); ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * 64);
          for (int ch = 0; ch < p.nchunks && ok; ++ch, ++fill) {
            const int s = (int)(fill % S);
            if (!mbar_wait(&sh->full[s], (uint32_t)((fill / S) & 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
            tc_fence_after();
            const uint32_t soff = (uint32_t)s * (uint32_t)p.stage_bytes;
            const uint32_t xoff = p.x_resident ? xres_off : soff + 2 * (uint32_t)p.c_box_bytes;
            for (int ks = 0; ks < ksteps; ++ks) {
              // A: rows 16 ks .. 16 ks + 15 of the chunk; two 64-column atoms p.c_box_bytes apart
              const uint64_t da = gM.at(soff + ks * 2048);
              // B: X^T box (npad rows x 64 of m), K offset within the 64-wide atom
              const uint64_t db = gK.at(xoff + (ks >> 2) * p.x_box_bytes + (ks & 3) * 32);
              mma_bf16(d, da, db, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&sh->empty[s]);
          }
          if (ok) mma_commit(&sh->dfull[buf]);
        }
      } else if (ga_tall) {
        const uint32_t idesc1 = idesc_bf16(128, p.npad, 1, 0);   // T = C_tile^T X
        const uint32_t idesc2 = idesc_bf16(128, p.npad, 0, 1);   // Z_r += C_chunk T
        const uint32_t dz = tmem + 128;                           // Z_r at column 128 + r npad
        if (!mbar_wait(&sh->xfull, 0, abortp)) { tc_abort(sh, p.status); ok = false; }
        tc_fence_after();
        auto next_stage = [&](uint32_t& soff) -> bool {
          const int s = (int)(fill % S);
          if (!mbar_wait(&sh->full[s], (uint32_t)((fill / S) & 1), abortp)) { tc_abort(sh, p.status); return false; }
          tc_fence_after();
          soff = (uint32_t)s * (uint32_t)p.stage_bytes;
          return true;
        };
        auto release_stage = [&]() {
          mma_commit(&sh->empty[(int)(fill % S)]);
          ++fill;
        };
        // T(it) = sum_r C_r^T X_r over the 128-row chunks r
        auto phase1 = [&](int64_t it) -> bool {
          const int buf = (int)(it & 1);
          const uint32_t use = (uint32_t)(it >> 1);
          if (!mbar_wait(&sh->dempty[buf], (use & 1) ^ 1, abortp)) { tc_abort(sh, p.status); return false; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * 64);
          for (int r = 0; r < p.nchunks; ++r) {
            uint32_t soff;
            if (!next_stage(soff)) return false;
            const uint32_t xoff = xres_off + (uint32_t)(2 * r * p.x_box_bytes);
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
              // A: rows 16 ks .. 16 ks + 15 of the chunk, MN-major; B: X^T box 2 r + ks / 4
              const uint64_t da = gM.at(soff + ks * 2048);
              const uint64_t db = gK.at(xoff + (ks >> 2) * p.x_box_bytes + (ks & 3) * 32);
              mma_bf16(d, da, db, idesc1, (r > 0 || ks > 0) ? 1u : 0u);
            }
            release_stage();
          }
          mma_commit(&sh->dfull[buf]);
          return true;
        };
        // Z_r += C_r T(it), T(it) in BF16 from the epilogue
        auto phase2 = [&](int64_t it) -> bool {
          const int buf = (int)(it & 1);
          const uint32_t use = (uint32_t)(it >> 1);
          if (!mbar_wait(&sh->tfull[buf], use & 1, abortp)) { tc_abort(sh, p.status); return false; }
          tc_fence_after();
          const uint32_t toff = tbuf_off + (uint32_t)(buf * p.t_bytes);
          for (int r = 0; r < p.nchunks; ++r) {
            uint32_t soff;
            if (!next_stage(soff)) return false;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
              const uint64_t da = gK.at(soff + (ks >> 2) * p.c_box_bytes + (ks & 3) * 32);
              const uint64_t db = gT.at(toff + ks * 256);
              mma_bf16(dz + (uint32_t)(r * p.npad), da, db, idesc2, (it > 0 || ks > 0) ? 1u : 0u);
            }
            release_stage();
          }
          mma_commit(&sh->tempty[buf]);
          return true;
        };
        for (int64_t it = 0; it < my_tiles && ok; ++it) {
          ok = phase1(it);
          if (ok && it > 0) ok = phase2(it - 1);
        }
        if (ok && my_tiles > 0) ok = phase2(my_tiles - 1);
        mma_commit(&sh->zfull);
      } else {  // OPK_GA
        const uint32_t idesc1 = idesc_bf16(128, p.npad, 1, 0);   // T = C_tile^T X
        const uint32_t idesc2 = idesc_bf16(128, p.npad, 0, 1);   // Z += C_tile T (T MN-major)
        const uint32_t dz = tmem + 128;                           // Z accumulators (mb x npad)
        if (!mbar_wait(&sh->xfull, 0, abortp)) { tc_abort(sh, p.status); ok = false; }
        tc_fence_after();
        auto gemm1 = [&](int64_t it, int s) {
          const int buf = (int)(it & 1);
          const uint32_t d = tmem + (uint32_t)(buf * 64);
          const uint32_t soff = (uint32_t)s * (uint32_t)p.stage_bytes;
          for (int ks = 0; ks < p.c_box_rows / 16; ++ks) {
            const uint64_t da = gM.at(soff + ks * 2048);
            const uint64_t db = gK.at(xres_off + (ks >> 2) * p.x_box_bytes + (ks & 3) * 32);
            mma_bf16(d, da, db, idesc1, ks > 0 ? 1u : 0u);
          }
          mma_commit(&sh->dfull[buf]);
        };
        auto gemm2 = [&](int64_t it, int s) {
          const int buf = (int)(it & 1);
          const uint32_t soff = (uint32_t)s * (uint32_t)p.stage_bytes;
          const uint32_t toff = tbuf_off + (uint32_t)(buf * p.t_bytes);
          for (int b = 0; b < p.mb; ++b)
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
              const uint64_t da = gK.at(soff + (ks >> 2) * p.c_box_bytes + b * 16384 + (ks & 3) * 32);
              // T_j: MN-major, no swizzle: 8x8 core matrices; K groups 128 B apart,
              // MN groups (8 columns of T) 2048 B apart
              const uint64_t db = gT.at(toff + ks * 256);
              mma_bf16(dz + (uint32_t)(b * p.npad), da, db, idesc2, (it > 0 || ks > 0) ? 1u : 0u);
            }
          mma_commit(&sh->tempty[buf]);
          mma_commit(&sh->empty[s]);
        };
        int64_t prev_it = -1;
        int prev_s = 0;
        for (int64_t it = 0; it < my_tiles && ok; ++it, ++fill) {
          const int s = (int)(fill % S);
          const int buf = (int)(it & 1);
          const uint32_t use = (uint32_t)(it >> 1);
          if (!mbar_wait(&sh->full[s], (uint32_t)((fill / S) & 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
          if (!mbar_wait(&sh->dempty[buf], (use & 1) ^ 1, abortp)) { tc_abort(sh, p.status); ok = false; break; }
          tc_fence_after();
          gemm1(it, s);
          if (prev_it >= 0) {
            const uint32_t pu = (uint32_t)(prev_it >> 1);
            if (!mbar_wait(&sh->tfull[prev_it & 1], pu & 1, abortp)) { tc_abort(sh, p.status); ok = false; break; }
            tc_fence_after();
            gemm2(prev_it, prev_s);
          }
          prev_it = it;
          prev_s = s;
        }
        if (ok && prev_it >= 0) {
          const uint32_t pu = (uint32_t)(prev_it >> 1);
          if (!mbar_wait(&sh->tfull[prev_it & 1], pu & 1, abortp)) { tc_abort(sh, p.status); ok = false; }
          else { tc_fence_after(); gemm2(prev_it, prev_s); }
        }
        mma_commit(&sh->zfull);
      }
      // drain: all issued MMAs complete before TMEM can be freed
      mma_commit(&sh->drain);
      int zero = 0;
      mbar_wait(&sh->drain, 0, &zero);
    }
  }
  // =========================================================== epilogue
  else {
    const int q = warp & 3;                         // TMEM lane quarter of this warp
    const int lrow = q * 32 + lane;                 // TMEM lane of this thread
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    if (OP == OPK_PROJ || OP == OPK_GA) {
      for (int64_t it = 0; it < my_tiles; ++it) {
        const int buf = (int)(it & 1);
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(&sh->dfull[buf], use & 1, abortp)) { tc_abort(sh, p.status); break; }
        tc_fence_after();
        // this lane's 64 accumulator columns of the tile (npad <= 64)
        uint32_t r[64];
        const uint32_t ta = tmem + lane_addr + (uint32_t)(buf * 64);
        tmem_ld16<0>(ta, r);
        if (p.npad > 16) tmem_ld16<16>(ta + 16, r);
        if (p.npad > 32) tmem_ld16<32>(ta + 32, r);
        if (p.npad > 48) tmem_ld16<48>(ta + 48, r);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->dempty[buf]);
        const int64_t tile = cta_in_group + it * ctas_in_group;
        const int64_t col = tile * 128 + lrow;
        if (OP == OPK_PROJ && p.o_bytes) {
          // the warp's 32 columns of the b output rows go through shared
          // memory (row-major b x 32, conflict-free), then out as 16-byte
          // stores: 8 rows (BF16) or 4 rows (FP32) per warp instruction
          // instead of one 2- or 4-byte store per row
          uint8_t* ob = obuf + (size_t)q * p.o_bytes;
          __syncwarp();
          // rows c < b; the loops stop at b instead of running predicated
          // over every accumulator column
          auto stage = [&](int c, float x) {
            if (p.out_bf16)
              reinterpret_cast<__nv_bfloat16*>(ob)[c * 32 + lane] = __float2bfloat16_rn(x);
            else
              reinterpret_cast<float*>(ob)[c * 32 + lane] = x;
          };
          if (p.split_hi_lo) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (c >= p.b) break;
              stage(c, __uint_as_float(r[c]) + __uint_as_float(r[c + 32]));
            }
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) {
              if (c >= p.b) break;
              stage(c, __uint_as_float(r[c]));
            }
          }
          __syncwarp();
          const int esz = p.out_bf16 ? 2 : 4;
          const int cpr = 2 * esz;             // 16-byte chunks per staged row
          const int ch = lane % cpr;
          // first column of this lane's chunk; n % 8 == 0, so a chunk that
          // starts inside the row ends inside it
          const int64_t xc = tile * 128 + q * 32 + (int64_t)ch * (16 / esz);
          for (int c0 = 0; c0 < p.b; c0 += 32 / cpr) {
            const int c = c0 + lane / cpr;
            if (c < p.b && xc < p.n) {
              const uint4 v = *reinterpret_cast<const uint4*>(ob + (size_t)c * 32 * esz + ch * 16);
              *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(p.out) + ((int64_t)c * p.ld_out + xc) * esz) = v;
            }
          }
        } else if (OP == OPK_PROJ) {
          if (col < p.n) {
            if (p.split_hi_lo) {
              // S[c] = hi part (column c) + lo part (column c + 32), c < b <= 32
#pragma unroll
              for (int c = 0; c < 32; ++c)
                if (c < p.b) {
                  const float x = __uint_as_float(r[c]) + __uint_as_float(r[c + 32]);
                  if (p.out_bf16)
                    reinterpret_cast<__nv_bfloat16*>(p.out)[(int64_t)c * p.ld_out + col] = __float2bfloat16_rn(x);
                  else
                    reinterpret_cast<float*>(p.out)[(int64_t)c * p.ld_out + col] = x;
                }
            } else {
#pragma unroll
              for (int c = 0; c < 64; ++c)
                if (c < p.b) {
                  const float x = __uint_as_float(r[c]);
                  if (p.out_bf16)
                    reinterpret_cast<__nv_bfloat16*>(p.out)[(int64_t)c * p.ld_out + col] = __float2bfloat16_rn(x);
                  else
                    reinterpret_cast<float*>(p.out)[(int64_t)c * p.ld_out + col] = x;
                }
            }
          }
        } else {
          // T_j row lrow (tile column) -> BF16, MN-major core-matrix layout
          if (!mbar_wait(&sh->tempty[buf], (use & 1) ^ 1, abortp)) { tc_abort(sh, p.status); break; }
          uint8_t* tb = tbuf + (size_t)buf * p.t_bytes;
          const int kgrp = lrow >> 3, krow = lrow & 7;
#pragma unroll
          for (int g = 0; g < 8; ++g)
            if (g < p.npad / 8) {
              uint32_t w[4];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 pr =
                    __floats2bfloat162_rn(__uint_as_float(r[8 * g + 2 * h]), __uint_as_float(r[8 * g + 2 * h + 1]));
                w[h] = *reinterpret_cast<const uint32_t*>(&pr);
              }
              *reinterpret_cast<uint4*>(tb + (size_t)g * 2048 + kgrp * 128 + krow * 16) =
                  make_uint4(w[0], w[1], w[2], w[3]);
            }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh->tfull[buf]);
        }
      }
    }
    if (OP == OPK_GRAM) {
      // chunk sums of this lane's row (npad <= 128 columns) added in FP32
      float acc[128];
#pragma unroll
      for (int i = 0; i < 128; ++i) acc[i] = 0.f;
      bool ok = true;
      for (int64_t c = 0; c < gram_chunks; ++c) {
        const int buf = (int)(c & 1);
        if (!mbar_wait(&sh->dfull[buf], (uint32_t)((c >> 1) & 1), abortp)) { tc_abort(sh, p.status); ok = false; break; }
        tc_fence_after();
        const uint32_t ta = tmem + lane_addr + (uint32_t)(buf * p.npad);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          if (g * 16 < p.npad) {
            uint32_t r[16];
            tmem_ld16<0>(ta + (uint32_t)(g * 16), r);
            tmem_wait_ld();
#pragma unroll
            for (int t = 0; t < 16; ++t) acc[g * 16 + t] += __uint_as_float(r[t]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->dempty[buf]);
      }
      if (ok && !*abortp && lrow < p.m) {
        float* P = reinterpret_cast<float*>(p.out) + (int64_t)blockIdx.x * p.m * p.m + (int64_t)lrow * p.m;
#pragma unroll
        for (int i = 0; i < 128; ++i)
          if (i < p.m) P[i] = acc[i];
      }
    } else if (OP != OPK_PROJ) {
      // final accumulators -> per-CTA partials (rows of this CTA, FP32),
      // 16 columns at a time
      if (mbar_wait(&sh->zfull, 0, abortp)) {
        tc_fence_after();
        float* P = reinterpret_cast<float*>(p.out) + (int64_t)blockIdx.x * p.m * p.b;
        const int mbn = p.mb;
        const uint32_t zoff = (OP == OPK_GA) ? 128u : 0u;
        const int ncol = p.b;
        for (int b = 0; b < mbn; ++b) {
          const int64_t row = row0 + (int64_t)b * 128 + lrow;
          for (int c0 = 0; c0 < p.npad; c0 += 16) {
            uint32_t r[16];
            tmem_ld16<0>(tmem + lane_addr + zoff + (uint32_t)(b * p.npad + c0), r);
            tmem_wait_ld();
            if (row < p.m && !*abortp) {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (c0 + i < ncol) P[row * ncol + c0 + i] = __uint_as_float(r[i]);
            }
          }
        }
        tc_fence_before();
      } else {
        tc_abort(sh, p.status);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// ================================================================ host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_enc_mu;

cudaError_t get_encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lk(g_enc_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return cudaSuccess;
}

// 2-D BF16 map over a row-major (rows x cols) array with row stride ld
// elements; box = (64 columns, box_rows rows); 128-byte swizzle.
cudaError_t make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  cudaError_t e = get_encoder(&enc);
  if (e != cudaSuccess) return e;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

size_t tc_smem_bytes(const TcParams& p) {
  return 1024 + (size_t)p.stages * p.stage_bytes + p.slack_bytes + p.x_res_bytes + 2 * (size_t)p.t_bytes +
         4 * (size_t)p.o_bytes + sizeof(TcShared) + 64;
}

// Rows of a C box: the 16-rounded row count when it is below 128.
int box_rows_for(int64_t m, int cap) { return (int)imin(cap, (m + 15) / 16 * 16); }

// Ring depth and residency: two CTAs per SM (each with half the shared
// memory) whenever a ring of at least three stages fits, since two
// independent TMA -> MMA -> epilogue pipelines per SM keep more bytes in
// flight than one deeper ring; else one CTA with the whole shared memory.
// Sets p.stages; returns the CTAs per SM.
int choose_residency(TcParams& p, int maxst, bool allow_two = true) {
  const int64_t fixed = 1024 + (int64_t)p.slack_bytes + p.x_res_bytes + 2 * (int64_t)p.t_bytes + 4 * (int64_t)p.o_bytes +
                        sizeof(TcShared) + 64;
  const int64_t half = (SMEM_HALF - fixed) / p.stage_bytes;
  if (allow_two && half >= 3) {
    p.stages = (int)imin(maxst, half);
    return 2;
  }
  p.stages = (int)imin(maxst, (SMEM_LIMIT - fixed) / p.stage_bytes);
  return 1;
}

// A tuning-table entry's ring depth and residency on a copy of p (two CTAs
// per SM only where the entry asks for them, `allow_two` permits and three
// stages fit half the shared memory); taken only if the ring keeps at least
// two stages.  Returns whether p changed.
bool apply_tuned(TcParams& p, int& per_sm, const TcParams& q0, const TuneEntry& e, bool allow_two) {
  TcParams q = q0;
  const int per = choose_residency(q, e.stages, allow_two && e.per_sm == 2);
  if (q.stages < 2) return false;
  p = q;
  per_sm = per;
  return true;
}

template <int OP>
cudaError_t launch_tc(const CUtensorMap& mc, const CUtensorMap& mb, const TcParams& p, int ctas, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(p);
  if (smem > (size_t)SMEM_LIMIT) return cudaErrorInvalidValue;
  cudaError_t e = raise_smem_limit(k_tc_stream<OP>);
  if (e != cudaSuccess) return e;
  k_tc_stream<OP><<<ctas, TC_THREADS, smem, st>>>(mc, mb, p);
  return cudaGetLastError();
}

int pad16(int x) { return (x + 15) & ~15; }

// X (m x b FP32, ld ldx) -> X^T (rows x ldt BF16), zero padded; with split,
// rows [lo_off, lo_off + b) hold bf16(X - bf16(X)).
__global__ void k_prep_xt(const float* __restrict__ X, int64_t ldx, int64_t m, int b, int split, int lo_off,
                          int rows, int64_t ldt, __nv_bfloat16* __restrict__ Xt) {
  const int64_t total = (int64_t)rows * ldt;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ldt);
    const int64_t i = e % ldt;
    float v = 0.f;
    if (i < m) {
      if (r < b) {
        v = __bfloat162float(__float2bfloat16_rn(X[i * ldx + r]));
      } else if (split && r >= lo_off && r < lo_off + b) {
        const float x = X[i * ldx + (r - lo_off)];
        v = x - __bfloat162float(__float2bfloat16_rn(x));
      }
    }
    Xt[e] = __float2bfloat16_rn(v);
  }
}

cudaError_t prep_xt(const float* X, int64_t ldx, int64_t m, int b, int split, int lo_off, int rows, int64_t ldt,
                    __nv_bfloat16* Xt, cudaStream_t st) {
  const int64_t total = (int64_t)rows * ldt;
  note_launch("prep_xt");
  k_prep_xt<<<(int)imin(ceil_div(total, 256), 1024), 256, 0, st>>>(X, ldx, m, b, split, lo_off, rows, ldt, Xt);
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- public launchers
bool tc_shape_ok(int64_t m, int64_t n) { return n % 8 == 0 && n >= 64 && m >= 1 && n < (int64_t(1) << 31); }

// Launch shape of a pass: parameters, CTAs per SM, grid size.
struct TcShape {
  TcParams p{};
  int per_sm = 1;
  int ctas = 0;
};

TcShape gram_shape(int64_t m, int64_t n) {
  TcShape t;
  TcParams& p = t.p;
  p.m = m; p.n = n; p.b = (int)m; p.npad = pad16((int)m); p.mb = 1;
  p.c_box_rows = box_rows_for(m, 128); p.c_box_bytes = p.c_box_rows * 128;
  // short unfoldings take 8 boxes (512 columns) per stage: each row then
  // arrives as one 1 KB run instead of 256-byte pieces, which measured ~12%
  // faster from HBM at m = 40
  p.kb = p.c_box_rows <= 48 ? 8 : 2;
  p.stage_bytes = p.kb * p.c_box_bytes;
  p.slack_bytes = 16384;
  p.tiles = ceil_div(n, 64 * p.kb);
  p.row_groups = 1;
  t.per_sm = choose_residency(p, 8);
  TuneEntry e;
  if (tune_lookup(TT_PASS_GRAM, m, p.npad, n, &e)) {
    TcParams q = p;
    q.kb = e.kb;
    q.stage_bytes = q.kb * q.c_box_bytes;
    q.tiles = ceil_div(n, 64 * q.kb);
    apply_tuned(p, t.per_sm, q, e, true);
  }
  t.ctas = (int)imin(p.tiles, (int64_t)num_sms() * t.per_sm);
  return t;
}

// Partial sums for any launch shape (at most two CTAs per SM, tiles of at
// least 64 columns), so that workspace sizes do not depend on the tuning table.
int64_t tc_gram_partials(int64_t m, int64_t n) { return imin(ceil_div(n, 64), 2 * (int64_t)num_sms()) * m * m; }

cudaError_t tc_gram(const __nv_bfloat16* C, int64_t m, int64_t n, float* partials, float* out, int* status,
                    cudaStream_t st) {
  if (m > 128 || !tc_shape_ok(m, n)) return cudaErrorInvalidValue;
  TcShape t = gram_shape(m, n);
  TcParams& p = t.p;
  p.out = partials; p.status = status;
  CUtensorMap mc;
  cudaError_t e = make_map(&mc, C, m, n, n, p.c_box_rows);
  if (e != cudaSuccess) return e;
  {
    ProfScope prof("gram_tc", st, (double)m * n * 2, 2.0 * m * m * n);
    note_launch("gram_tc");
    e = launch_tc<OPK_GRAM>(mc, mc, p, t.ctas, st);
  }
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(partials, t.ctas, m, (int)m, out, m, st);
}

// Y (m x b, ld ldo) = C S^T with S (b x n BF16, row stride lds).
TcShape cs_shape(int64_t m, int64_t n, int b) {
  TcShape t;
  TcParams& p = t.p;
  p.m = m; p.n = n; p.b = b; p.npad = pad16(b); p.kb = 1;
  p.row_groups = ceil_div(m, 512);
  p.mb = (int)imin(4, ceil_div(ceil_div(m, p.row_groups), 128));
  p.c_box_rows = box_rows_for(m, 128); p.c_box_bytes = p.c_box_rows * 128;
  p.s_box_bytes = p.npad * 128;
  p.stage_bytes = (p.mb * p.c_box_bytes + p.s_box_bytes + 1023) / 1024 * 1024;
  p.slack_bytes = 16384;
  p.tiles = ceil_div(n, 64);
  t.per_sm = choose_residency(p, 8);
  TuneEntry e;
  if (tune_lookup(TT_PASS_SKETCH, m, p.npad, n, &e)) apply_tuned(p, t.per_sm, p, e, true);
  const int64_t per = imax(1, imin(p.tiles, (int64_t)num_sms() * t.per_sm / p.row_groups));
  t.ctas = (int)(per * p.row_groups);
  return t;
}

int64_t tc_cs_partials(int64_t m, int64_t n, int b) {
  const int64_t groups = ceil_div(m, 512);
  const int64_t per = imax(1, imin(ceil_div(n, 64), 2 * (int64_t)num_sms() / groups));
  return per * groups * m * b;
}

cudaError_t tc_cs(const __nv_bfloat16* C, int64_t m, int64_t n, const __nv_bfloat16* S, int64_t lds, int b,
                  float* partials, float* out, int64_t ldo, int* status, cudaStream_t st) {
  if (b > 64 || !tc_shape_ok(m, n) || lds % 8 != 0) return cudaErrorInvalidValue;
  TcShape t = cs_shape(m, n, b);
  TcParams& p = t.p;
  if (p.stages < 2) return cudaErrorInvalidValue;
  p.out = partials; p.status = status;
  CUtensorMap mc, ms;
  cudaError_t e = make_map(&mc, C, m, n, n, p.c_box_rows);
  if (e == cudaSuccess) e = make_map(&ms, S, b, n, lds, p.npad);
  if (e != cudaSuccess) return e;
  const int per = t.ctas / (int)p.row_groups;
  {
    ProfScope prof("cs_tc", st, (double)m * n * 2 + (double)b * n * 2, 2.0 * m * n * b);
    note_launch("cs_tc");
    e = launch_tc<OPK_CS>(mc, ms, p, t.ctas, st);
  }
  if (e != cudaSuccess) return e;
  // partial slot = CTA index; rows outside a CTA's row group are not written,
  // so each group's partials are reduced over its own CTAs
  return launch_reduce_partials_grouped(partials, per, (int)p.row_groups, m, b, (int64_t)p.mb * 128, out, ldo, st);
}

// S (b x n, row stride lds, BF16 or FP32) = X^T C; X m x b FP32 (ld ldx).
// With split, X is applied as BF16 hi + lo parts (FP32-accurate products).
size_t tc_proj_scratch_bytes(int64_t m, int b, int split) {
  const int rows = split ? 64 : pad16(b);
  const int64_t ldt = (m + 7) / 8 * 8;
  return (size_t)rows * ldt * 2 + 256;
}

TcShape proj_shape(int64_t m, int64_t n, int b, int split, int o_bytes) {
  TcShape t;
  TcParams& p = t.p;
  p.m = m; p.n = n; p.b = b;
  p.o_bytes = o_bytes;
  p.split_hi_lo = split;
  p.lo_off = split ? 32 : 0;
  p.npad = split ? 64 : pad16(b);
  p.kb = 2; p.mb = 1; p.row_groups = 1;
  p.x_box_bytes = p.npad * 128;
  p.tiles = ceil_div(n, 128);
  auto set_chunks = [&](TcParams& q, int rows) {
    q.chunk_rows = box_rows_for(m, rows);
    q.nchunks = (int)ceil_div(m, q.chunk_rows);
    q.x_resident = q.nchunks == 1 ? 1 : 0;
    q.mpad = (int)ceil_div(q.chunk_rows, 64) * 64;
    q.c_box_rows = q.chunk_rows; q.c_box_bytes = q.chunk_rows * 128;
    q.x_res_bytes = q.x_resident ? (q.mpad / 64) * q.x_box_bytes : 0;
    q.stage_bytes = (2 * q.c_box_bytes + (q.x_resident ? 0 : 2 * q.x_box_bytes) + 1023) / 1024 * 1024;
  };
  // unfoldings taller than one chunk stream 64-row chunks: the smaller ring
  // stages let two CTAs share an SM
  set_chunks(p, m > 128 ? 64 : 128);
  t.per_sm = choose_residency(p, 8);
  TuneEntry e;
  if (tune_lookup(TT_PASS_PROJECT, m, p.npad, n, &e)) {
    TcParams q = p;
    if (m > 128 && e.chunk_rows) set_chunks(q, e.chunk_rows);
    apply_tuned(p, t.per_sm, q, e, true);
  }
  t.ctas = (int)imin(p.tiles, (int64_t)num_sms() * t.per_sm);
  return t;
}

cudaError_t tc_proj(const __nv_bfloat16* C, int64_t m, int64_t n, const float* X, int64_t ldx, int b, int split,
                    void* S, int s_bf16, int64_t lds, void* scratch, int* status, cudaStream_t st) {
  if (!tc_shape_ok(m, n) || (split ? b > 32 : b > 64)) return cudaErrorInvalidValue;
  // staged 16-byte stores need S and its row stride 16-byte aligned; the
  // four warps' buffers take at most 32 KB (b <= 64)
  const int esz = s_bf16 ? 2 : 4;
  const int o_bytes = (int)(((int64_t)b * 32 * esz + 127) / 128 * 128);
  const bool staged = reinterpret_cast<uintptr_t>(S) % 16 == 0 && (lds * esz) % 16 == 0 && 4 * o_bytes <= 32768;
  TcShape t = proj_shape(m, n, b, split, staged ? o_bytes : 0);
  TcParams& p = t.p;
  p.out_bf16 = s_bf16; p.ld_out = lds; p.out = S; p.status = status;
  const int rows = p.npad;
  const int64_t ldt = (m + 7) / 8 * 8;
  __nv_bfloat16* Xt = reinterpret_cast<__nv_bfloat16*>(scratch);
  cudaError_t e = prep_xt(X, ldx, m, b, split, p.lo_off, rows, ldt, Xt, st);
  if (e != cudaSuccess) return e;
  CUtensorMap mc, mx;
  e = make_map(&mc, C, m, n, n, p.chunk_rows);
  if (e == cudaSuccess) e = make_map(&mx, Xt, rows, m, ldt, p.npad);
  if (e != cudaSuccess) return e;
  ProfScope prof("proj_tc", st, (double)m * n * 2 + (double)b * n * (s_bf16 ? 2 : 4), 2.0 * m * n * p.npad);
  note_launch("proj_tc");
  return launch_tc<OPK_PROJ>(mc, mx, p, t.ctas, st);
}

// Y (m x b, ld ldo) = C (C^T X), b <= 64; X m x b FP32 (ld ldx).  For
// m <= 256 a stage holds the whole height of a 128-column tile; taller C
// streams each tile as 128-row chunks twice (C^T X, then C T), so T and the
// m x b accumulators stay on chip: 128 + ceil(m / 128) pad16(b) TMEM columns
// must fit in 512.
TcShape ga_shape(int64_t m, int64_t n, int b) {
  TcShape t;
  TcParams& p = t.p;
  p.m = m; p.n = n; p.b = b; p.npad = pad16(b);
  p.kb = 2; p.row_groups = 1;
  p.mb = (int)ceil_div(m, 128);
  p.x_box_bytes = p.npad * 128;
  p.t_bytes = p.npad / 8 * 2048;
  p.tiles = ceil_div(n, 128);
  if (m <= 256) {
    p.nchunks = 1;
    p.c_box_rows = box_rows_for(m, 256);
    p.mpad = (int)ceil_div(p.c_box_rows, 64) * 64;
    p.slack_bytes = 16384;               // C T reads 128 rows of a shorter box
  } else {
    p.nchunks = p.mb;
    p.c_box_rows = 128;
    p.mpad = 128 * p.nchunks;            // X^T boxes past m are zero-filled
    p.slack_bytes = 0;
  }
  p.c_box_bytes = p.c_box_rows * 128;
  p.x_res_bytes = (p.mpad / 64) * p.x_box_bytes;
  p.stage_bytes = 2 * p.c_box_bytes;
  // 512 TMEM columns (128 + mb npad > 256) leave room for one CTA per SM
  t.per_sm = choose_residency(p, 8, 128 + p.mb * p.npad <= 256);
  TuneEntry e;
  if (tune_lookup(TT_PASS_GRAMAPPLY, m, p.npad, n, &e)) apply_tuned(p, t.per_sm, p, e, 128 + p.mb * p.npad <= 256);
  t.ctas = (int)imin(p.tiles, (int64_t)num_sms() * t.per_sm);
  return t;
}

bool tc_ga_ok(int64_t m, int64_t n, int b) {
  if (b > 64 || b < 1 || !tc_shape_ok(m, n)) return false;
  if (m <= 256) return true;
  if (128 + ceil_div(m, 128) * pad16(b) > 512) return false;
  return ga_shape(m, n, b).p.stages >= 2;
}

size_t tc_ga_scratch_bytes(int64_t m, int b) {
  const int64_t ldt = (m + 7) / 8 * 8;
  return (size_t)pad16(b) * ldt * 2 + 256;
}

int64_t tc_ga_partials(int64_t m, int64_t n, int b) {
  return imin(ceil_div(n, 128), 2 * (int64_t)num_sms()) * m * b;
}

cudaError_t tc_ga(const __nv_bfloat16* C, int64_t m, int64_t n, const float* X, int64_t ldx, int b, float* partials,
                  float* out, int64_t ldo, void* scratch, int* status, cudaStream_t st) {
  if (!tc_ga_ok(m, n, b)) return cudaErrorInvalidValue;
  TcShape t = ga_shape(m, n, b);
  TcParams& p = t.p;
  if (p.stages < 2) return cudaErrorInvalidValue;
  p.out = partials; p.status = status;
  const int64_t ldt = (m + 7) / 8 * 8;
  __nv_bfloat16* Xt = reinterpret_cast<__nv_bfloat16*>(scratch);
  cudaError_t e = prep_xt(X, ldx, m, b, 0, 0, p.npad, ldt, Xt, st);
  if (e != cudaSuccess) return e;
  CUtensorMap mc, mx;
  e = make_map(&mc, C, m, n, n, p.c_box_rows);
  if (e == cudaSuccess) e = make_map(&mx, Xt, p.npad, m, ldt, p.npad);
  if (e != cudaSuccess) return e;
  {
    ProfScope prof("gram_apply_tc", st, (double)m * n * 2, 4.0 * m * n * b);
    note_launch("gram_apply_tc");
    e = launch_tc<OPK_GA>(mc, mx, p, t.ctas, st);
  }
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(partials, t.ctas, m, b, out, ldo, st);
}

}  // namespace ttr

// ---------------------------------------------------------------- test aid
namespace ttr {

// One thread waits, with the bounded wait every tensor-core kernel uses, on
// an mbarrier that nothing ever arrives on; the wait gives up after about
// two seconds and the status word records TT_ETIMEOUT.
__global__ void k_wait_selftest(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
    int no_abort = 0;
    if (!tc::mbar_wait(&bar, 0, &no_abort)) set_status(status, TT_ETIMEOUT);
  }
}

}  // namespace ttr

extern "C" tt_status tt_debug_wait_timeout(void* workspace, void* stream) {
  if (!workspace) {
    ttr::set_last_error("workspace is NULL");
    return TT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* status = (int*)workspace;
  if (cudaMemsetAsync(status, 0, 256, st) != cudaSuccess) {
    ttr::set_last_error("cudaMemsetAsync failed");
    return TT_ECUDA;
  }
  ttr::k_wait_selftest<<<1, 32, 0, st>>>(status);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ttr::set_last_error(cudaGetErrorString(e));
    return TT_ECUDA;
  }
  return TT_OK;
}
