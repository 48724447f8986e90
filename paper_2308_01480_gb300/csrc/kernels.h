// Internal launcher declarations shared by the kernel files and the host
// driver.  Every launcher enqueues on the given stream and returns the
// launch status; none synchronises.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ttr {

// ---- error message returned by tt_rbki_last_error (api.cu)
void set_last_error(const char* msg);

// ---- accounting (profile.cu)
void note_launch(const char* family, int count = 1);
// Brackets the launches made during its lifetime with CUDA events on `st`
// and adds bytes/flops to the family, when profiling is on.
class ProfScope {
 public:
  ProfScope(const char* family, cudaStream_t st, double bytes, double flops);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* fam_;
  cudaStream_t st_;
  cudaEvent_t a_{}, b_{};
  bool timed_ = false;
};

// ---- SIMT streaming passes (stream_simt.cu)
// partials (optional): b x n x simt_proj_splits(m, n) floats enabling the
// row-split form for tall-thin unfoldings
template <typename TIn, typename TOut>
cudaError_t simt_proj(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b, TOut* S,
                      int64_t lds, cudaStream_t st, float* partials = nullptr);
int64_t simt_proj_splits(int64_t m, int64_t n);
template <typename TIn>
cudaError_t simt_cs(const TIn* C, int64_t m, int64_t n, const float* S, int64_t lds, int b,
                    float* partials, float* out, int64_t ldo, cudaStream_t st);
template <typename TIn>
cudaError_t simt_ga(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b,
                    float* partials, float* out, int64_t ldo, cudaStream_t st);
template <typename TIn>
cudaError_t simt_gram(const TIn* C, int64_t m, int64_t n, float* partials, float* out, cudaStream_t st);
template <typename TIn>
cudaError_t simt_ga_with_ctas(const TIn* C, int64_t m, int64_t n, const float* X, int ldx, int b,
                              float* partials, int64_t max_ctas, float* out, int64_t ldo, cudaStream_t st);
bool simt_ga_fused_ok(int64_t m, int b);
cudaError_t launch_reduce_partials(const float* P, int S, int64_t rows, int cols, float* out, int64_t ldo,
                                   cudaStream_t st);
cudaError_t launch_reduce_partials_grouped(const float* P, int per, int groups, int64_t rows, int cols,
                                           int64_t group_rows, float* out, int64_t ldo, cudaStream_t st);

// ---- tuning table of the streaming passes' launch shapes (tune.cu)
struct TuneEntry {
  int stages;      // ring depth cap (2 .. 8)
  int per_sm;      // CTAs per SM wanted (1 or 2; 2 only where three stages fit half the shared memory)
  int kb;          // Gram: 64-column boxes per stage (1, 2, 4, 8); 0 elsewhere
  int chunk_rows;  // projection of unfoldings taller than 128 rows: rows per chunk (64, 128); 0 = rule
};
int tune_row_bucket(int64_t m);
int tune_n_class(int64_t n);
bool tune_lookup(int op, int64_t m, int npad, int64_t n, TuneEntry* out);

// ---- tensor-core streaming passes on BF16 unfoldings (stream_tc.cu)
bool tc_shape_ok(int64_t m, int64_t n);
int64_t tc_gram_partials(int64_t m, int64_t n);
cudaError_t tc_gram(const __nv_bfloat16* C, int64_t m, int64_t n, float* partials, float* out, int* status,
                    cudaStream_t st);
int64_t tc_cs_partials(int64_t m, int64_t n, int b);
cudaError_t tc_cs(const __nv_bfloat16* C, int64_t m, int64_t n, const __nv_bfloat16* S, int64_t lds, int b,
                  float* partials, float* out, int64_t ldo, int* status, cudaStream_t st);
size_t tc_proj_scratch_bytes(int64_t m, int b, int split);
cudaError_t tc_proj(const __nv_bfloat16* C, int64_t m, int64_t n, const float* X, int64_t ldx, int b, int split,
                    void* S, int s_bf16, int64_t lds, void* scratch, int* status, cudaStream_t st);
bool tc_ga_ok(int64_t m, int64_t n, int b);
size_t tc_ga_scratch_bytes(int64_t m, int b);
int64_t tc_ga_partials(int64_t m, int64_t n, int b);
cudaError_t tc_ga(const __nv_bfloat16* C, int64_t m, int64_t n, const float* X, int64_t ldx, int b, float* partials,
                  float* out, int64_t ldo, void* scratch, int* status, cudaStream_t st);
int64_t simt_ga_partials(int64_t m, int64_t n, int b);   // floats
int64_t simt_cs_partials(int64_t m, int64_t n, int b);   // floats
int64_t simt_gram_partials(int64_t m, int64_t n);        // floats

// ---- small dense algebra (small.cu)
size_t orth_scratch_floats(int64_t m, int zc, int kq);
cudaError_t launch_orth_block(const float* Z, int64_t ldz, int64_t m, int zc, float* Q, int64_t ldq, int kq,
                              int c, float* scratch, uint64_t seed, int* status, const int* only_if,
                              cudaStream_t st);

// ---- multi-CTA block orthonormalisation (orth.cu)
bool orth_fast_ok(int64_t m, int kq, int b);
size_t orth_fast_scratch_floats(int64_t m, int kq, int b);
cudaError_t launch_orth_fast(const float* W, int64_t ldw, int64_t m, int b, float* Q, int64_t ldq, int kq,
                             float* scratch, unsigned* ticket, int* flag, cudaStream_t st);

// ---- block orthonormalisation on one thread-block cluster (orth_cluster.cu)
bool orth_cluster_ok(int64_t m, int kq, int b);
// c <= b columns are kept (c < b: the Krylov dimension cap)
cudaError_t launch_orth_cluster(const float* W, int64_t ldw, int64_t m, int b, int c, float* Q, int64_t ldq, int kq,
                                int* flag, cudaStream_t st);

// ---- one block on a cluster of up to 16 CTAs, reduce-scatter sums and
// in-launch repair of deficient columns (orth_cluster_rs.cu): Y (m x zc,
// row stride ldy) orthonormalised against Q[:, :kq0], c columns appended to
// Q; when Xg is given the new block is also written there (m x xld, zero
// padded to pad4(c) columns, 16-byte rows for the Gram power).  Returns
// cudaErrorNotSupported when the device cannot hold the cluster.
// The same sequence over all CTAs of one cooperative launch (at most one
// per SM, shares reduced through global memory, bounded barriers) for blocks
// with more rows than a cluster holds; scratch holds
// orth_grid_rs_scratch_floats floats (barrier words, shares, sums).
bool orth_grid_rs_ok(int64_t m, int kq0, int zc, int c);
size_t orth_grid_rs_scratch_floats(int64_t m, int kq0, int zc);
cudaError_t launch_orth_grid_rs(const float* Y, int64_t ldy, int zc, int64_t m, int c, int kq0, float* Q,
                                int64_t ldq, float* Xg, int xld, uint64_t seed, float* scratch, int* status,
                                cudaStream_t st);
bool orth_cluster_rs_ok(int64_t m, int kq0, int zc, int c);
cudaError_t launch_orth_cluster_rs(const float* Y, int64_t ldy, int zc, int64_t m, int c, int kq0, float* Q,
                                   int64_t ldq, float* Xg, int xld, uint64_t seed, int* status, cudaStream_t st);

// ---- Gram matrix for 128 < m <= 2048 and the Gram power W = G X (gram.cu)
bool gram_tiled_ok(int64_t m);
bool gram_tc_tiled_ok(int64_t m, int64_t n);
size_t gram_tiled_partials(int64_t m, int64_t n, int c_bf16);   // floats
// G (m x m, FP32, both triangles) = C C^T; C BF16 (tensor cores when
// tc_shape_ok) or FP32 (SIMT)
cudaError_t gram_tiled(const void* C, int c_bf16, int64_t m, int64_t n, float* partials, float* G, int* status,
                       cudaStream_t st);
bool gram_power_ok(int64_t m, int c);
// W (m x c, row stride ldw) = G X, G m x m FP32, X m x c, 16-byte aligned
// with row stride ldx % 4 == 0 (a padded copy of the block)
cudaError_t gram_power(const float* G, int64_t m, const float* X, int64_t ldx, int c, float* W, int64_t ldw,
                       cudaStream_t st);

// ---- register-tiled symmetric eigensolver, k <= 160, r <= 32 (eig_reg.cu)
bool eig_reg_ok(int k, int r);
// scratch: k * k + 3 k floats
cudaError_t launch_eig_reg(const float* H, int64_t ldh, int k, int r, float* V, int ldv, float* evals,
                           float* scratch, cudaStream_t st);

// ---- Rayleigh-Ritz through a tridiagonal eigensolver (eig.cu)
// Rayleigh-Ritz through the singular vectors of B = Q^T C (rr_svd.cu):
// H = B B^T with exact FP32 products and compensated sums (per-CTA partials
// summed in FP64), FP64 Cholesky, one-sided Jacobi in FP32 on the factor.
constexpr int RR_SVD_KMAX = 160;
int gram_df_splits(int k, int64_t n);
size_t gram_df_partial_doubles(int k, int64_t n);
template <typename T>
cudaError_t gram_df(const T* B, int k, int64_t n, int64_t ldb, double* partials, double* H, cudaStream_t st);
bool rr_svd_ok(int k, int r);
cudaError_t launch_rr_svd(const double* H, int k, int r, const float* Q, int64_t m, int64_t ldq, float* U,
                          float* core, int* status, cudaStream_t st);
bool eig_top_ok(int k);
size_t rr_fast_scratch_floats(int64_t m, int k, int r);
size_t eig_scratch_floats(int k, int r);
cudaError_t launch_eig_top(const float* H, int64_t ldh, int k, int r, float* V, float* scratch, float* evals,
                           cudaStream_t st);
cudaError_t launch_rr_fast(const float* Q, const float* W, int64_t ld, int64_t m, int k, int r, int identity_q,
                           float* scratch, float* U, float* core, cudaStream_t st);
size_t rr_scratch_floats(int k);
// exhaustion with D = n < m: Y = C V' (m x r), V' the top-r eigenvectors of
// C^T C (n x n, n <= 224); scratch: colgram_scratch_floats(m, n, r)
size_t colgram_scratch_floats(int64_t m, int n, int r);
template <typename T>
cudaError_t launch_colgram(const T* C, int64_t m, int n, int r, float* scratch, float* Y, cudaStream_t st);
cudaError_t launch_rayleigh_ritz(const float* Q, const float* W, int64_t ld, int64_t m, int k, int r,
                                 int identity_q, float* scratch, float* U, float* core, cudaStream_t st);
// The last core (the last remainder of dtype TT_F32/TT_BF16, last_count
// entries) and a non-finite check of it and of cores[0..ncores) (counts[k]
// entries each), one launch; ncores <= kFinaliseMaxCores.
constexpr int kFinaliseMaxCores = 63;
cudaError_t launch_finalise(const void* R, int dtype, int64_t last_count, float* last_core,
                            const float* const* cores, const int64_t* counts, int ncores, int* status,
                            cudaStream_t st);

// ---- inputs (misc.cu)
cudaError_t launch_omega(uint64_t seed, int mode, int64_t n, int b, void* out, int dtype, int64_t si,
                         int64_t sc, cudaStream_t st, int64_t slab_w = 0, int64_t slab_nd = 0, int64_t slab_lo = 0);
cudaError_t launch_omega_transpose_any(const float* src, int64_t n, int b, void* dst, int dtype, cudaStream_t st);
cudaError_t launch_permute(const void* src, int sdt, void* dst, int ddt, const int64_t* dims,
                           const int64_t* sstrides, const int* perm, int d, cudaStream_t st);

}  // namespace ttr
