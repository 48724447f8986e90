// TT-SVD (Alg. 1): sequential truncated SVDs of the unfoldings with the
// prescribed accuracy delta = eps ||A||_F / sqrt(d - 1), on the GPU.
//
// The tensor is converted to FP64 once; per mode the unfolding C (m x n,
// row-major) gives its Gram G = C C^T by a cuBLAS DGEMM; cuSOLVER's Dsyevd
// returns all eigenpairs of G (ascending); the eigenvalues come back to
// the host, which picks the smallest rank whose discarded tail
// sum_{i > r} lambda_i is at most delta^2 (capped); core k is the top r
// eigenvectors (left singular vectors of C, stored as FP32) and the next
// remainder U^T C = S V^T is a second DGEMM.  FP64 throughout because the
// Gram squares the singular values: in FP32 the smooth tensors of the
// paper's experiments (singular values decaying below 1e-4 of the first)
// would lose the directions that decide their error.  This is the
// deterministic baseline of the paper, off the randomized hot path:
// host-synchronous, library GEMMs and eigendecompositions.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace ttr {
namespace {

constexpr int64_t kMaxGram = 16384;

struct Handles {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
};

// One handle pair per host thread and device, created on first use.
tt_status handles(Handles** out) {
  thread_local std::map<int, Handles> per_device;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_last_error("cudaGetDevice failed");
    return TT_ECUDA;
  }
  Handles& h = per_device[dev];
  if (!h.blas && cublasCreate(&h.blas) != CUBLAS_STATUS_SUCCESS) {
    h.blas = nullptr;
    set_last_error("cublasCreate failed");
    return TT_ECUDA;
  }
  if (!h.solver && cusolverDnCreate(&h.solver) != CUSOLVER_STATUS_SUCCESS) {
    h.solver = nullptr;
    set_last_error("cusolverDnCreate failed");
    return TT_ECUDA;
  }
  *out = &h;
  return TT_OK;
}

struct SvdLayout {
  std::vector<int64_t> cap;   // clamped rank caps, cap[0] = cap[d] = 1
  std::vector<int64_t> m, n;  // unfolding sizes at the caps, modes 0 .. d-2
  size_t off_A = 0, off_R0 = 0, off_R1 = 0, off_G = 0, off_W = 0, off_U = 0, off_work = 0, off_info = 0,
         total = 0;
  int lwork = 0;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

tt_status svd_layout(const int64_t* dims, int d, const int64_t* max_ranks, int storage, SvdLayout& L) {
  if (!dims) { set_last_error("dims is NULL"); return TT_EINVAL; }
  if (d < 2 || d > 64) { set_last_error("order d must be in [2, 64]"); return TT_EINVAL; }
  if (storage != TT_F32 && storage != TT_BF16) { set_last_error("storage must be TT_F32 or TT_BF16"); return TT_EINVAL; }
  int64_t total = 1;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1) { set_last_error("mode sizes must be >= 1"); return TT_EINVAL; }
    if (total > (int64_t(1) << 46) / dims[k]) { set_last_error("tensor too large"); return TT_EINVAL; }
    total *= dims[k];
  }
  if (max_ranks)
    for (int k = 0; k < d - 1; ++k)
      if (max_ranks[k] < 1) { set_last_error("max_ranks must be >= 1"); return TT_EINVAL; }
  L.cap.assign(d + 1, 1);
  L.m.assign(d - 1, 0);
  L.n.assign(d - 1, 0);
  int64_t n = total;
  size_t maxR = 1, maxG = 1, maxW = 1, maxU = 1;
  for (int k = 0; k < d - 1; ++k) {
    n /= dims[k];
    const int64_t m = L.cap[k] * dims[k];
    if (m > kMaxGram) { set_last_error("unfolding with more than 16384 rows"); return TT_EUNSUPPORTED; }
    if (n > INT32_MAX) { set_last_error("unfolding with more than 2^31 - 1 columns"); return TT_EUNSUPPORTED; }
    L.m[k] = m;
    L.n[k] = n;
    int64_t c = std::min(m, n);
    if (max_ranks) c = std::min(c, max_ranks[k]);
    L.cap[k + 1] = c;
    maxR = std::max(maxR, (size_t)(c * n));
    maxG = std::max(maxG, (size_t)(m * m));
    maxW = std::max(maxW, (size_t)m);
    maxU = std::max(maxU, (size_t)(m * c));
  }
  L.cap[d] = 1;
  Handles* h = nullptr;
  tt_status s = handles(&h);
  if (s != TT_OK) return s;
  int lwork = 0;
  for (int k = 0; k < d - 1; ++k) {
    int lw = 0;
    if (cusolverDnDsyevd_bufferSize(h->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, (int)L.m[k], nullptr,
                                    (int)L.m[k], nullptr, &lw) != CUSOLVER_STATUS_SUCCESS) {
      set_last_error("cusolverDnDsyevd_bufferSize failed");
      return TT_ECUDA;
    }
    lwork = std::max(lwork, lw);
  }
  L.lwork = lwork;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1)); return o; };
  L.off_A = take((size_t)total * 8);
  L.off_R0 = take(maxR * 8);
  L.off_R1 = take(maxR * 8);
  L.off_G = take(maxG * 8);
  L.off_W = take(maxW * 8);
  L.off_U = take(maxU * 8);
  L.off_work = take((size_t)lwork * 8);
  L.off_info = take(sizeof(int));
  L.total = off;
  return TT_OK;
}

// U (m x r, row-major, FP64) = the eigenvectors of the r largest
// eigenvalues, in descending order, from syevd's column-major ascending
// output; also to core (FP32).
__global__ void k_gather_top(const double* __restrict__ Gv, int m, int r, double* __restrict__ U,
                             float* __restrict__ core) {
  const int64_t total = (int64_t)m * r;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(x / r), c = (int)(x % r);
    const double v = Gv[(int64_t)(m - 1 - c) * m + i];
    U[x] = v;
    core[x] = (float)v;
  }
}

// The tensor (FP32 or BF16) to FP64, exactly.
template <typename T>
__global__ void k_to_f64(const T* __restrict__ x, int64_t count, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)ld_elem(x, i);
}

// The last remainder (FP64) to the last core (FP32).
__global__ void k_to_f32(const double* __restrict__ x, int64_t count, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

tt_status blas_check(cublasStatus_t s, const char* what) {
  if (s == CUBLAS_STATUS_SUCCESS) return TT_OK;
  set_last_error((std::string(what) + " failed (cuBLAS status " + std::to_string((int)s) + ")").c_str());
  return TT_ECUDA;
}

tt_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TT_OK;
  set_last_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
  return TT_ECUDA;
}

}  // namespace
}  // namespace ttr

using namespace ttr;

#define SVD_TRY(expr)               \
  do {                              \
    const tt_status s_ = (expr);    \
    if (s_ != TT_OK) return s_;     \
  } while (0)

extern "C" tt_status tt_svd_workspace_size(const int64_t* dims, int d, const int64_t* max_ranks, int storage,
                                           int64_t* core_elems, size_t* bytes) {
  if (!bytes) { set_last_error("bytes is NULL"); return TT_EINVAL; }
  SvdLayout L;
  SVD_TRY(svd_layout(dims, d, max_ranks, storage, L));
  if (core_elems)
    for (int k = 0; k < d; ++k) core_elems[k] = L.cap[k] * dims[k] * L.cap[k + 1];
  *bytes = L.total;
  return TT_OK;
}

extern "C" tt_status tt_svd_decompose(const void* tensor, int storage, const int64_t* dims, int d, double eps,
                                      const int64_t* max_ranks, float* const* cores_out, int64_t* ranks_out,
                                      void* workspace, size_t ws_bytes, void* stream) {
  if (!tensor || !cores_out || !ranks_out || !workspace) {
    set_last_error("tensor, cores_out, ranks_out and workspace must not be NULL");
    return TT_EINVAL;
  }
  if (!(eps >= 0.0) || !std::isfinite(eps)) { set_last_error("eps must be finite and >= 0"); return TT_EINVAL; }
  SvdLayout L;
  SVD_TRY(svd_layout(dims, d, max_ranks, storage, L));
  if (ws_bytes < L.total) { set_last_error("workspace too small"); return TT_ENOMEM; }
  for (int k = 0; k < d; ++k)
    if (!cores_out[k]) { set_last_error("cores_out[k] is NULL"); return TT_EINVAL; }
  Handles* h = nullptr;
  SVD_TRY(handles(&h));
  cudaStream_t st = (cudaStream_t)stream;
  SVD_TRY(blas_check(cublasSetStream(h->blas, st), "cublasSetStream"));
  if (cusolverDnSetStream(h->solver, st) != CUSOLVER_STATUS_SUCCESS) {
    set_last_error("cusolverDnSetStream failed");
    return TT_ECUDA;
  }
  char* ws = static_cast<char*>(workspace);
  double* A64 = (double*)(ws + L.off_A);
  double* G = (double*)(ws + L.off_G);
  double* W = (double*)(ws + L.off_W);
  double* U = (double*)(ws + L.off_U);
  double* work = (double*)(ws + L.off_work);
  int* info = (int*)(ws + L.off_info);
  const double one = 1.0, zero = 0.0;
  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= dims[k];
  {
    const int blocks = (int)imin(ceil_div(total, 256), 4096);
    note_launch("svd_convert");
    if (storage == TT_BF16)
      k_to_f64<__nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)tensor, total, A64);
    else
      k_to_f64<float><<<blocks, 256, 0, st>>>((const float*)tensor, total, A64);
    SVD_TRY(cuda_check(cudaGetLastError(), "k_to_f64"));
  }
  std::vector<double> w;
  double delta2 = 0.0;
  int64_t r_prev = 1;
  const double* C = A64;
  ranks_out[0] = 1;
  for (int k = 0; k < d - 1; ++k) {
    const int m = (int)(r_prev * dims[k]);
    const int n = (int)L.n[k];
    // Alg. 1 step 3 (as a Gram): G = C C^T, C row-major m x n is the
    // column-major n x m matrix C', so G = C'^T C'
    SVD_TRY(blas_check(cublasDgemm(h->blas, CUBLAS_OP_T, CUBLAS_OP_N, m, m, n, &one, C, n, C, n, &zero, G, m),
                       "Gram DGEMM"));
    if (cusolverDnDsyevd(h->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, G, m, W, work, L.lwork,
                         info) != CUSOLVER_STATUS_SUCCESS) {
      set_last_error("cusolverDnDsyevd failed");
      return TT_ECUDA;
    }
    w.resize(m);
    int hinfo = 0;
    SVD_TRY(cuda_check(cudaMemcpyAsync(w.data(), W, sizeof(double) * m, cudaMemcpyDeviceToHost, st), "eigenvalues"));
    SVD_TRY(cuda_check(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st), "syevd info"));
    SVD_TRY(cuda_check(cudaStreamSynchronize(st), "cudaStreamSynchronize"));
    if (hinfo != 0) {
      set_last_error(("cusolverDnDsyevd did not converge (info " + std::to_string(hinfo) + ")").c_str());
      return TT_ECUDA;
    }
    // descending eigenvalues (squared singular values).  The discarded
    // tails are suffix sums of the eigenvalues as computed: the small ones
    // are rounding noise of either sign, so they are summed unclamped and
    // cancel instead of adding a bias; the first Gram's trace is ||A||_F^2
    std::vector<double> lam(m);
    for (int i = 0; i < m; ++i) lam[i] = w[m - 1 - i];
    const int64_t cap = L.cap[k + 1];
    std::vector<double> tail(m + 1, 0.0);
    for (int i = m - 1; i >= 0; --i) tail[i] = tail[i + 1] + lam[i];
    if (k == 0) delta2 = eps * eps * std::max(0.0, tail[0]) / (double)(d - 1);
    // Alg. 1 step 4: the smallest r with sum_{i >= r} lam_i <= delta^2
    int64_t r = cap;
    for (int64_t rr = 1; rr <= cap; ++rr)
      if (tail[rr] <= delta2) {
        r = rr;
        break;
      }
    ranks_out[k + 1] = r;
    // Alg. 1 step 5: core k = the top r left singular vectors
    const int64_t cnt = (int64_t)m * r;
    note_launch("svd_gather");
    k_gather_top<<<(int)imin(ceil_div(cnt, 256), 1024), 256, 0, st>>>(G, m, (int)r, U, cores_out[k]);
    SVD_TRY(cuda_check(cudaGetLastError(), "k_gather_top"));
    // Alg. 1 step 6: the next remainder U^T C (r x n, row-major) is the
    // column-major n x r matrix C' U
    double* R = (double*)(ws + ((k % 2 == 0) ? L.off_R0 : L.off_R1));
    SVD_TRY(blas_check(cublasDgemm(h->blas, CUBLAS_OP_N, CUBLAS_OP_T, n, (int)r, m, &one, C, n, U, (int)r, &zero, R,
                                   n),
                       "projection DGEMM"));
    C = R;
    r_prev = r;
  }
  // Alg. 1 step 8: the last core is the last remainder
  {
    const int64_t cnt = r_prev * dims[d - 1];
    note_launch("svd_convert");
    k_to_f32<<<(int)imin(ceil_div(cnt, 256), 1024), 256, 0, st>>>(C, cnt, cores_out[d - 1]);
    SVD_TRY(cuda_check(cudaGetLastError(), "k_to_f32"));
  }
  ranks_out[d] = 1;
  return cuda_check(cudaStreamSynchronize(st), "cudaStreamSynchronize");
}
