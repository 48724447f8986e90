// cuBLAS for the plain GEMMs of the Gram-power route: one handle per host
// thread and device, created on first use; every call sets the stream and
// a workspace inside the caller's workspace, so nothing is allocated while
// work is enqueued (or captured into a graph).
#include <cublas_v2.h>

#include <map>

#include "common.cuh"
#include "kernels.h"

namespace ttr {

namespace {
// The handles live until the process exits: a destructor run at thread or
// process exit could come after the CUDA context is already torn down.
cudaError_t handle(cublasHandle_t* out) {
  thread_local std::map<int, cublasHandle_t> per_device;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cublasHandle_t& h = per_device[dev];
  if (!h && cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
    h = nullptr;
    return cudaErrorUnknown;
  }
  *out = h;
  return cudaSuccess;
}

cudaError_t prepare(cublasHandle_t* h, void* ws, size_t ws_bytes, cudaStream_t st) {
  cudaError_t e = handle(h);
  if (e != cudaSuccess) return e;
  if (cublasSetStream(*h, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  if (cublasSetWorkspace(*h, ws, ws_bytes) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  return cudaSuccess;
}
}  // namespace

// Creates this thread's handle for the current device ahead of the first
// GEMM, so that no handle is created while a stream is being captured.
cudaError_t blas_init() {
  cublasHandle_t h;
  return handle(&h);
}

// G (m x m, FP32) = C C^T for a row-major m x n C (BF16 or FP32); FP32
// accumulation (no TF32).  C row-major is the column-major n x m C', so
// G = C'^T C'.
cudaError_t blas_gram(const void* C, int c_bf16, int64_t m, int64_t n, float* G, void* ws, size_t ws_bytes,
                      cudaStream_t st) {
  cublasHandle_t h;
  cudaError_t e = prepare(&h, ws, ws_bytes, st);
  if (e != cudaSuccess) return e;
  const float one = 1.f, zero = 0.f;
  const cudaDataType_t t = c_bf16 ? CUDA_R_16BF : CUDA_R_32F;
  ProfScope prof("gram_blas", st, (double)m * n * (c_bf16 ? 2 : 4), 2.0 * m * m * n);
  note_launch("gram_blas");
  const cublasStatus_t s = cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)m, (int)m, (int)n, &one, C, t, (int)n, C, t,
                                        (int)n, &zero, G, CUDA_R_32F, (int)m, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  return s == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

// W (m x c, row stride ldw) = G X, G m x m symmetric FP32, X m x c (row
// stride ldx): column-major W' (c x m) = X' G.
cudaError_t blas_gram_apply(const float* G, int64_t m, const float* X, int64_t ldx, int c, float* W, int64_t ldw,
                            void* ws, size_t ws_bytes, cudaStream_t st) {
  cublasHandle_t h;
  cudaError_t e = prepare(&h, ws, ws_bytes, st);
  if (e != cudaSuccess) return e;
  const float one = 1.f, zero = 0.f;
  // G (at most 16 MB) is read from L2 by every power: no algorithmic HBM
  // bytes are counted for it
  ProfScope prof("gram_power", st, 0.0, 2.0 * m * m * c);
  note_launch("gram_power");
  const cublasStatus_t s = cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, c, (int)m, (int)m, &one, X, (int)ldx, G, (int)m,
                                       &zero, W, (int)ldw);
  return s == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace ttr
