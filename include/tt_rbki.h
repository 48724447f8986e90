/*
 * tt_rbki.h - C ABI of the GB300 (sm_103a) randomized block Krylov
 * tensor-train library.
 *
 * The library computes the TT approximation of Alg. 3 (TT-rBKI) of
 * "A Randomized Block Krylov Method for Tensor Train Approximation"
 * (Yu, Feng, Chen, Cai, Qi): for each mode k = 1..d-1 it unfolds the
 * remainder to C = reshape(R, [r_{k-1} I_k, I_{k+1}...I_d]) (Alg. 3 step 2),
 * builds an orthonormal basis Q of the block Krylov space
 * [C W, (C C^T) C W, ..., (C C^T)^q C W] with a Gaussian W of r_k + p
 * columns (Alg. 3 steps 3-5, left-side reading), takes the top-r_k left
 * singular vectors of Q^T C by Rayleigh-Ritz (Alg. 3 steps 6-8), stores
 * them as core k (step 9) and carries U^T C forward (step 10).  The last
 * remainder is core d (step 12).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Tensors are dense, row-major, i_1 slowest (the unfolding at mode k is a
 *    free view).  Cores are row-major [r_{k-1}][I_k][r_k] float32.
 *  - Pointers documented as "device" must be device-accessible CUDA memory
 *    of the current device; "host" pointers are ordinary host memory.
 *  - The caller owns every buffer: the input tensor, the cores, the
 *    workspace.  No entry point allocates device memory (the batched graph
 *    form's CUDA graph excepted), and none keeps a pointer after it returns
 *    (the graph keeps the device pointers it was built with).
 *  - All device work is enqueued on `stream` (a cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Entry points do not synchronise
 *    the stream; results are ready once the stream has reached that point.
 *    A call enqueues a fixed sequence of kernels with no host round trip,
 *    so it may be captured into a CUDA graph.
 *  - Errors are returned as tt_status.  Argument errors are detected on the
 *    host before anything is enqueued.  Numerical conditions found on the
 *    device (non-finite input) are written to a status word inside the
 *    workspace and read with tt_rbki_device_status().  Device code never
 *    traps.  tt_rbki_last_error() returns a message for the last failing
 *    call of the calling thread.
 *  - Ranks larger than feasible are clamped, not rejected:
 *    r_k' = min(r_k, r_{k-1}' I_k, I_{k+1}...I_d), r_0' = r_d' = 1.
 */
#ifndef TT_RBKI_H
#define TT_RBKI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TT_API __attribute__((visibility("default")))
#else
#define TT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_EINVAL = 1,        /* bad argument (shape, rank, pointer, size)          */
  TT_ENOMEM = 2,        /* workspace smaller than tt_rbki_workspace_size()   */
  TT_ECUDA = 3,         /* a CUDA runtime call failed                         */
  TT_EBREAKDOWN = 4,    /* (device status) a basis block could not be made
                           orthonormal even after random replacement         */
  TT_ENONFINITE = 5,    /* (device status) NaN or Inf found in the input      */
  TT_EUNSUPPORTED = 6,  /* shape outside the supported envelope               */
  TT_ETIMEOUT = 7       /* (device status) a bounded wait inside a kernel
                           gave up; the results of that call are invalid     */
} tt_status;

typedef enum {
  TT_F32 = 0,           /* IEEE binary32                                      */
  TT_BF16 = 1           /* bfloat16, round-to-nearest-even from binary32      */
} tt_dtype;

/* Options; a NULL pointer means all defaults (the zero-initialised struct
 * is NOT the default: use tt_rbki_default_options). */
typedef struct {
  int32_t storage;      /* tt_dtype of the input tensor and of the streamed
                           unfoldings.  TT_F32: FP32 storage, FP32 arithmetic
                           (the plain FP32 form).  TT_BF16: BF16 storage with
                           BF16 tensor-core products accumulated in FP32 (the
                           precision form).  Default TT_F32.                  */
  int32_t remainder;    /* tt_dtype of the remainders R_1..R_{d-1};
                           default = storage.                                 */
  int32_t exhaust_gram; /* 1 (default): when the Krylov basis of a mode would
                           reach all m = r_{k-1} I_k rows (exhaustion), form
                           the m x m Gram C C^T in one pass instead of the
                           sketch + Krylov passes; the result is the same
                           exact truncated SVD.  0: always run the Krylov
                           passes with the dimension cap.                     */
  int32_t batch_streams;/* batched entry points: number of concurrent worker
                           streams the problems are spread over (1..64);
                           0 (default) = 16.  Ignored by single problems.    */
  int32_t method;       /* TT_METHOD_RBKI (default): Alg. 3, block Krylov
                           basis [C W, ..., (C C^T)^q C W].  TT_METHOD_RSI:
                           Alg. 4, subspace iteration, basis of
                           (C C^T)^q C W only (b columns), re-orthonormalised
                           after every power.  Either with q = 0 is TT-rSVD
                           (Alg. 2).  Both truncate by Rayleigh-Ritz.         */
  int32_t gram_power;   /* 1 (default): when a mode has several Krylov powers
                           over an unfolding with n <= 8192 columns (at most
                           2048 rows), or at least three over a BF16 one of
                           at most 1024 rows, form G = C C^T once (tensor
                           cores for BF16, FP32 accumulation) and compute
                           each power as G X: the same Krylov space, fewer
                           passes over C.  0: every power streams C.          */
  int32_t paper_literal;/* 0 (default): Rayleigh-Ritz truncation of the left
                           Krylov basis (above).  1: the paper's steps taken
                           literally, a study form: Alg. 3 builds its Krylov
                           matrix on the right and keeps the first r_k
                           columns of an unpivoted QR of Y = C U (steps 4-8);
                           those columns span (C C^T) C W(:, 1:r_k), which is
                           what this form computes (one power of the first
                           r_k columns of W for q >= 1; Alg. 2, C W(:, 1:r_k),
                           for q = 0), orthonormalised and stored as the core
                           without Rayleigh-Ritz.  With TT_METHOD_RSI, Alg. 4
                           taken literally: (C C^T)^q C W(:, 1:r_k).  The
                           exhaustion Gram routes are not used.               */
  int32_t accurate_rr;  /* 0 (default): Rayleigh-Ritz on H = Q^T C C^T Q
                           formed from the FP32 powers, eigenvectors in FP32
                           (H holds squared singular values: directions with
                           sigma_j / sigma_1 below ~2.4e-4 drown in its
                           rounding).  1: the singular vectors of
                           B = Q^T C (Alg. 3 step 7) without that loss: B by
                           an FP32 projection pass, H = B B^T with exact FP32
                           products and compensated (double-FP32) sums, FP64
                           partial sums and an FP64 Cholesky H = L L^T, and
                           one-sided Jacobi on L in FP32; the exhaustion
                           route over rows takes B = C.  Needs bases of at
                           most 160 columns; the column-Gram exhaustion route
                           is not used.  Not combined with paper_literal.     */
  int32_t reserved;     /* must be zero                                       */
} tt_options;

enum { TT_METHOD_RBKI = 0, TT_METHOD_RSI = 1 };

/* Fills *opts with the defaults described above. */
TT_API tt_status tt_rbki_default_options(tt_options* opts);

/*
 * Rank clamp and core sizes (Def. 2; Alg. 3 input).
 *   dims       host, d mode sizes I_1..I_d, each >= 1; 2 <= d <= 64.
 *   ranks      host, d-1 target ranks r_1..r_{d-1}, each >= 1.
 *   ranks_out  host, d+1 entries: r_0' = 1, r_1'..r_{d-1}', r_d' = 1.
 *   core_elems host, d entries: r_{k-1}' I_k r_k' (may be NULL).
 * Errors: TT_EINVAL on d outside [2, 64], a dimension or rank < 1, or
 *         overflow.
 */
TT_API tt_status tt_rbki_core_sizes(const int64_t* dims, int d, const int64_t* ranks,
                             int64_t* ranks_out, int64_t* core_elems);

/*
 * Workspace bytes needed by tt_rbki_decompose / _omega for this problem.
 * oversample = p >= 0, q >= 0 (Alg. 3 input).  opts may be NULL.
 */
TT_API tt_status tt_rbki_workspace_size(const int64_t* dims, int d, const int64_t* ranks,
                                 int oversample, int q, const tt_options* opts,
                                 size_t* bytes);

/*
 * How each mode of a decomposition will run (the plan tt_rbki_decompose
 * follows for the same arguments).  Planning only: no GPU work, no
 * allocation, callable without a device.  Every route computes the rank-r_k'
 * truncation of Alg. 3 steps 3-10 for the unfolding C (m x n, D = min(m, n)):
 *   TT_ROUTE_KRYLOV      sketch C W, Krylov powers C (C^T X) streamed over C,
 *                        block orthonormalisation, Rayleigh-Ritz;
 *   TT_ROUTE_GRAM_ROWS   the basis would span all D = m rows (exhaustion):
 *                        one Gram pass C C^T and its top r_k' eigenvectors
 *                        (the exact truncated SVD);
 *   TT_ROUTE_GRAM_COLS   exhaustion with D = n < m: the n x n Gram C^T C;
 *   TT_ROUTE_GRAM_POWER  as TT_ROUTE_KRYLOV, with G = C C^T formed once and
 *                        every power computed as G X.
 *   modes      host, at least d-1 entries; entry k-1 describes mode k.
 *   max_modes  capacity of modes.
 * Errors: TT_EINVAL for a NULL modes or max_modes < d-1; otherwise the
 * errors of tt_rbki_workspace_size.
 */
enum { TT_ROUTE_KRYLOV = 0, TT_ROUTE_GRAM_ROWS = 1, TT_ROUTE_GRAM_COLS = 2, TT_ROUTE_GRAM_POWER = 3 };

typedef struct tt_mode_plan {
  int64_t m, n;          /* unfolding: r_{k-1}' I_k rows, I_{k+1}..I_d columns  */
  int64_t r_in, r_out;   /* clamped ranks r_{k-1}', r_k'                        */
  int32_t b;             /* block width r_k' + p                                */
  int32_t basis_cols;    /* columns of the Krylov (Alg. 3) or subspace (Alg. 4)
                            basis, at most D                                    */
  int32_t blocks;        /* Krylov blocks; 1 for Alg. 4                         */
  int32_t powers;        /* products C (C^T X) applied, the one that feeds
                            Rayleigh-Ritz included; 0 on the Gram routes        */
  int32_t route;         /* TT_ROUTE_*                                          */
  int32_t tensor_cores;  /* 1: the passes over C run on the tensor cores (BF16
                            C with n % 8 == 0 and n >= 64)                      */
  int32_t fused_power;   /* 1: a power streaming C is one fused pass            */
  int32_t reserved;      /* 0                                                   */
} tt_mode_plan;

TT_API tt_status tt_rbki_plan_modes(const int64_t* dims, int d, const int64_t* ranks, int oversample,
                                    int q, const tt_options* opts, tt_mode_plan* modes, int max_modes);

/*
 * TT-rBKI decomposition (Alg. 3) with Omega drawn on the device.
 *   tensor     device, prod(dims) elements of opts->storage, row-major.
 *   omega_seed 64-bit seed.  Omega_k (n_k x (r_k' + p), n_k = I_{k+1}..I_d)
 *              has entry (i, c) = the (c mod 4)-th output of the Box-Muller
 *              transform applied to Philox4x32-10 (Salmon et al., SC'11) with
 *              counter (i mod 2^32, i >> 32, c / 4, k) and key
 *              (seed mod 2^32, seed >> 32); outputs (x0,x1) and (x2,x3) give
 *              the cosine/sine pairs with uniforms ((x >> 9) + 1/2) 2^-23.
 *              Evaluated in binary32 on the device.
 *   cores_out  host array of d device pointers; core k receives
 *              r_{k-1}' I_k r_k' float32 values [r_{k-1}'][I_k][r_k'].
 *   ranks_out  host, d+1 entries (as tt_rbki_core_sizes); may be NULL.
 *   workspace  device, ws_bytes >= tt_rbki_workspace_size(); 256-byte
 *              aligned.  Holds intermediates and the device status word.
 *   stream     cudaStream_t.
 * Errors: TT_EINVAL, TT_ENOMEM (workspace too small), TT_EUNSUPPORTED,
 *         TT_ECUDA (launch failure).  Device-side conditions: see
 *         tt_rbki_device_status.
 */
TT_API tt_status tt_rbki_decompose(const void* tensor, const int64_t* dims, int d,
                            const int64_t* ranks, int oversample, int q,
                            uint64_t omega_seed, float* const* cores_out,
                            int64_t* ranks_out, void* workspace, size_t ws_bytes,
                            void* stream, const tt_options* opts);

/*
 * As tt_rbki_decompose, with explicit Gaussian test matrices (Alg. 3 step 3):
 *   omegas     host array of d-1 device pointers; omegas[k] holds
 *              n_k x (r_k' + p) float32 values, row-major.
 * Used to give the GPU and a reference implementation identical Omega.
 */
TT_API tt_status tt_rbki_decompose_omega(const void* tensor, const int64_t* dims, int d,
                                  const int64_t* ranks, int oversample, int q,
                                  const float* const* omegas, float* const* cores_out,
                                  int64_t* ranks_out, void* workspace, size_t ws_bytes,
                                  void* stream, const tt_options* opts);

/*
 * Reads the device status word of the last decomposition that used
 * `workspace` (synchronises `stream`).  *device_status receives TT_OK,
 * TT_ENONFINITE, TT_EBREAKDOWN or TT_ETIMEOUT.
 */
TT_API tt_status tt_rbki_device_status(const void* workspace, void* stream, int* device_status);

/* Message describing the last error returned on the calling thread. */
TT_API const char* tt_rbki_last_error(void);

/* ------------------------------------------------------------------------
 * Batched form.  The paper decomposes one tensor per call; this runs many
 * independent TT-rBKI problems (Alg. 3 each, Omega from each problem's
 * seed) of uneven order, mode sizes and ranks in one call.  Problems are
 * spread over opts->batch_streams concurrent worker streams (longest
 * estimated cost first, each to the least-loaded worker) forked from and
 * joined back to `stream`, so that the small-algebra kernels of different
 * problems, which each occupy only a few SMs, run side by side.  Problems on
 * the same worker run one after another and share that worker's part of
 * the workspace.  The result of every problem is bit-identical to
 * tt_rbki_decompose of that problem alone with the same options.
 * ---------------------------------------------------------------------- */
typedef struct {
  const void* tensor;        /* device, prod(dims) elements of opts->storage,
                                row-major                                      */
  const int64_t* dims;       /* host, d mode sizes (read during the call only) */
  const int64_t* ranks;      /* host, d-1 target ranks                         */
  float* const* cores_out;   /* host array of d device pointers, as in
                                tt_rbki_decompose                              */
  int64_t* ranks_out;        /* host, d+1 entries, or NULL                     */
  uint64_t omega_seed;       /* seed of this problem's Omega_k                 */
  int32_t d;                 /* order, 2..64                                   */
  int32_t oversample;        /* p >= 0                                         */
  int32_t q;                 /* Krylov depth >= 0                              */
  int32_t reserved;          /* must be zero                                   */
} tt_problem;

/* Workspace bytes for tt_rbki_decompose_batched / _graph_create with these
 * problems and options (count status areas of 256 bytes plus one region per
 * worker, sized for the largest problem it runs). */
TT_API tt_status tt_rbki_batched_workspace_size(int count, const tt_problem* problems,
                                                const tt_options* opts, size_t* bytes);

/*
 * Enqueues all `count` problems on `stream` (fork/join over the library's
 * worker streams of the current device, created on first use and kept for
 * the life of the process).  Every problem is checked on the host first; if
 * any is invalid nothing is enqueued, per_problem[i] (host, count entries,
 * may be NULL) receives each problem's status and the first error is
 * returned.  The workspace (device, 256-byte aligned) must not be used by
 * another call until the stream has passed this one.
 * Errors: as tt_rbki_decompose, per problem; TT_EINVAL for count < 0 or
 * batch_streams outside [0, 64].
 */
TT_API tt_status tt_rbki_decompose_batched(int count, const tt_problem* problems, void* workspace,
                                           size_t ws_bytes, void* stream, const tt_options* opts,
                                           tt_status* per_problem);

/* Device status word of each problem of the last batch that used `workspace`
 * (synchronises `stream`): device_status[i] receives TT_OK, TT_ENONFINITE,
 * TT_EBREAKDOWN or TT_ETIMEOUT for problem i. */
TT_API tt_status tt_rbki_batched_device_status(const void* workspace, int count, void* stream,
                                               int* device_status);

/*
 * The same batch captured once into an executable CUDA graph, so that the
 * whole batch is one cudaGraphLaunch.  The graph records the device
 * pointers of the problems and the workspace: launch it again after
 * refilling the same input buffers.  Creating it enqueues no work; it is
 * the one entry point that allocates (the executable graph, inside CUDA).
 * Release it with tt_rbki_graph_destroy once no launch of it is pending.
 */
typedef struct tt_graph_t* tt_graph;
TT_API tt_status tt_rbki_batched_graph_create(int count, const tt_problem* problems, void* workspace,
                                              size_t ws_bytes, const tt_options* opts,
                                              tt_status* per_problem, tt_graph* graph);
TT_API tt_status tt_rbki_graph_launch(tt_graph graph, void* stream);
TT_API tt_status tt_rbki_graph_destroy(tt_graph graph);

/* ------------------------------------------------------------------------
 * Step-level entry points.  Each runs one kernel family of the path on
 * caller-owned device buffers; tests use them to check kernels one by one.
 * ---------------------------------------------------------------------- */

/*
 * Canonicalise a strided tensor into a dense row-major one, optionally
 * permuting modes and converting FP32 -> BF16 (round-to-nearest-even).
 * The free unfolding of Alg. 3 step 2 and Def. 1 needs i_1 slowest; the
 * paper permutes the modes of its colour video before decomposing (Sec. 4.1).
 *   src        device, elements of src_dtype at offsets sum_j i_j src_strides[j]
 *              (strides in elements, >= 0), for the SOURCE mode order.
 *   dims       host, d source mode sizes.
 *   perm       host, d entries: destination mode j is source mode perm[j]
 *              (NULL = identity).
 *   dst        device, prod(dims) elements of dst_dtype, dense row-major in
 *              the destination order.  Must not overlap src.
 * Conversions: F32->F32, F32->BF16, BF16->BF16, BF16->F32.  d <= 8.
 */
TT_API tt_status tt_permute_convert(const void* src, int src_dtype, const int64_t* dims,
                             const int64_t* src_strides, const int* perm, int d,
                             void* dst, int dst_dtype, void* stream);

/*
 * Gaussian test matrix of mode k from a seed (Alg. 3 step 3), with the
 * Philox4x32-10 / Box-Muller definition given at tt_rbki_decompose.
 *   out        device, n x b values of out_dtype (TT_F32 or TT_BF16),
 *              row-major with row stride ld >= b.
 */
TT_API tt_status tt_omega_generate(uint64_t seed, int mode, int64_t n, int b, void* out,
                            int out_dtype, int64_t ld, void* stream);

/*
 * One streaming pass over an unfolding C (m x n, row-major, dtype c_dtype).
 *   op = TT_PASS_SKETCH   : Y = C W          W = x: n x b FP32 (device)
 *   op = TT_PASS_GRAMAPPLY: Y = C (C^T X)    X = x: m x b FP32 (device)
 *   op = TT_PASS_PROJECT  : Y = X^T C        X = x: m x b FP32; Y is b x n,
 *                                            written in y_dtype (F32/BF16)
 *   op = TT_PASS_GRAM     : Y = C C^T        x unused; Y is m x m, m <= 2048
 * For SKETCH/GRAMAPPLY/GRAM, y is m x b (m x m) FP32.  The pass needs the
 * workspace size returned by tt_pass_workspace_size for the same arguments.
 * These are Alg. 3 steps 4 (sketch and Krylov powers), 10 (projection) and
 * the Gram formed at exhaustion or for the Gram-power route.
 */
enum { TT_PASS_SKETCH = 0, TT_PASS_GRAMAPPLY = 1, TT_PASS_PROJECT = 2, TT_PASS_GRAM = 3 };

TT_API tt_status tt_pass_workspace_size(int op, int64_t m, int64_t n, int b, int c_dtype,
                                 size_t* bytes);
TT_API tt_status tt_pass(int op, const void* C, int c_dtype, int64_t m, int64_t n, int b,
                  const float* x, void* y, int y_dtype, void* workspace, size_t ws_bytes,
                  void* stream);

/*
 * Tuning table of the BF16 tensor-core passes' launch shapes (the passes of
 * Alg. 3 steps 3, 4 and 10 and the exhaustion / Gram-power Gram).  Host-only
 * calls; process-wide state guarded by a lock.  An entry changes only how a
 * pass is launched, never what it computes (results differ at most by the
 * order of FP32 partial sums), and never the workspace sizes.
 *
 * Key:   op     TT_PASS_* of the pass;
 *        rows   row bucket of the unfolding: m rounded up to a multiple of
 *               16 for m <= 128, else 256, 512, 1024 or 4096 (m > 1024);
 *               the Gram takes rows <= 128 only;
 *        npad   the MMA width: b rounded up to a multiple of 16 (the Gram:
 *               m rounded; the projection at b <= 32 splits X into BF16
 *               high and low parts and has npad = 64);
 *        nclass 0 for n < 16,384 columns, 1 for n < 262,144, else 2.
 * Entry: stages     ring depth cap, 2..8;
 *        per_sm     CTAs per SM wanted, 1 or 2 (2 is taken only where three
 *                   stages fit half of the shared memory);
 *        kb         the Gram: 64-column boxes per stage, 1, 2, 4 or 8; else 0;
 *        chunk_rows the projection of unfoldings taller than 128 rows: rows
 *                   per streamed chunk, 64 or 128, or 0 for the built-in
 *                   rule; else 0.
 * An entry whose ring would keep fewer than two stages is ignored where it
 * applies (the built-in rules then hold).  tt_tune_set / tt_tune_get return
 * TT_EINVAL on an invalid key or entry (get: also on a missing key).
 * tt_tune_load replaces the whole table from a text file, one entry per
 * line: "op rows npad nclass stages per_sm kb chunk_rows", further text on
 * the line ignored, '#' lines and blank lines skipped; on a missing file or
 * any bad line it returns TT_EINVAL and leaves the table unchanged.
 */
TT_API tt_status tt_tune_set(int op, int rows, int npad, int nclass, int stages, int per_sm, int kb,
                             int chunk_rows);
TT_API tt_status tt_tune_get(int op, int rows, int npad, int nclass, int* entry4);
TT_API tt_status tt_tune_clear(void);
TT_API int tt_tune_entries(void);
TT_API tt_status tt_tune_load(const char* path);

/*
 * One Krylov power through a formed Gram matrix (Alg. 3 step 4 on the
 * Gram-power route): W = G X.
 *   G      device, m x m float32 row-major, symmetric (G = C C^T).
 *   X      device, m x c float32, 16-byte aligned, row stride ldx a
 *          multiple of 4 with ldx >= c rounded up to 4 (columns past c are
 *          read but do not affect W); 1 <= c <= 64.
 *   W      device, m x c float32, row stride ldw >= c, written; must not
 *          overlap X or G.
 * FP32 products with FP32 accumulation in a fixed order (bit-reproducible).
 * Allocates nothing.  Errors: TT_EINVAL (including a misaligned X),
 * TT_EUNSUPPORTED (c > 64), TT_ECUDA.
 */
TT_API tt_status tt_gram_power(const float* G, int64_t m, const float* X, int64_t ldx, int c, float* W,
                               int64_t ldw, void* stream);

/*
 * Top-r eigenpairs of a small symmetric matrix: the Rayleigh-Ritz step of
 * Alg. 3 (steps 6-8) takes the r largest eigenpairs of H = Q^T C C^T Q.
 *   H       device, k x k float32, row stride ldh >= k; only (H + H^T)/2 is
 *           used.  1 <= r <= k <= 224.
 *   V       device, k x r float32 row-major: eigenvectors as columns, in
 *           descending eigenvalue order, orthonormal.
 *   evals   device, r float32 eigenvalues, descending (may be NULL).
 *   workspace / ws_bytes: device scratch of tt_sym_eig_workspace_size bytes.
 * Errors: TT_EINVAL, TT_EUNSUPPORTED (k > 224), TT_ENOMEM, TT_ECUDA.
 */
TT_API tt_status tt_sym_eig_workspace_size(int k, int r, size_t* bytes);
TT_API tt_status tt_sym_eig_top(const float* H, int64_t ldh, int k, int r, float* V, float* evals,
                                void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * TT-SVD (Alg. 1, Sec. 2.2): the deterministic baseline, sequential
 * truncated SVDs of the unfoldings with prescribed accuracy.
 *
 * delta = eps * ||A||_F / sqrt(d - 1) (Alg. 1 step 1).  At mode k the
 * unfolding C (m = r_{k-1} I_k rows, n = I_{k+1} ... I_d columns) has the
 * Gram G = C C^T, whose eigenvalues are the squared singular values of C;
 * r_k is the smallest rank whose discarded tail sum_{i > r_k} lambda_i is
 * at most delta^2 (Alg. 1 step 4), capped by max_ranks[k] and min(m, n);
 * core k is the top r_k eigenvectors of G (the left singular vectors), and
 * the next remainder is U^T C = S V^T (Alg. 1 step 6).  ||A||_F^2 is the
 * trace of the first Gram.  eps = 0 with max_ranks gives the fixed-rank
 * form.
 *
 *   tensor    device, row-major (i_1 slowest), dtype storage (TT_F32 or
 *             TT_BF16); converted to FP64 once, remainders are FP64.
 *   dims, d   mode sizes, d >= 2.
 *   eps       >= 0.
 *   max_ranks host, d - 1 rank caps >= 1, or NULL for none (min(m, n)).
 *   cores_out d device FP32 buffers, core k sized for the clamped caps
 *             (tt_svd_workspace_size reports them through core_elems);
 *             written as [r_{k-1}][I_k][r_k] with the chosen ranks.
 *   ranks_out host, d + 1 chosen ranks (r_0 = r_d = 1).
 * Host-synchronous: the call waits on `stream` once per mode to read the
 * eigenvalues back and returns when the cores are written; it cannot be
 * captured in a CUDA graph.  The Gram matrices and the projections are
 * cuBLAS DGEMMs and the eigendecompositions cuSOLVER's Dsyevd, in FP64
 * (the Gram squares the singular values, which FP32 could not resolve for
 * fast-decaying spectra); cores are returned in FP32.  The workspace holds
 * the FP64 copy of the tensor.  One cuBLAS and one cuSOLVER handle per
 * host thread and device are created on first use.  Errors: TT_EINVAL,
 * TT_ENOMEM (workspace too small), TT_EUNSUPPORTED (a Gram larger than
 * 16384 x 16384, more than 2^31 - 1 columns), TT_ECUDA.
 * ---------------------------------------------------------------------- */
TT_API tt_status tt_svd_workspace_size(const int64_t* dims, int d, const int64_t* max_ranks, int storage,
                                       int64_t* core_elems, size_t* bytes);
TT_API tt_status tt_svd_decompose(const void* tensor, int storage, const int64_t* dims, int d, double eps,
                                  const int64_t* max_ranks, float* const* cores_out, int64_t* ranks_out,
                                  void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free Gram-apply.  The paper has no counterpart: this entry
 * point exists for deployment, not for the method.
 *
 * Computes Y = C (C^T X) exactly like tt_pass(TT_PASS_GRAMAPPLY, ...) but
 * takes no workspace.  It is meant for callers that cannot allocate device
 * memory at the point of the call: code running inside another framework's
 * stream capture or memory pool, latency-critical loops in which cudaMalloc
 * would synchronise the device, or plugins whose host application owns all
 * device memory.  The per-CTA partial sums go to one fixed array of 16 MiB
 * (4,194,304 floats) in the library's device image, so every GPU on which
 * the library is loaded holds those 16 MiB until the process exits.
 *   C      device, m x n row-major, c_dtype TT_F32 or TT_BF16.
 *   x      device, m x b float32 row-major.
 *   y      device, m x b float32 row-major, written.
 * Limits: 1 <= m <= 256 and 1 <= b <= 48, else TT_EUNSUPPORTED.  The pass
 * runs at most 4,194,304 / (m b) CTAs so their partials fit the array.
 * The first call on a device looks up the array's device address on the
 * current device; make that first call before any stream capture.  All
 * calls share the array; each call overwrites the part it reads, so nothing
 * needs clearing, but calls whose kernels overlap on the GPU (several
 * streams, or several host threads at once) race on it and give wrong
 * results.  Allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine.  Errors: TT_EINVAL (NULL pointer, dtype, size < 1),
 * TT_EUNSUPPORTED, TT_ECUDA; the message is in tt_rbki_last_error().
 */
TT_API tt_status tt_gram_apply_noalloc(const void* C, int c_dtype, int64_t m, int64_t n, int b,
                                       const float* x, float* y, void* stream);

/* ------------------------------------------------------------------------
 * Test aid (no counterpart in the paper).  Fills the shared memory of every
 * SM with the 32-bit pattern `bits` (e.g. a NaN) by launching maximal CTAs
 * on `stream`, so that a kernel launched afterwards which reads shared
 * memory it never wrote sees that pattern.  Used by the tests in place of
 * a memory-checking tool.  Errors: TT_ECUDA.
 * ---------------------------------------------------------------------- */
TT_API tt_status tt_debug_fill_shared(uint32_t bits, void* stream);

/* Test aid: runs, on `stream`, one wait of the kind every tensor-core kernel
 * uses (an mbarrier wait bounded at about two seconds) on a barrier that
 * nothing ever completes, so the wait gives up and records TT_ETIMEOUT in
 * the 256-byte status area at `workspace` (device; read it back with
 * tt_rbki_device_status).  Exercises the timeout path without a fault; the
 * context stays usable.  Errors: TT_EINVAL, TT_ECUDA. */
TT_API tt_status tt_debug_wait_timeout(void* workspace, void* stream);

/* ------------------------------------------------------------------------
 * Sharded form: one problem split over `world` ranks (one GPU each) by its
 * last mode.  Rank g holds the slab A[..., lo_g : lo_g + w_g] of the last
 * index (slab g = [ceil(g I_d / world), ceil((g + 1) I_d / world))), so
 * every unfolding C_k of Alg. 3 splits by columns (the last index is the
 * fastest part of every column index) and each rank streams only its own
 * columns.  The sketch Y = C Omega (Alg. 3 step 4, first block), each
 * streamed Krylov power C C^T X (step 4) and, on the Gram routes, the Gram
 * C C^T are sums over the ranks of the ranks' partial products; the block
 * orthonormalisation, Rayleigh-Ritz and the cores 1..d-1 then run
 * replicated on the summed blocks, and the projection U^T C_k (step 10)
 * stays on its rank as its slab of the next unfolding.  The last core is
 * returned as this rank's slab (r_{d-1} x w_g); the caller gathers it.
 * The column-Gram exhaustion route, paper_literal and accurate_rr are not
 * available in this form.  The paper runs on one machine and has no
 * counterpart.
 * ---------------------------------------------------------------------- */

/* Sums `count` floats at device address `buf` over all ranks, in place.
 * Called on the host in stream order: the library has enqueued the kernels
 * that produce buf on `stream` (a cudaStream_t) and enqueues its next
 * kernels after the call returns; the sum must be visible to work enqueued
 * on `stream` afterwards (e.g. ncclAllReduce on that stream, or a stream
 * synchronisation, a host exchange and a copy back).  Every rank must
 * obtain bit-identical sums (the replicated steps rely on it).  Returns 0
 * on success; anything else aborts the decomposition with TT_ECUDA. */
typedef int32_t (*tt_allreduce_fn)(float* buf, int64_t count, void* stream, void* ctx);

typedef struct {
  int64_t m;             /* rows of the unfolding C_k                           */
  int64_t n_global;      /* columns of the whole unfolding                      */
  int64_t n_local;       /* this rank's columns (n_global / I_d * w)            */
  int32_t route;         /* TT_ROUTE_* (never TT_ROUTE_GRAM_COLS)               */
  int32_t allreduces;    /* calls of the sum callback in this mode              */
  int64_t allreduce_floats;  /* floats summed in this mode, all calls           */
} tt_shard_mode;

/* The host-side plan of rank `rank` of `world`: its slab of the last mode
 * (*slab_lo, *slab_w) and, per mode k = 1..d-1, the entry modes[k-1].  Pure
 * host computation (no device, no stream).  Errors: TT_EINVAL (bad
 * arguments, world > I_d, NULL outputs, max_modes < d-1), TT_EUNSUPPORTED
 * (options outside the sharded form), and those of tt_rbki_workspace_size. */
TT_API tt_status tt_rbki_shard_plan(const int64_t* dims, int d, const int64_t* ranks, int oversample, int q,
                                    const tt_options* opts, int32_t world, int32_t rank, int64_t* slab_lo,
                                    int64_t* slab_w, tt_shard_mode* modes, int max_modes);

/* Workspace bytes of tt_rbki_decompose_sharded for this rank. */
TT_API tt_status tt_rbki_sharded_workspace_size(const int64_t* dims, int d, const int64_t* ranks,
                                                int oversample, int q, const tt_options* opts, int32_t world,
                                                int32_t rank, size_t* bytes);

/* Alg. 3 (or Alg. 4 with opts->method) on this rank's slab.
 *   local_tensor  device, the slab A[..., lo : lo + w] row-major
 *                 (I_1 x ... x I_{d-1} x w elements of opts->storage).
 *   dims, ranks   the whole problem's sizes (host), as tt_rbki_decompose.
 *   omega_seed    seed of the whole problem's Omega_k; each rank draws the
 *                 rows of its own columns, identical to the single-GPU draw.
 *   cores_out     d device pointers: cores 1..d-1 in full (replicated),
 *                 core d as this rank's slab (r_{d-1} x w floats).
 *   allreduce, ctx the sum callback (above) and its argument.
 * Orders the work on `stream`; the sum callback is called from this call.
 * Errors: as tt_rbki_decompose, TT_EINVAL for a NULL allreduce with
 * world > 1, TT_ECUDA when the callback fails. */
TT_API tt_status tt_rbki_decompose_sharded(const void* local_tensor, const int64_t* dims, int d,
                                           const int64_t* ranks, int oversample, int q, uint64_t omega_seed,
                                           float* const* cores_out, int64_t* ranks_out, void* workspace,
                                           size_t workspace_bytes, int32_t world, int32_t rank,
                                           tt_allreduce_fn allreduce, void* ctx, void* stream,
                                           const tt_options* opts);

/* ------------------------------------------------------------------------
 * Kernel accounting for benchmarks (no counterpart in the paper).
 * Between tt_rbki_profile_begin and tt_rbki_profile_end every kernel launch
 * of the library is counted per kernel family; with event_timing = 1 each
 * launch of a family is also bracketed by CUDA events on its stream, and
 * the family's algorithmic bytes and flops are summed.  Process-global;
 * tt_rbki_profile_end synchronises the recorded events.
 * ---------------------------------------------------------------------- */
typedef struct {
  char name[32];        /* kernel family                                       */
  int64_t launches;     /* kernel launches                                     */
  double ms;            /* summed event durations (0 without event timing)     */
  double bytes;         /* summed algorithmic HBM bytes                        */
  double flops;         /* summed algorithmic flops                            */
} tt_kernel_stat;

TT_API tt_status tt_rbki_profile_begin(int event_timing);
TT_API tt_status tt_rbki_profile_end(tt_kernel_stat* stats, int max_stats, int* n_stats);

#ifdef __cplusplus
}
#endif

#endif /* TT_RBKI_H */
