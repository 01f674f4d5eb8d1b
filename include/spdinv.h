/*
 * spdinv -- inversion of symmetric positive definite matrices on GB300
 * (sm_103a) as the three tiled steps of Agullo, Bouwmeester, Dongarra,
 * Kurzak, Langou and Rosenberg, "Towards an Efficient Tile Matrix Inversion
 * of Symmetric Positive Definite Matrices on Multicore Architectures"
 * (Sec. 2, Algorithm 1):
 *
 *   Step 1  tile Cholesky factorisation       A = L L^T      (POTRF, TRSM, SYRK, GEMM)
 *   Step 2  tile triangular inversion         X = L^{-1}     (TRTRI, TRMM, GEMM)
 *   Step 3  tile product of lower triangles   A^{-1} = X^T X (TRMM, LAUUM, GEMM, SYRK)
 *
 * The tile DAG runs as one persistent kernel: tile readiness is tracked by
 * device-side dependency counters, the write-after-read hazards of Sec. 3
 * ("array renaming") are removed by renamed temporaries, and the three steps
 * are overlapped ("pipelining", Sec. 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major with leading dimension lda >= max(1, n);
 *    element (i, j) is at A[i + j*lda].  Only the lower triangle (i >= j) is
 *    read or written; the strictly upper part is never touched.
 *  - Device pointers must point to device memory of the current CUDA device.
 *    The caller owns every pointer it passes; the library keeps none after
 *    the call returns except inside the work queued on `stream`.
 *  - Every call is asynchronous on `stream` (0 = legacy default stream).
 *    Argument errors are returned synchronously and nothing is launched.
 *  - d_info (nullable) is a device int written when the queued work ends:
 *      0   success;
 *      k>0 the leading minor of order k is not positive definite (POTRF,
 *          POTRI: the pivot of global column k-1 was <= 0 or NaN), or the
 *          diagonal entry k-1 of the triangular factor is exactly zero
 *          (TRTRI);
 *      <0  a device-side failure with the value of an spdinv_status below
 *          (SPDINV_ERR_TIMEOUT: a dependency wait ran past its limit; all
 *          CTAs stopped and the kernel returned).
 *    After k>0 or k<0 the contents of the lower triangle are unspecified,
 *    except for TRTRI with k>0, which leaves A unchanged (LAPACK dtrtri).
 *  - n == 0 returns SPDINV_OK at once and writes 0 to d_info.
 *  - The library keeps a per-device workspace (the renamed temporaries and
 *    the dependency counters, about n*n + n*b elements) and a plan cache;
 *    both grow on demand with cudaMalloc.  A call made for the first time
 *    with a given size may therefore allocate and must come before any CUDA
 *    graph capture that later replays the same size.  The single-matrix
 *    calls can use a caller's buffer instead (spdinv_workspace_size,
 *    spdinv_set_workspace).
 *  - Calls on different streams of the same device share that workspace and
 *    must not overlap in time; calls on one stream are ordered by the stream.
 *  - Environment (read once per process):
 *      SPDINV_LOG=1       each call that returns an error status prints one
 *                         line to stderr (name, size, status, CUDA error
 *                         text); =2 every call.  Device-side results
 *                         (d_info) are not known at return and not logged.
 *      SPDINV_TILE=32|64  the default tile of the FP64 single-matrix calls.
 *      SPDINV_WAIT_TIMEOUT_S  the default limit of one dependency wait (60 s).
 *      SPDINV_BATCHED_TILE=16|32|64  one tile for every batched size class.
 *      SPDINV_PLAN_ORDER=bottom_level (or 0)  the bottom-level ticket order
 *                         instead of the default ALAP order (see
 *                         spdinv_set_plan_order).
 *      SPDINV_SLICE_TILE=128  the 128 x 128 slice GEMM instead of the
 *                         default 128 x 256 one (emulated residual).
 *      SPDINV_DEBUG       initial debug flags (spdinv_set_debug_flags).
 */
#ifndef SPDINV_H
#define SPDINV_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define SPDINV_API __attribute__((visibility("default")))
#else
#define SPDINV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPDINV_OK = 0,
    SPDINV_ERR_N = -1,            /* n < 0, or n beyond the supported maximum */
    SPDINV_ERR_LDA = -2,          /* lda < max(1, n) */
    SPDINV_ERR_NULL = -3,         /* a required pointer is NULL */
    SPDINV_ERR_CUDA = -4,         /* a CUDA runtime call failed (see spdinv_last_cuda_error) */
    SPDINV_ERR_TIMEOUT = -5,      /* device-side: a dependency wait exceeded its limit */
    SPDINV_ERR_UNSUPPORTED = -6,  /* an option value this library does not implement */
    SPDINV_ERR_WORKSPACE = -7     /* a caller-provided buffer is too small, misaligned or not
                                     device memory of the current device */
} spdinv_status;

/* Precision of the bulk tile updates (GEMM/SYRK/TRMM). */
typedef enum {
    SPDINV_PREC_FP64 = 0,         /* every operation in native FP64 (FMA on the FP64 pipe) */
    SPDINV_PREC_MIXED_FP32 = 1,   /* bulk updates FP32 (FMA on the CUDA cores); diagonal POTRF/TRTRI
                                     FP32 (FP64 with spdinv_opts.diag_fp64); the residual FP64 */
    SPDINV_PREC_MIXED_BF16X3 = 2, /* as MIXED_FP32, the bulk updates on the BF16 tensor cores as three
                                     products of two-term BF16 splits (hi hi + hi lo + lo hi, FP32
                                     accumulation): about 2^-16 relative per product */
    SPDINV_PREC_MIXED_TF32X3 = 3  /* as MIXED_FP32, the bulk updates on the TF32 tensor cores as three
                                     products of two-term TF32 splits (3xTF32, FP32 accumulation):
                                     about 2^-21 relative per product, near FP32 */
} spdinv_precision;

/* Options for spdinv_potri_ex.  Zero-initialise and set what you need. */
typedef struct {
    int tile;            /* tile order b, 32, 64 or (FP64 potri only) 128; 0 = automatic (FP64: 32
                            up to n = 16384, 64 above; mixed precision: 32 up to n = 8192, 64 above) */
    int ctas_per_sm;     /* resident CTAs per SM of the persistent kernel; 0 = automatic */
    int precision;       /* spdinv_precision */
    int refine_steps;    /* mixed precision only: residual corrections X <- X + X(I - A X); 0 = none */
    double wait_timeout_s; /* limit for one dependency wait; 0 = default (60 s) */
    int fault_drop_task; /* failure-detection test hook: when >= 0, the task with this ticket
                            never signals completion, so its consumers hit the wait limit and
                            the call ends with d_info = SPDINV_ERR_TIMEOUT; -1 (or any value
                            below 0) = off.  Only honoured when wait_timeout_s > 0. */
    int residual;        /* mixed precision: how R = I - A X is formed.
                            SPDINV_RESIDUAL_EMULATED (0, default): FP64-accurate products of
                            exact 8-bit slices on the BF16 tensor cores (tcgen05, TMA);
                            SPDINV_RESIDUAL_FP64 (1): native FP64 tensor-core products;
                            SPDINV_RESIDUAL_EMULATED_MMA_SYNC (2): the slice products on the
                            warp-level mma.sync tensor-core path (for comparison). */
    int refine_order;    /* mixed precision: order p of each correction,
                            X <- X (I + R + R^2 + ... + R^{p-1}) with R = I - A X, whose new
                            residual is R^p; 0 = 2 (Newton-Schulz).  2..8; p > 2 needs
                            residual = SPDINV_RESIDUAL_EMULATED. */
    int variant;         /* FP64 spdinv_potri_ex only: an execution variant of Sec. 3's study
                            (SPDINV_VARIANT_* ORed; 0 = renamed and pipelined, the default).
                            The result is the same up to rounding (the integer test case:
                            bit for bit); the variants differ in memory and critical path. */
    int split_segment;   /* SPDINV_VARIANT_SPLIT3: chain segment length in tiles (0 = 16) */
    int diag_fp64;       /* mixed precision only: precision of the FP32 tile DAG's diagonal-tile
                            POTRF and TRTRI.  0 (default): FP32 (warp-level register sweeps for
                            32-tiles, block-wide sweeps for 64-tiles); 1: native FP64 (the tile
                            converted to FP64, block-wide sweeps, X_jj rounded back to FP32 for
                            the bulk products).  Any other value: SPDINV_ERR_UNSUPPORTED.  The
                            corrected result's accuracy is the same either way; FP64 sweeps
                            lengthen the DAG's critical path. */
} spdinv_opts;

/* Execution variants (spdinv_opts.variant), for the study of Sec. 3 on the GPU:
 *   SPDINV_VARIANT_UUU       Step 2's update chains in increasing k ("loop
 *                            reversal" undone: U, U, U instead of U, D, U).
 *   SPDINV_VARIANT_SHARE_BC  the copy of L^{-1} shares the storage of the copy of
 *                            L (Sec. 4, renaming under a memory budget): X_ij is
 *                            stored over L_ij once every task that reads L_ij has
 *                            read it (write-after-read waits on read counters).
 *   SPDINV_VARIANT_INPLACE   no renaming: one store holds L, then X = L^{-1}, then
 *                            A^{-1}, tile by tile, each version stored once all
 *                            readers of the previous one have read it; the lower
 *                            triangle of A receives A^{-1} at the end.
 *   SPDINV_VARIANT_SPLIT3    Step 3's chains of more than split_segment products
 *                            split into segments whose partial sums other CTAs
 *                            form in parallel; the tile's own task adds them
 *                            (the associative reduction of Sec. 4).
 * SPLIT3 does not combine with SHARE_BC or INPLACE (SPDINV_ERR_UNSUPPORTED). */
#define SPDINV_VARIANT_UUU 1
#define SPDINV_VARIANT_SHARE_BC 2
#define SPDINV_VARIANT_INPLACE 4
#define SPDINV_VARIANT_SPLIT3 8

#define SPDINV_RESIDUAL_EMULATED 0
#define SPDINV_RESIDUAL_FP64 1
#define SPDINV_RESIDUAL_EMULATED_MMA_SYNC 2

/* ------------------------------------------------------------------------
 * The three steps, separately (LAPACK lower-triangle semantics)
 * ------------------------------------------------------------------------ */

/* Step 1 (Algorithm 1, Step 1; Sec. 2): tile Cholesky factorisation.
 * On entry the lower triangle of A holds the SPD matrix; on exit it holds L
 * with A = L L^T (LAPACK dpotrf, uplo = 'L'). */
SPDINV_API spdinv_status spdinv_potrf(int64_t n, double* dA, int64_t lda, int* d_info, cudaStream_t stream);

/* Step 2 (Algorithm 1, Step 2; Sec. 2): inversion of a lower triangular,
 * non-unit matrix in place, X = L^{-1} (LAPACK dtrtri, uplo 'L', diag 'N').
 * d_info = k > 0 if L(k-1, k-1) == 0; A is then left unchanged. */
SPDINV_API spdinv_status spdinv_trtri(int64_t n, double* dA, int64_t lda, int* d_info, cudaStream_t stream);

/* Step 3 (Algorithm 1, Step 3; Sec. 2): lower triangle of X^T X for a lower
 * triangular X, in place (LAPACK dlauum, uplo 'L'). */
SPDINV_API spdinv_status spdinv_lauum(int64_t n, double* dA, int64_t lda, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * The whole inversion
 * ------------------------------------------------------------------------ */

/* Steps 1-3 pipelined in one persistent launch (Algorithm 1 with the
 * renaming and pipelining of Sec. 3): the lower triangle of A is replaced by
 * the lower triangle of A^{-1}.  Note: unlike LAPACK dpotri, which takes the
 * Cholesky factor, this takes A itself; spdinv_trtri followed by
 * spdinv_lauum gives dpotri's semantics on a factor. */
SPDINV_API spdinv_status spdinv_potri(int64_t n, double* dA, int64_t lda, int* d_info, cudaStream_t stream);

/* spdinv_potri with options (tile size, residency, precision, correction
 * steps and order, wait limit).  opts may be NULL (= all defaults).
 * Mixed precision (opts->precision == SPDINV_PREC_MIXED_FP32, tile 32 or 64):
 * the tile DAG runs with FP32 bulk updates and FP32 diagonal POTRF/TRTRI
 * (FP64 with opts->diag_fp64),
 * then refine_steps times R = I - A X (FP64-accurate; A read from its lower
 * triangle, intact until the end) and X <- X + X R + ... + X R^{p-1} (p =
 * refine_order; sums in FP64); the lower triangle of A then holds X in FP64.
 * opts->residual selects how the products are formed: by default from exact
 * BF16 slices on the tensor cores (R to FP64 accuracy, the terms X R^m to the
 * relative accuracy their size calls for), or R with native FP64 MMA and X R
 * in FP32 (p = 2 only).  A step of order p takes a residual R to about R^p,
 * so the FP32 result's error e (about 1e-5 at cond 1e2, 1e-3 at cond 1e4 for
 * n = 16384) falls to about e^p times a modest factor that grows with
 * cond(A): one step of order 3 reaches 1e-10 at cond 1e2, one of order 4 at
 * cond 1e4, two of order 3 at cond 1e6.  The workspace holds three n x n FP64
 * matrices when refine_steps > 0, plus 23 n^2 BF16 slices with the emulated
 * products. */
SPDINV_API spdinv_status spdinv_potri_ex(int64_t n, double* dA, int64_t lda, const spdinv_opts* opts,
                              int* d_info, cudaStream_t stream);

/* Selected inverse: the diagonal of A^{-1} (the variances in a
 * variance-covariance matrix A^{-1}, the use the paper's introduction names
 * for an explicit inverse; Sec. 1) without forming the rest
 * of A^{-1}.  Steps 1 and 2 run in full; of Step 3 only the diagonal tiles'
 * LAUUM + SYRK chains run (about n^2 b / 2 of its n^3 / 3 multiply-adds), all
 * in the same persistent launch.  dA: lower triangle of the SPD matrix
 * (column-major, lda >= n), only read.  d_diag: n doubles (device), receives
 * diag(A^{-1}).  d_info (nullable device int): 0, or k > 0 if the leading
 * minor of order k is not positive definite (d_diag is then unspecified).
 * Argument errors return synchronously and launch nothing. */
SPDINV_API spdinv_status spdinv_potri_diag(int64_t n, const double* dA, int64_t lda, double* d_diag, int* d_info,
                                           cudaStream_t stream);

/* Residual of an approximate inverse (used by the mixed-precision
 * correction; the paper has none): R = I - A X with A symmetric, given by the
 * lower triangle of dA (column-major, lda), X full n x n (leading dimension n)
 * and R full n x n (leading dimension n).  residual = SPDINV_RESIDUAL_EMULATED
 * forms the products from 7 exact 8-bit slices of each operand on the BF16
 * tensor cores, keeping the 34 slice products whose levels s + t are <= 7
 * (error about 1e-16 |A||X|, like the native residual;
 * SPDINV_RESIDUAL_EMULATED_MMA_SYNC the same on the
 * warp-level MMA); SPDINV_RESIDUAL_FP64 uses native FP64 MMA.
 * Uses the library workspace (may allocate on first use).  An unknown
 * `residual` returns SPDINV_ERR_UNSUPPORTED. */
SPDINV_API spdinv_status spdinv_inverse_residual(int64_t n, const double* dA, int64_t lda, const double* dX,
                                                 double* dR, int residual, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Inversion without device allocation (the paper has no counterpart)
 * ------------------------------------------------------------------------ */

/* Largest n spdinv_potri_noalloc accepts. */
#define SPDINV_NOALLOC_MAX_N 1024

/* spdinv_potri (FP64, tile 32) for callers that must not allocate device
 * memory.  Some callers cannot call cudaMalloc: plug-ins whose host
 * application owns all device memory through its own allocator or a fixed
 * budget, and latency-bound loops in which an allocation, which can
 * synchronise the whole device, would stall the work of other streams.  This
 * entry point allocates nothing: its scratch (status words, readiness flags,
 * the renamed tile stores and the task list, about 8 MiB) is one fixed array
 * in the library's device memory, which every GPU that loads the library
 * holds until the process exits.  The caller still passes A and d_info as for
 * spdinv_potri.
 *  - n > SPDINV_NOALLOC_MAX_N returns SPDINV_ERR_N and launches nothing.
 *  - The first call on a device (with that device current) looks up the
 *    array's device address, a host-side query of the loaded module.
 *    A device reset (cudaDeviceReset) ends the context the address belongs
 *    to: the first call in the new context looks it up again.
 *  - Every call uses the same array, which keeps the last call's contents
 *    (the call clears what must start at zero).  Calls whose GPU work
 *    overlaps in time -- on different streams, or from different threads --
 *    race on the array and give wrong results; order them on one stream.
 *  - The wait limit of the persistent kernel is spdinv_potri's default
 *    (SPDINV_WAIT_TIMEOUT_S, else 60 s). */
SPDINV_API spdinv_status spdinv_potri_noalloc(int64_t n, double* dA, int64_t lda, int* d_info,
                                              cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Caller-owned workspace (capture-safe use; the paper has no counterpart)
 * ------------------------------------------------------------------------ */

/* Routines for spdinv_workspace_size. */
#define SPDINV_ROUTINE_POTRI 0            /* spdinv_potri, spdinv_potri_ex (FP64 or mixed, per opts) */
#define SPDINV_ROUTINE_POTRF 1            /* spdinv_potrf */
#define SPDINV_ROUTINE_TRTRI 2            /* spdinv_trtri */
#define SPDINV_ROUTINE_LAUUM 3            /* spdinv_lauum */
#define SPDINV_ROUTINE_POTRI_DIAG 4       /* spdinv_potri_diag */
#define SPDINV_ROUTINE_INVERSE_RESIDUAL 5 /* spdinv_inverse_residual (opts->residual: its path) */

/* Bytes of device workspace one call of `routine` on an order-n matrix uses
 * (host only, no GPU needed).  opts (nullable) are those the call would get:
 * spdinv_potri_ex's options for SPDINV_ROUTINE_POTRI (tile, precision,
 * correction steps and path), and only `residual` for
 * SPDINV_ROUTINE_INVERSE_RESIDUAL; the other routines take none.  The same
 * argument checks as the call: an option the call would reject returns the
 * call's status.  n == 0 needs 0 bytes.  Layout, in order, each part on a
 * 256-byte boundary: FP64 -- status words and readiness flags
 * (4 + 2t^2 + t ints, t = ceil(n/b)), B and C (t(t-1)/2 b x b FP64 tiles each,
 * B absent for lauum and C for potrf), D (t tiles); mixed -- status words
 * and flags, B, C and D as FP32 b x (b+1) tiles, the FP64 n x n matrix X
 * (three of them with correction steps) and the BF16 slice planes. */
SPDINV_API spdinv_status spdinv_workspace_size(int64_t n, int routine, const spdinv_opts* opts, size_t* bytes);

/* Makes the single-matrix calls of the current device (potrf, trtri, lauum,
 * potri, potri_ex, potri_diag, inverse_residual) use the caller's device
 * buffer [d_ws, d_ws + bytes) as their workspace instead of the library's
 * own: they then allocate no workspace, and a call that needs more than
 * `bytes` (spdinv_workspace_size) returns SPDINV_ERR_WORKSPACE and launches
 * nothing.  d_ws must be 256-byte aligned device (or managed) memory of the
 * current device, else SPDINV_ERR_WORKSPACE.  d_ws == NULL returns to the
 * library's workspace.  The caller keeps ownership: the buffer must stay
 * valid until the work queued with it has finished, and calls whose work
 * overlaps in time must not share it.  The plan of each (size, tile,
 * routine) is still built, and uploaded with one allocation, by the first
 * call with it; later calls with a caller buffer allocate nothing and can be
 * captured in a CUDA graph.  The batched, backward and no-allocation calls
 * keep their own buffers. */
SPDINV_API spdinv_status spdinv_set_workspace(void* d_ws, size_t bytes);

/* ------------------------------------------------------------------------
 * Many independent matrices of uneven sizes in one persistent launch
 * ------------------------------------------------------------------------ */

/* Inverts batch matrices A_k (k < batch) in place, each with Algorithm 1's
 * three steps, in ONE kernel launch: CTAs take matrices from a device queue
 * ordered by decreasing n (largest first), and each matrix runs the tile
 * algorithm with the tile shape the autotuner chose for its size class.
 *   h_n[k], h_lda[k]  host arrays: order and leading dimension of A_k
 *                     (0 <= h_n[k] <= 4096, h_lda[k] >= max(1, h_n[k]));
 *   d_Aptrs           device array of batch device pointers;
 *   d_info            device int[batch] (nullable): per-matrix info as above.
 * The per-size plan (queue order, tile choice) is cached by the exact size
 * list.  The first call with a size list builds it: it takes the per-class
 * table of spdinv_batched_tiles capped at each tile size (one kernel holds
 * the largest tile any matrix uses, which sets the occupancy of all), times
 * each capped table on a synthetic batch of the same sizes (skipped above
 * 2 GiB), keeps the fastest and uploads it; this call allocates and
 * synchronises.  A later call with the same list queues only the kernel
 * launch and can be captured in a CUDA graph.  Plans stay cached for the
 * life of the process (16 bytes of device memory and 8 bytes of host memory
 * per matrix), since a captured graph may still use them: a caller with
 * ever-changing size lists should pad them to a few fixed lists. */
SPDINV_API spdinv_status spdinv_potri_batched(int batch, const int* h_n, double* const* d_Aptrs,
                                   const int* h_lda, int* d_info, cudaStream_t stream);

/* FP32 twin of spdinv_potri_batched (float data, FP32 arithmetic). */
SPDINV_API spdinv_status spdinv_spotri_batched(int batch, const int* h_n, float* const* d_Aptrs,
                                    const int* h_lda, int* d_info, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Differentiation (added form: backward of X = A^{-1})
 * ------------------------------------------------------------------------ */

/* grad_A = -sym(X G X) = -(X G X + (X G X)^T) / 2 for `batch` matrices of
 * order n, from the saved inverse X (full symmetric, column-major, ldx) and
 * the incoming gradient G (full, ldg).  Writes the full symmetric grad_A
 * (ldgrad).  Matrix k starts at element offset k*stride_* of each pointer.
 * X, G and grad_A must not overlap.  0 <= batch <= 65535 (else SPDINV_ERR_N);
 * the library workspace holds 2 batch n^2 elements (Y = X G and sym(G)). */
SPDINV_API spdinv_status spdinv_potri_backward(int batch, int64_t n, const double* dX, int64_t ldx, int64_t stride_x,
                                    const double* dG, int64_t ldg, int64_t stride_g,
                                    double* dGrad, int64_t ldgrad, int64_t stride_grad,
                                    cudaStream_t stream);

/* FP32 twin of spdinv_potri_backward, on the tensor cores: each product is a
 * sum of three TF32 products of split operands (3xTF32: x = hi + lo, hi the
 * TF32 rounding of x), FP32 accumulation; close to FP32 accuracy.  The
 * library workspace holds 6 batch npad^2 floats, npad = n rounded up to 128
 * (hi and lo planes of X, sym(G) and Y). */
SPDINV_API spdinv_status spdinv_spotri_backward(int batch, int64_t n, const float* dX, int64_t ldx, int64_t stride_x,
                                     const float* dG, int64_t ldg, int64_t stride_g,
                                     float* dGrad, int64_t ldgrad, int64_t stride_grad,
                                     cudaStream_t stream);

/* Split of a batch across `world` GPUs (one process per GPU; no counterpart
 * in the paper, whose unit of work is one matrix).  The matrices are
 * independent, so a multi-GPU batch needs no collective: rank r inverts the
 * matrices with owner[k] == r through spdinv_potri_batched.  The split
 * balances the work (n^3 per matrix) by longest processing time first:
 * matrices by decreasing n, each to the rank with the least total so far,
 * ties to the lower index and the lower rank; every rank's total is within
 * 4/3 of the best possible split.  Deterministic and host-only (no GPU).
 *   h_n[batch]     host: orders of the matrices (>= 0);
 *   owner[batch]   host, out: rank in [0, world) of each matrix;
 *   load[world]    host, out (nullable): each rank's total n^3. */
SPDINV_API spdinv_status spdinv_batch_shard(int batch, const int* h_n, int world, int* owner, double* load);

/* The autotuner's tile choice for spdinv_potri_batched (fp32 == 0) or
 * spdinv_spotri_batched (fp32 != 0): tiles[c] is the tile order used for
 * matrices with 32c < n <= 32(c+1) (c = 7 also for n > 256).  The first call
 * per device and precision times every candidate tile on synthetic batches
 * (this allocates, synchronises, and must come before any graph capture);
 * SPDINV_BATCHED_TILE=16|32|64 in the environment forces one tile. */
SPDINV_API spdinv_status spdinv_batched_tiles(int fp32, int tiles[8]);

/* Copies the lower triangle of `batch` column-major n x n matrices onto their
 * strictly upper triangle (A_ij = A_ji, i < j); matrix k starts at element
 * k*stride.  Used to form the full symmetric A^{-1} (no counterpart in the
 * paper, whose result is the lower triangle).  0 <= batch <= 65535 (else
 * SPDINV_ERR_N). */
SPDINV_API spdinv_status spdinv_mirror_lower(int batch, int64_t n, double* dA, int64_t lda, int64_t stride,
                                             cudaStream_t stream);
SPDINV_API spdinv_status spdinv_smirror_lower(int batch, int64_t n, float* dA, int64_t lda, int64_t stride,
                                              cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Host-side planner queries (no GPU needed)
 * ------------------------------------------------------------------------ */

/* Flags describing a variant of the paper's task DAG (Sec. 3). */
#define SPDINV_DAG_OUT_OF_PLACE 1  /* renaming: Step 2 reads B (copy of L), Step 3 reads C (copy of L^{-1}) */
#define SPDINV_DAG_RENAME_DIAG  2  /* also keep the inverted diagonal tiles in their own store D */
#define SPDINV_DAG_UUU          4  /* all innermost GEMM loops increasing (default: U, D, U) */
#define SPDINV_DAG_PIPELINE     8  /* one DAG across the three steps (else a barrier between steps) */
#define SPDINV_DAG_TREE        16  /* each commutative update chain of m products reduced as a tree:
                                      m independent products into temporaries, a pairwise sum, one
                                      update (the associative reduction Sec. 3 names for shortening
                                      the critical path; analysis only: the GPU kernel runs chains) */
#define SPDINV_DAG_TREE_STEP3  32  /* the same for the chains of Step 3 only */
#define SPDINV_DAG_SHARE_BC    64  /* with SPDINV_DAG_OUT_OF_PLACE: C (the copy of L^{-1}) shares B's storage
                                      (the copy of L), renaming under a memory budget (Sec. 4) */

/* Critical path, in tasks of unit weight (tile copies weigh 0), of the
 * fine-grained task DAG of Algorithm 1 (Sec. 2) or its variants (Sec. 3)
 * for t x t tiles: out[0..2] = each step's own DAG, out[3] = the whole
 * inversion (pipelined or with barriers, per SPDINV_DAG_PIPELINE).
 * Table 1 of the paper gives out[0..2] for the in-place and out-of-place
 * cases.  1 <= t <= 256 (with a tree flag, t <= 128). */
SPDINV_API spdinv_status spdinv_dag_critical_path(int t, int flags, int64_t out[4]);

/* Number of tasks of each kind in Algorithm 1 for t x t tiles, in the order
 * POTRF, TRSM, SYRK(step 1), GEMM(step 1), TRTRI, TRMM(step 2, left),
 * GEMM(step 2), TRMM(step 2, right), TRMM(step 3), LAUUM, GEMM(step 3),
 * SYRK(step 3): out[0..11]. */
SPDINV_API spdinv_status spdinv_dag_task_counts(int t, int64_t out[12]);

/* Check of the planner (host only): builds the plan for t x t tiles and
 * `steps` (as for spdinv_plan_tasks) twice -- with the bottom levels that
 * order it computed from running maxima over the task grids (O(t^2), the
 * planner's own path for every `steps`) and by walking every
 * dependency edge (O(t^3)) -- and compares them; the same for the ALAP
 * ticket order (spdinv_set_plan_order), whose grid-walk passes are compared
 * with a walk over every chain element's producers.  out[0] = tasks, out[1] =
 * positions where the two builds' orders differ (both orders summed), out[2]
 * = 1 if the critical path or the total work differ. */
SPDINV_API spdinv_status spdinv_plan_check(int t, int steps, int64_t out[3]);

/* Launch order of the emulated residual's slice GEMM (host only; no GPU): one
 * CTA per output tile of R = I - A X (lower = 0) or of a symmetric correction
 * term X R^m (lower = 1: only the tiles holding an entry on or below the
 * diagonal), for the order-n product padded to npad = n rounded up to 256.
 * wide = 1: 128 x 256 output tiles (the default kernel); 0: 128 x 128
 * (SPDINV_SLICE_TILE=128).  Launch index pid computes the tile of 128-row
 * block bm[pid] and column block bn[pid] (256 or 128 columns), in a grouped
 * raster that keeps the CTAs resident at one time on shared operand blocks;
 * the replay calls the kernels' own index functions.  *count = number of
 * launched tiles; bm and bn (both NULL to query the count, else both of
 * *count entries, caller-owned) receive the order.  Errors: n outside
 * 1 .. 2^20 (SPDINV_ERR_N); count NULL, or only one of bm, bn NULL
 * (SPDINV_ERR_NULL). */
SPDINV_API spdinv_status spdinv_slice_tile_order(int64_t n, int lower, int wide, int* bm, int* bn, int* count);

/* The execution plan the persistent kernel runs for an order-n matrix with
 * tile b: the chain tasks (one per output tile and step; each holds its
 * whole commutative update chain, Sec. 3 "loop reversal") in the order CTAs
 * take them.  Each task is encoded as (kind << 28) | (i << 14) | j with kind
 * 0 = Step-1 diagonal, 1 = Step-1 off-diagonal, 2 = Step-2 diagonal,
 * 3 = Step-2 off-diagonal, 4 = Step-3 diagonal, 5 = Step-3 off-diagonal.
 * steps: 1 = potrf, 2 = trtri, 3 = lauum, 0 = potri (all three),
 * 4 = potri_diag (Steps 1 and 2, and Step 3's diagonal tiles only).
 * Writes at most cap tasks to out (NULL allowed when cap == 0), the task
 * count to *ntasks and the weighted critical path (in units of one b^3
 * multiply-add tile product) to *crit (nullable). */
SPDINV_API spdinv_status spdinv_plan_tasks(int64_t n, int b, int steps, uint32_t* out, int64_t cap,
                                int64_t* ntasks, double* crit);

/* Host emulation of the persistent kernel's scheduling protocol (no GPU; no
 * counterpart in the paper, whose runtime schedules on CPU cores).  `workers`
 * threads stand in for CTAs: each takes the next ticket of the execution plan
 * for t x t tiles and `steps` (as for spdinv_plan_tasks), waits for each input
 * tile's readiness flag in the order the kernel reads them (bounded by
 * wait_limit_s; a wait that runs out stops every worker), spends a seeded
 * random 0 .. max_delay_us microseconds per chain element and per tile
 * kernel, stores its output tiles and publishes their flags.  Every tile
 * location carries the task that last stored it, and every read checks it
 * against what Algorithm 1 needs there (the input for A's tiles, the
 * producing task for the renamed stores): a read before the producer stored,
 * or after Step 3 overwrote a tile of A, is a hazard.
 *   drop_task >= 0: the task with that ticket never publishes (the
 *     fault_drop_task hook of spdinv_opts);
 *   skip_wait_task >= 0: the task with that ticket reads without waiting (a
 *     protocol with a wait missing, to show that the hazard check sees it).
 *   out[0] tasks completed, out[1] tasks in the plan, out[2] protocol errors
 *   (a flag published twice), out[3] hazards, out[4] the longest wait in
 *   microseconds.
 * Returns SPDINV_OK when every task completed, SPDINV_ERR_TIMEOUT when a wait
 * ran out; 1 <= t <= 256, 0 <= steps <= 4, 1 <= workers <= 1024. */
SPDINV_API spdinv_status spdinv_plan_emulate(int t, int steps, int workers, uint64_t seed, int drop_task,
                                             int skip_wait_task, double wait_limit_s, int max_delay_us,
                                             int64_t out[5]);

/* spdinv_plan_emulate for an execution variant's plan (spdinv_opts.variant,
 * SPDINV_VARIANT_*; the whole inversion), with the kernel's write-after-read
 * protocol: every read of a tile that a later version overwrites is counted,
 * and the writer of that version waits (bounded) for the count the planner
 * expects.  A read that finds a later version than it needs counts as a
 * hazard; a read count that differs from the expected one at the end counts
 * as a protocol error.  split_segment: as in spdinv_opts.  Same outputs and
 * limits as spdinv_plan_emulate (no skip-wait hook). */
SPDINV_API spdinv_status spdinv_plan_emulate_variant(int t, int variant, int split_segment, int workers,
                                                     uint64_t seed, int drop_task, double wait_limit_s,
                                                     int max_delay_us, int64_t out[5]);

/* Deterministic schedule of the execution plan for t x t tiles and `steps`
 * on `workers` CTAs (host only; a list-scheduling model of the persistent
 * kernel, no counterpart in the paper, whose Sec. 3 analyses critical paths
 * only).  The next ticket goes to the CTA that becomes free first; the CTA
 * runs the task's chain elements in the kernel's order, each one starting
 * when the previous one is done and its input tiles are final.  Costs are in
 * units of one b x b x b tile product: 1 per chain element and per TRMM,
 * 0.7 for a diagonal POTRF + TRTRI, 0.4 for a TRTRI alone.
 *   out[0] makespan, out[1] total work (the sum of the costs), out[2] the
 *   plan's weighted critical path (task granularity, as spdinv_plan_tasks).
 * work / (workers * makespan) is the fraction of CTA time the schedule keeps
 * busy.  1 <= t <= 4096, 0 <= steps <= 4, workers >= 1. */
SPDINV_API spdinv_status spdinv_plan_simulate(int t, int steps, int workers, double out[3]);

/* Ticket order of the persistent kernel's plans (the result does not depend
 * on it: every output tile keeps its own accumulation order, and both orders
 * are topological, so no grid can deadlock).
 *   SPDINV_PLAN_BOTTOM_LEVEL  decreasing task-level bottom level;
 *   SPDINV_PLAN_ALAP          increasing latest finish time of each task when
 *                             every chain element starts as soon as its own
 *                             inputs are final (unlimited CTAs), raised to the
 *                             largest key among the task's producers (the
 *                             default).  Measured on a GB300 (tile 32): 2.2 %
 *                             faster than the bottom-level order at n = 4096,
 *                             0.6 % at 8192, 0.3 % at 16384; never slower.
 *                             Its passes visit every chain element, O(t^3)
 *                             host time on the first call per size (about
 *                             0.02 s at t = 128, 0.15 s at 256, 1 s at 512;
 *                             the bottom-level order takes O(t^2)).
 * Sets the order for plans built after the call (plans are cached per order)
 * and for the host queries; returns the previous order, or
 * SPDINV_ERR_UNSUPPORTED for an unknown one (nothing changes).  The initial
 * order is SPDINV_PLAN_ORDER=bottom_level (or 0) from the environment, else
 * the default. */
#define SPDINV_PLAN_BOTTOM_LEVEL 0
#define SPDINV_PLAN_ALAP 1
SPDINV_API int spdinv_set_plan_order(int order);

/* ------------------------------------------------------------------------
 * Debugging
 * ------------------------------------------------------------------------ */

/* Fill the renamed stores B, C and D of every FP64 single-matrix call with
 * NaN (all bits set) before its kernel runs, so that a tile read before it
 * was written turns the result into NaN instead of passing unseen. */
#define SPDINV_DEBUG_POISON 1u

/* Sets the debug flags of the process (SPDINV_DEBUG_* ORed; the initial value
 * is SPDINV_DEBUG from the environment, else 0) and returns the previous
 * ones.  Host only; takes effect for calls made after it returns. */
SPDINV_API unsigned spdinv_set_debug_flags(unsigned flags);

/* ------------------------------------------------------------------------
 * Measurement (the paper has no counterpart: utilities for reporting rates
 * against this GPU's measured peak)
 * ------------------------------------------------------------------------ */

/* Peak microbenchmark.  Queues one kernel on `stream` that keeps one pipe
 * busy on register operands -- kind SPDINV_PROBE_DMMA: the FP64 tensor-core
 * MMA mma.sync m8n8k4, SPDINV_PROBE_DFMA: the FP64 fused multiply-add (the
 * instruction of the FP64 tile products, the faster of the two on GB300),
 * SPDINV_PROBE_FFMA: the FP32
 * fused multiply-add (the CUDA-core FP32 tile products) -- with 16
 * independent accumulators per thread, `iters` iterations, `blocks_per_sm`
 * CTAs of 128 threads per SM (1..16).  *flops receives the number of
 * floating-point operations the kernel performs (host, set before return);
 * the caller times the kernel with CUDA events on `stream`.  d_sink: device
 * buffer of at least 4 * blocks_per_sm * (number of SMs) doubles, written
 * with the accumulators so that no work is optimised away. */
#define SPDINV_PROBE_DMMA 0
#define SPDINV_PROBE_DFMA 1
#define SPDINV_PROBE_FFMA 2
SPDINV_API spdinv_status spdinv_fp64_peak_probe(int kind, int64_t iters, int blocks_per_sm, double* d_sink,
                                                double* flops, cudaStream_t stream);

/* Kernel timing: while on (spdinv_set_kernel_timing(1)), the library records
 * a CUDA event pair around each of its launches of the kernels below, on the
 * launch's stream.  spdinv_kernel_time_ms(which, &ms, &launches) waits for the
 * recorded launches of one kind to finish, returns their summed duration,
 * count and algorithmic work (*flops: the slice GEMM counts 2 * 128 * N * K
 * per launched 128 x N output tile and slice pair, N = 256 or 128 by the
 * kernel's form, K the padded order; the DAGs n^3), and
 * forgets them.  Host only; timing costs two event records per launch. */
#define SPDINV_TIMED_SLICE_GEMM 0  /* the tcgen05 slice products (ozaki_tc_wide / ozaki_tc_kernel) */
#define SPDINV_TIMED_MIXED_DAG 1   /* the persistent FP32/FP64 tile DAG of the mixed precision */
#define SPDINV_TIMED_FP64_DAG 2    /* the persistent FP64 tile DAG */
#define SPDINV_TIMED_KERNELS 3
SPDINV_API spdinv_status spdinv_set_kernel_timing(int on);
SPDINV_API spdinv_status spdinv_kernel_time_ms(int which, double* ms, int* launches, double* flops);

/* Per-task trace of the persistent FP64 kernel (the paper has no
 * counterpart).  While a trace buffer is set for the current
 * device, every FP64 single-matrix call (spdinv_potrf, _trtri, _lauum,
 * _potri, _potri_ex, _potri_diag) runs the kernel's tracing build and writes
 * one record per task, at index = its ticket (the position in the plan's
 * order): the task word (kind << 28 | i << 14 | j; kind 6 = a split-chain
 * segment with its id in the low 28 bits), the SM and CTA that ran it, and
 * the global timer (ns) when the CTA took it and when it finished it, and
 * the part of that time spent waiting for input tiles' flags.  The
 * tracing build is the variant build of the kernel: a traced run measures
 * that build, within a few percent of the default one.
 * spdinv_set_trace(d_records, capacity): device array of `capacity` records
 * (48 bytes each)
 * (NULL = off).  A call whose plan has more tasks than `capacity` returns
 * SPDINV_ERR_WORKSPACE and launches nothing.  The caller owns the buffer;
 * records of tasks that did not run (after an error) are left as they were. */
typedef struct {
    uint32_t task, sm, ticket, cta;
    uint64_t t_start_ns, t_end_ns;
    uint64_t t_wait_ns;  /* of that time, spent waiting for the flags of input tiles */
    uint64_t reserved;
} spdinv_trace_record;
SPDINV_API spdinv_status spdinv_set_trace(spdinv_trace_record* d_records, int64_t capacity);

/* ------------------------------------------------------------------------
 * Library information
 * ------------------------------------------------------------------------ */

/* Name of a status code ("SPDINV_ERR_N", ...; "unknown status" otherwise),
 * a static string. */
SPDINV_API const char* spdinv_status_name(int status);

/* Text of the last CUDA runtime error seen by this thread's calls (or ""). */
SPDINV_API const char* spdinv_last_cuda_error(void);

/* Number of kernels this library has queued since it was loaded (all
 * devices, all threads): a host-side counter, incremented per launch. */
SPDINV_API uint64_t spdinv_kernel_launches(void);

/* Version as major*10000 + minor*100 + patch.  1.2 appended diag_fp64 to
 * spdinv_opts (the library reads the whole struct: rebuild callers compiled
 * against an older header) and added spdinv_slice_tile_order. */
SPDINV_API int spdinv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPDINV_H */
