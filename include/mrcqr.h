/*
 * mrcqr.h -- C ABI of the GB300 MRCQR library (libmrcqr.so).
 *
 * MRCQR (Garrison, Chen, Ipsen, "Numerically Stable Cholesky-QR on GPU via
 * Mixed-Precision Randomized Preconditioning") computes the thin QR
 * factorization A = QR of a tall-skinny FP64 matrix (m >> n, full column
 * rank) with an explicit Q, ||I - Q^T Q||_2 = O(u) for kappa_2(A) up to 1e16
 * (Sec. I, Eq. 1).  Algorithm 2: a randomized trigonometric sketch
 * Y = sqrt(m/s) P F D A taken in a reduced precision p gives a preconditioner
 * R_s (the R of Y); Cholesky-QR (Algorithm 1) of W = A R_s^{-1} runs in FP64;
 * R = R_c R_s.
 *
 * Conventions for every entry point:
 *  - Matrices are DEVICE memory, column-major (LAPACK/cuBLAS convention), on
 *    the device that is current when the call is made.  The caller owns A, Q
 *    and R.  A is read only and must not overlap Q or R.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; 0 = legacy default
 *    stream).  Argument errors return at once, before anything is enqueued.
 *    Errors found on the device (breakdown, non-finite input, failed
 *    orthogonality) go to a device status record read by
 *    mrcqr_get_last_status() or written to opts->stats_device.
 *  - The library allocates its workspace with the stream-ordered allocator
 *    (cudaMallocAsync / cudaFreeAsync on `stream`) inside each call.
 *  - Results are deterministic for a fixed seed, shape, precision and build:
 *    every reduction runs in a fixed order, no floating-point atomics.
 *  - Return value: an mrcqr_status_t (MRCQR_OK when the work was enqueued).
 */
#ifndef MRCQR_H
#define MRCQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mrcqr_stream_t; /* same type as cudaStream_t */

/* Sketch precision p of Algorithm 2 (Sec. II-B: half suffices for
 * kappa <~ 1e4, single for kappa <~ 1e8, double beyond).  BF16 is an extra
 * tier (unit roundoff 2^-8: safe for kappa <~ 1e2).  AUTO lets the learned
 * selector pick from an FP16 sketch's R_s (see mrcqr_selector_load). */
typedef enum {
  MRCQR_PREC_FP16 = 0,
  MRCQR_PREC_BF16 = 1,
  MRCQR_PREC_FP32 = 2,
  MRCQR_PREC_FP64 = 3,
  MRCQR_PREC_AUTO = 4
} mrcqr_prec_t;

typedef enum {
  MRCQR_OK = 0,
  MRCQR_ERR_INVALID = 1,   /* bad argument; nothing enqueued */
  MRCQR_ERR_BREAKDOWN = 2, /* Cholesky of the Gram matrix met a non-positive pivot (Sec. I-A) */
  MRCQR_ERR_NONFINITE = 3, /* A holds NaN or Inf */
  MRCQR_ERR_ORTHO = 4,     /* ||I - Q^T Q||_F above tolerance at the highest precision tried */
  MRCQR_ERR_ALLOC = 5,     /* workspace allocation failed */
  MRCQR_ERR_CUDA = 6,      /* a CUDA call or launch failed */
  MRCQR_ERR_TIMEOUT = 7    /* a bounded device wait gave up (batched persistent kernels) */
} mrcqr_status_t;

/* Sketch transform F of Algorithm 2 (Sec. II-A).
 *  DCT:       c rows k of the orthonormal DCT-II, sampled from {0..m-1}, scale sqrt(m/c):
 *             Y_i = sqrt(2/c) c_k sum_j cos(pi k (2j+1) / (2m)) d_j A_j, c_0 = 1/sqrt(2), else 1.
 *  RFFT:      the paper's transform: c bins k of the real FFT, sampled from the
 *             floor(m/2) + 1 distinct bins of a real column, real parts, scale sqrt(c/m):
 *             Y_i = sqrt(c/m) sum_j cos(2 pi k j / m) d_j A_j (unnormalised DFT).
 *  RFFT_REIM: as RFFT, with the imaginary parts -sqrt(c/m) sum_j sin(2 pi k j / m) d_j A_j
 *             of the same c bins stacked below: a 2c x n sketch.
 * Bins and rows are 0-based (the paper's bin k + 1); a scalar scale of Y cancels in
 * Q and R. */
typedef enum {
  MRCQR_TRANSFORM_DCT = 0,
  MRCQR_TRANSFORM_RFFT = 1,
  MRCQR_TRANSFORM_RFFT_REIM = 2
} mrcqr_transform_t;

typedef struct mrcqr_opts {
  int32_t s_factor;   /* sampled rows or bins c = s_factor * n (default 2; the paper uses 3, Sec. II-A);
                         Y has c rows, 2c for MRCQR_TRANSFORM_RFFT_REIM (at most 8192), and c is at
                         most m (DCT) or floor(m/2) + 1 (real FFT) */
  int32_t check;      /* 1 (default): measure ||I - Q^T Q||_F on device and judge the result */
  int32_t escalate;   /* 1 (default): on failure re-run at the next precision (Sec. II-C),
                         FP16/BF16 -> FP32 -> FP64 */
  int32_t sketch_variant; /* 0 (default): for FP16/BF16/FP32, the faster of the two tensor-core variants
                             by a table measured on GB300 (dense sampled rows, or the four-step
                             transform where it applies) when A is 16-byte aligned and lda is even,
                             SIMT otherwise; the FP64 sketch as emulated FP64 on the tensor cores
                             (unless fp64_products = 1) from digit planes of D A sliced once (5)
                             where they fit, else sliced per work item (3); 1: SIMT (FP64 FMA for
                             FP64); 2: tensor-core dense sampled rows when possible; 4: the four-step
                             transform (a radix-64 DFT of the strided subsequences on the tensor
                             cores, then only the sampled outputs) when possible -- DCT,
                             FP16/BF16/FP32, m a multiple of 1024 up to 2^22, at most 1024 sampled
                             rows -- else as 2; 3: FP64 only, the emulated sketch sliced per work
                             item.  The digit planes take 16 bytes per entry of A: a factorization
                             writes them into its Q buffer (Q is overwritten before stage 2 of the
                             level), in row chunks of at most half of Q; mrcqr_sketch and
                             mrcqr_sketch_ex hold them in their workspace. */
  double ortho_tol;   /* acceptance threshold on ||I - Q^T Q||_F (default 1e-13) */
  void* stats_device; /* optional DEVICE pointer to an mrcqr_stats_t written at the end */
  int32_t fp64_products; /* 0 (default): the FP64 sketch, the off-diagonal updates of W = A R_s^{-1},
                            the Gram matrix W^T W, the product Q = W R_c^{-1} and the check Q^T Q
                            as emulated FP64 on the FP16 tensor cores (exact 8-bit digit slicing,
                            integer recombination, one final rounding; see mrcqr_trsm, mrcqr_gram
                            and mrcqr_finalize_q); 1: FP64 FMA kernels throughout */
  int32_t transform;  /* mrcqr_transform_t, default MRCQR_TRANSFORM_DCT (0) */
} mrcqr_opts_t;

typedef struct mrcqr_stats {
  int32_t status;          /* mrcqr_status_t of the device-side result */
  int32_t prec_used;       /* sketch precision of the accepted (or last) run */
  int32_t retries;         /* re-runs at a higher precision */
  int32_t prec_first;      /* precision of the first run (AUTO: the selector's choice) */
  int32_t selector_choice; /* AUTO only: 0 fp16, 1 fp32, 2 fp64; else -1 */
  int32_t reserved[3];
  double ortho_fro;        /* measured ||I - Q^T Q||_F of the accepted (or last) run */
} mrcqr_stats_t;

/* Library version (major*10000 + minor*100 + patch). */
int mrcqr_version(void);

/* Static text for a status code. */
const char* mrcqr_status_string(int status);

/* Algorithm 2 (MRCQR) on one matrix.
 *   m, n        : A is m x n, 1 <= n <= 512, m >= s = 2n, m < 2^31.
 *   A, lda      : input, lda >= m.  Read only.
 *   Q, ldq      : output m x n with orthonormal columns, ldq >= m.  Also
 *                 used as scratch for W = A R_s^{-1}.
 *   R           : output n x n upper triangular (ld = n), positive diagonal,
 *                 strict lower triangle set to zero.
 *   sketch_prec : mrcqr_prec_t; with the default options a failed check
 *                 re-runs at the next precision.  MRCQR_PREC_AUTO needs
 *                 selector weights (mrcqr_selector_load).
 *   seed        : Philox key of the random signs D and the sample set S.
 * Same as mrcqr_factor_ex(..., ldr = n, opts = NULL, stream). */
int mrcqr_factor(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                 int sketch_prec, uint64_t seed, mrcqr_stream_t stream);

/* As mrcqr_factor with an explicit ldr (>= n) and options (NULL = defaults). */
int mrcqr_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                    int64_t ldr, int sketch_prec, uint64_t seed, const mrcqr_opts_t* opts, mrcqr_stream_t stream);

/* Synchronizes `stream` and returns the device status record of the last
 * factorization enqueued on it by this process (MRCQR_ERR_INVALID if none). */
int mrcqr_get_last_status(mrcqr_stream_t stream, mrcqr_stats_t* out);

/* Many independent factorizations (the repeated QRs of block Krylov and
 * randomized-SVD power steps, Sec. II-C) in grouped launches over the whole
 * batch (a one-shot plan, see mrcqr_batched_plan_create).
 *   count          : number of problems (>= 1).
 *   m, n, lda, ldq : HOST arrays[count] (used for planning).
 *   A, Q, R        : HOST arrays[count] of DEVICE pointers; R_i is n_i x n_i, ld n_i.
 *   sketch_prec    : HOST array[count] of mrcqr_prec_t (AUTO not accepted here).
 *   seeds          : HOST array[count].
 *   status         : DEVICE int32[count] receiving each problem's mrcqr_status_t.
 * Per-problem rules are those of mrcqr_factor with m >= 2n; problems are
 * independent.  The workspace comes from the stream-ordered allocator. */
int mrcqr_factor_batched(int count, const int64_t* m, const int64_t* n, const double* const* A, const int64_t* lda,
                         double* const* Q, const int64_t* ldq, double* const* R, const int* sketch_prec,
                         const uint64_t* seeds, int32_t* status, mrcqr_stream_t stream);

/* Reusable batched plans.  A plan owns the batch workspace (allocated once)
 * and the per-phase work lists; executing it enqueues one grouped launch per
 * phase and kernel variant (about 20 per escalation level for the whole
 * batch) or, with use_graph, replays them as one CUDA graph (captured at the
 * first execute on a private stream, then launched on the caller's stream).
 * The buffers named at creation are the ones every execute reads and writes.
 * autotune = 1 times the grouped SYRK and sketch kernels on this batch for
 * a few split sizes at creation (synchronous; results cached per batch shape
 * and, when the environment variable MRCQR_TUNE_CACHE names a file, stored
 * there). */
typedef struct mrcqr_batched_plan_s* mrcqr_batched_plan_t;

typedef struct mrcqr_batched_opts {
  int32_t use_graph;      /* 1: capture the launch sequence into a CUDA graph */
  int32_t autotune;       /* 1: tune rows_per_split / rows_per_chunk at creation */
  int32_t check;          /* 1 (default): device orthogonality judge */
  int32_t escalate;       /* 1 (default): re-run failed problems at the next precision */
  double ortho_tol;       /* default 1e-13 */
  int64_t rows_per_split; /* SYRK rows per partial (0: tuned or default 4096) */
  int64_t rows_per_chunk; /* sketch rows per partial (0: tuned or default 8192) */
  int32_t fp64_products;  /* 0 (default): emulated FP64 products on the tensor cores; 1: every phase grouped with
                             FP64 FMA kernels */
  int32_t transform;      /* mrcqr_transform_t of every problem's sketch (default DCT): 2n sampled rows, or 2n
                             bins of the real FFT (then 2n <= floor(m/2) + 1 for every problem, and 4n <= 8192
                             for MRCQR_TRANSFORM_RFFT_REIM; INVALID otherwise) */
  int32_t oz_per_problem; /* with emulated FP64 products: 0 (default) runs the FP64 sketch, W = A R_s^-1, the
                             Gram, Q = W R_c^-1 and the check as one grouped persistent launch per kernel over
                             every problem's {problem, row block or tile} items; 1 runs the single-problem
                             kernels per problem on side streams (fork/join inside the plan) */
} mrcqr_batched_opts_t;

int mrcqr_batched_plan_create(int count, const int64_t* m, const int64_t* n, const double* const* A,
                              const int64_t* lda, double* const* Q, const int64_t* ldq, double* const* R,
                              const int* sketch_prec, const uint64_t* seeds, int32_t* status,
                              const mrcqr_batched_opts_t* opts, mrcqr_batched_plan_t* plan);
int mrcqr_batched_plan_execute(mrcqr_batched_plan_t plan, mrcqr_stream_t stream);
/* Tuned sizes, launches per execute and workspace bytes of a plan (host outputs, any may be NULL). */
int mrcqr_batched_plan_info(mrcqr_batched_plan_t plan, int64_t* rows_per_split, int64_t* rows_per_chunk,
                            int32_t* kernels_per_execute, int64_t* workspace_bytes);
/* Frees the plan; the caller must first make sure no execute is in flight. */
int mrcqr_batched_plan_destroy(mrcqr_batched_plan_t plan);

/* ---- step-level entry points (each is one step of Algorithm 2) ---------- */

/* Algorithm 2 step 1: d[i] = +-1, i < m (DEVICE double[m]). */
int mrcqr_signs(int64_t m, uint64_t seed, double* d, mrcqr_stream_t stream);

/* Algorithm 2 step 1: the sample set, s distinct rows of {0..m-1} sorted
 * ascending (DEVICE uint32[s]); 1 <= s <= min(m, 8192). */
int mrcqr_sample_rows(int64_t m, int64_t s, uint64_t seed, uint32_t* idx, mrcqr_stream_t stream);

/* Algorithm 2 step 1 for a given transform: c distinct rows (DCT, of {0..m-1})
 * or bins (real FFT, of {0..floor(m/2)}), uniform without replacement (Floyd,
 * the same Philox stream as mrcqr_sample_rows over that population), sorted
 * ascending, written to idx[0..c) (DEVICE uint32).  MRCQR_TRANSFORM_RFFT_REIM
 * also writes the Im rows of the same bins to idx[c..2c) as bin | 0x80000000.
 * INVALID when c exceeds the population or the rows of Y exceed 8192. */
int mrcqr_sample_transform_rows(int64_t m, int64_t c, int transform, uint64_t seed, uint32_t* idx,
                                mrcqr_stream_t stream);

/* fl_p of Algorithm 2 step 2 exactly as the tensor-core sketch applies it:
 * one round-to-nearest-even from FP64 to FP16, BF16 or FP32 (subnormal
 * targets included), y[i] = fl_p(x[i]) widened back to FP64 (DEVICE arrays
 * of count doubles).  FP64 copies. */
int mrcqr_round(int prec, int64_t count, const double* x, double* y, mrcqr_stream_t stream);

/* Algorithm 2 steps 1-4: Y = sqrt(m/s) P F D A in precision sketch_prec
 * (FP16/BF16/FP32/FP64), returned widened to FP64 (DEVICE double s x n,
 * ld = s). */
int mrcqr_sketch(int64_t m, int64_t n, const double* A, int64_t lda, int64_t s, int sketch_prec, uint64_t seed,
                 double* Y, mrcqr_stream_t stream);

/* As mrcqr_sketch with an explicit kernel variant (see mrcqr_opts_t.sketch_variant). */
int mrcqr_sketch_ex(int64_t m, int64_t n, const double* A, int64_t lda, int64_t s, int sketch_prec, uint64_t seed,
                    int variant, double* Y, mrcqr_stream_t stream);

/* Algorithm 2 steps 1-4 with the transform of mrcqr_transform_t: c sampled
 * rows or bins (mrcqr_sample_transform_rows with the same seed), Y = the
 * scaled transform rows times D A in precision sketch_prec, widened to FP64
 * (DEVICE double, ld = rows of Y: c, or 2c for MRCQR_TRANSFORM_RFFT_REIM with
 * the Re rows first).  variant as mrcqr_opts_t.sketch_variant.  A: DEVICE
 * double m x n, ld lda >= m, read-only.  Allocates its workspace with
 * cudaMallocAsync on `stream`; INVALID before any launch on bad arguments. */
int mrcqr_sketch_transform(int64_t m, int64_t n, const double* A, int64_t lda, int64_t c, int transform,
                           int sketch_prec, uint64_t seed, int variant, double* Y, mrcqr_stream_t stream);

/* Algorithm 2 steps 5-6: R_s of Y (DEVICE double s x n, ld = s) by
 * Householder QR in FP32 (prec FP16/BF16/FP32) or FP64, diag(R_s) > 0,
 * written to Rs (DEVICE double n x n, ld = n). */
int mrcqr_sketch_qr(int64_t n, int64_t s, const double* Y, int prec, double* Rs, mrcqr_stream_t stream);

/* CholQR2, the comparison method of the paper's stability experiment (Sec. I-A,
 * Sec. III-B): Algorithm 1 run twice, R_1 = chol(A^T A), then Q, R_2 = CholQR(A R_1^{-1})
 * (A R_1^{-1} by substitution) and R = R_2 R_1, all products in emulated FP64
 * (as mrcqr_factor).  A (m x n, ld lda), Q (m x n, ld ldq), R (n x n, ld ldr,
 * strict lower triangle set to 0): DEVICE doubles, column-major, caller-owned;
 * A is read-only and may not alias Q or R.  Asynchronous on stream; status
 * through mrcqr_get_last_status: BREAKDOWN when A^T A is not numerically
 * positive definite (kappa_2(A) beyond about 1e8), ORTHO when ||I - Q^T Q||_F
 * exceeds 1e-13.  INVALID on bad arguments (before any launch). */
int mrcqr_cholqr2(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                  int64_t ldr, mrcqr_stream_t stream);

/* Regime estimates without learning (Sec. II-C): an estimate of kappa_2(A)
 * and the sketch precision it calls for (0 half: kappa <= 1e4, 1 single:
 * kappa <= 1e8, 2 double), before any factorization.
 *  CHOLQR_PROBE: Algorithm 1 on A (Gram, Cholesky, Q = A R^{-1}, all products
 *    emulated FP64 as in mrcqr_factor), q = ||I - Q^T Q||_2 by power iteration
 *    on the n x n Gram of Q, kappa = sqrt(q / (u (1 + q))) with u = 2^-53 (the
 *    probe's lower bound).  out = {kappa, regime, q, 0}.
 *  ONENORM: G = A^T A, kappa = sqrt(n ||G||_1 est), est <= ||G^-1||_1 from the
 *    block 1-norm estimator of Higham and Tisseur (t = 2, at most 5 iterations,
 *    random +-1 columns from Philox with key `seed`, G^-1 applied through the
 *    Cholesky factor; exact for n <= 4).  out = {kappa, regime, ||G||_1, est}.
 * A Cholesky breakdown (kappa_2(A) beyond about 1e8) gives kappa = inf and
 * regime 2.  A: DEVICE double m x n, column-major, ld lda >= m, read-only,
 * 1 <= n <= 512, n <= m < 2^31; out: DEVICE double[4], written on `stream`.
 * Allocates its workspace (m x n doubles more for the probe) with
 * cudaMallocAsync on `stream`.  INVALID before any launch on bad arguments. */
typedef enum { MRCQR_REGIME_CHOLQR_PROBE = 0, MRCQR_REGIME_ONENORM = 1 } mrcqr_regime_method_t;
int mrcqr_regime_estimate(int64_t m, int64_t n, const double* A, int64_t lda, int method, uint64_t seed,
                          double* out, mrcqr_stream_t stream);

/* Algorithm 2 steps 7-9 with a given preconditioner: Q, R_c = CholQR(A R_s^{-1})
 * (Algorithm 1) and R = R_c R_s.  With Rs = I this is Algorithm 1 on A.
 * Status (breakdown) through mrcqr_get_last_status. */
int mrcqr_cholqr_precond(int64_t m, int64_t n, const double* A, int64_t lda, const double* Rs, double* Q,
                         int64_t ldq, double* R, int64_t ldr, mrcqr_stream_t stream);

/* Algorithm 2 step 7: W = A R^{-1} by substitution on the rows (R upper
 * triangular with nonzero diagonal).  A: DEVICE double m x n, column-major,
 * ld lda >= m; R: DEVICE double n x n, column-major, ld ldr >= n, only the
 * upper triangle is read; W: DEVICE double m x n, ld ldw >= m, must not
 * overlap A or R.  fp64_products = 0: blocked by 16 columns, the off-diagonal
 * updates W_{<J} R_{<J,J} as emulated FP64 on the FP16 tensor cores (one
 * rounding each, then one FP64 subtraction from A_J), the 16 x 16 diagonal
 * blocks by FP64 substitution; 1: FP64 substitution throughout.
 * 1 <= n <= 512, 1 <= m < 2^31.  Allocates its workspace with cudaMallocAsync
 * on `stream`. */
int mrcqr_trsm(int64_t m, int64_t n, const double* A, int64_t lda, const double* R, int64_t ldr, double* W,
               int64_t ldw, int fp64_products, mrcqr_stream_t stream);

/* Algorithm 1 step 1 (and the check of Sec. II-C): G = W^T W.  W: DEVICE
 * double m x n, column-major, ld ldw >= m; G: DEVICE double n x n, packed
 * column-major, receives the upper triangle (diagonal included), strictly
 * lower triangle set to zero.  fp64_products = 0: emulated FP64 on the FP16
 * tensor cores -- every column sliced against the exponent of its maximum
 * over all m rows, exact integer level sums, each entry rounded once (error
 * per term at most 2^-57 times the two column maxima; deterministic for any
 * launch configuration; a non-finite column gives NaN entries); 1: FP64 FMA
 * with fixed-order partial sums.  1 <= n <= 512, 1 <= m < 2^31.  Allocates its
 * workspace with cudaMallocAsync on `stream`. */
int mrcqr_gram(int64_t m, int64_t n, const double* W, int64_t ldw, double* G, int fp64_products,
               mrcqr_stream_t stream);

/* Algorithm 1 step 3 (and Algorithm 2 step 9): Q <- W X in place, with
 * X = R_c^{-1} upper triangular.  Q: DEVICE double m x n, column-major,
 * ld ldq >= m, holds W on entry; X: DEVICE double n x n, column-major,
 * ld ldx >= n, only the upper triangle (diagonal included) is read.
 * fp64_products = 0: emulated FP64 on the FP16 tensor cores (each entry the
 * once-rounded value of a 63-bit fixed-point evaluation of the exact sum,
 * error per term at most 2^-57 times the row maximum of W times the column
 * maximum of X; non-finite operands give NaN rows); 1: FP64 FMA.
 * 1 <= n <= 512, 1 <= m < 2^31; Q and X must not overlap.  Allocates its workspace with cudaMallocAsync on `stream`.
 * Returns MRCQR_ERR_INVALID / MRCQR_ERR_ALLOC before enqueueing anything. */
int mrcqr_finalize_q(int64_t m, int64_t n, double* Q, int64_t ldq, const double* X, int64_t ldx, int fp64_products,
                     mrcqr_stream_t stream);

/* Test hook for the bounded device waits: one CTA waits on a barrier that
 * nothing completes, with the bounded wait of the tensor-core pipelines
 * (each poll blocks for a hardware time slice), and writes MRCQR_ERR_TIMEOUT
 * to *status (DEVICE int32) when `polls` polls (1 .. 2^20) run out; the
 * context stays usable.  INVALID on bad arguments. */
int mrcqr_debug_wait_timeout(uint32_t polls, int32_t* status, mrcqr_stream_t stream);

/* Allocation-free variant of mrcqr_sketch_qr.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need R_s -- code running under another framework's memory
 * manager that forbids raw cudaMalloc, or a latency-critical loop where a
 * device allocation (and the synchronization it can imply) is not allowed.
 * Same arguments, layout and result as mrcqr_sketch_qr, but the scratch
 * (working copy of Y, padded R_s^T, 1/diag, control block; about 641 KiB) is
 * one static device array inside the library, held on every GPU that loads
 * the library until the process exits.  Limits: 1 <= n <= 128 and
 * n <= s <= 512; larger sizes return MRCQR_ERR_INVALID (with a message on
 * stderr) before anything is enqueued.  The call allocates nothing
 * (no cudaMalloc/cudaMallocAsync/cudaFree).  All calls share the array and it
 * keeps the last call's contents (each call clears what must start at zero),
 * so calls whose kernels overlap on the GPU race: order them on one stream
 * or with events.  The stream must belong to the current device (another
 * device's stream returns MRCQR_ERR_INVALID).  The first call in each CUDA
 * context looks up the array's address (cudaGetSymbolAddress, with that
 * device current) and caches it under the context's id, so a device reset
 * (a new context) is followed by a fresh lookup; make the first call on a
 * device, and the first after a reset, outside any stream capture. */
int mrcqr_sketch_qr_noalloc(int64_t n, int64_t s, const double* Y, int prec, double* Rs, mrcqr_stream_t stream);

/* ---- learned sketch-precision selector ------------------------------------
 * The paper lets the caller pick p from a coarse regime of kappa_2(A) and
 * names machine-learned condition estimators as one way to get it (Sec.
 * II-C).  With sketch_prec = MRCQR_PREC_AUTO an FP16 sketch is taken, 16
 * features of its R_s are computed on the device, and an MLP 16-64-64-3
 * (BF16 weights, FP32 accumulation) picks where the ladder FP16 -> FP32 ->
 * FP64 starts by minimising the expected cost (a too-low start costs every
 * run up to the right precision); the orthogonality judge still escalates.
 * Parameters (FP32, nparams = mrcqr_selector_num_params()): W1[64][16],
 * b1[64], W2[64][64], b2[64], W3[3][64], b3[3] (row-major); the features are
 * standardised with mu, sd before the first layer; costs[3] are the relative
 * costs of one run at FP16, FP32, FP64. */
int mrcqr_selector_num_params(void);
/* Installs selector weights for the current device (HOST arrays). */
int mrcqr_selector_set(const float* params, const float* mu, const float* sd, const float* costs);
/* Loads a weight file: "MRCQRSEL", uint32 version 1, uint32 nparams, float mu[16], sd[16], costs[3],
 * float params[nparams] (little endian). */
int mrcqr_selector_load(const char* path);
/* The 16 selector features of an upper-triangular Rs (DEVICE n x n, ld n) of a problem with m rows,
 * written to feat (DEVICE float[16]). */
int mrcqr_selector_features(int64_t m, int64_t n, const double* Rs, float* feat, mrcqr_stream_t stream);
/* Batched MLP inference: logits (DEVICE float[batch][3]) and, if choice is non-NULL, the expected-cost
 * choice (DEVICE int32[batch]) for raw features X (DEVICE float[batch][16]); w_bf16 DEVICE BF16
 * parameters, mu/sd/costs DEVICE. */
int mrcqr_mlp_forward(int batch, const float* X, const uint16_t* w_bf16, const float* mu, const float* sd,
                      const float* costs, float* logits, int32_t* choice, mrcqr_stream_t stream);
/* One training step on a minibatch (all DEVICE): class-weighted mean cross-entropy of labels y (0 fp16,
 * 1 fp32, 2 fp64) with weights class_w[3], gradient on the BF16 weights w_bf16 (FP32 accumulation,
 * deterministic fixed-order reduction); with apply = 1 an AdamW update (decoupled weight decay wd,
 * bias-corrected at step >= 1) of the FP32 master weights and moments, and w_bf16 refreshed.
 * grad_out (float[nparams]) and loss_out (float[1]) may be NULL. */
int mrcqr_mlp_train_step(int batch, const float* X, const int32_t* y, const float* class_w, const float* mu,
                         const float* sd, float* master, float* mom, float* var, uint16_t* w_bf16, float lr,
                         float beta1, float beta2, float eps, float wd, int step, int apply, float* grad_out,
                         float* loss_out, mrcqr_stream_t stream);

/* ---- instrumentation (per-kernel timing) ------ */

/* Sketch kernel variant used by the most recent sketch launch of this
 * process: 1 SIMT, 2 tensor-core dense sampled rows, 3 emulated FP64 on the
 * tensor cores sliced per work item, 4 four-step transform, 5 emulated FP64
 * from digit planes (0 before any). */
int mrcqr_last_sketch_variant(void);

/* Number of kernels this library has launched from the host in this process
 * (every <<<...>>> launch site counts itself; replaying a captured CUDA graph
 * runs its kernels without passing through the launch sites again). */
uint64_t mrcqr_launch_count(void);

/* Name of a profiling stage id (sketch, trsm, syrk, ...). */
const char* mrcqr_stage_name(int stage);

/* From now on bracket every kernel launch with a pair of CUDA events on its
 * stream (adds ~2 event records per launch). */
int mrcqr_profile_begin(void);

/* Stops recording, waits for the recorded events and returns up to
 * max_records (stage id, escalation level, milliseconds) triples in launch
 * order; *count receives the number recorded.  Arrays are HOST memory. */
int mrcqr_profile_end(int max_records, int32_t* stage, int32_t* level, float* ms, int32_t* count);

/* Releases per-stream status records.  Optional at exit. */
int mrcqr_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* MRCQR_H */
