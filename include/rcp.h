/*
 * rcp.h -- C ABI of the GB300 randomized CP decomposition library (librcp.so).
 *
 * The library computes the randomized CP decomposition of Erichson, Manohar,
 * Brunton & Kutz ("Randomized CP Tensor Decomposition", arXiv 1703.09074):
 *
 *   1. rcp_sketch   -- Algorithm 1 steps (4)-(12): for mode n, the sketch
 *                      Y = T_(n) Omega_n with a Gaussian test matrix of
 *                      l_n = min(R + p, I_n, J_n) columns (Eq. sampleMatrix),
 *                      q normalised power iterations (Eq. IMPsampleMatrix,
 *                      Algorithm 1 steps 7-11) and the QR Y = Q_n R.
 *   2. rcp_compress -- Algorithm 1 step (13): T_{n+1} = T_n x_n Q_n^T
 *                      (the n-mode product of Definition 1).
 *   3. rcp_als      -- Algorithm 2 steps (2)-(11): CP-ALS on the compressed
 *                      tensor B with the Khatri-Rao pseudo-inverse
 *                      (Definition 2), column normalisation, and the fit
 *                      test of Section 3.3.
 *   4. rcp_project  -- Algorithm 2 steps (12)-(13) / Eq. (qbs): A_n = Q_n Atilde_n,
 *                      re-normalised, with lambda updated.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Modes are numbered 1..N as in the paper.
 * - Tensors use the Kolda & Bader layout: element (i_1, ..., i_N) sits at
 *   linear index i_1 + I_1 (i_2 + I_2 (i_3 + ...)) -- mode 1 fastest.  A
 *   C-contiguous array of shape (I_N, ..., I_1) holds exactly these bytes.
 * - Matrices (Q_n, A_n, Atilde_n) are FP64, column-major, leading dimension
 *   equal to their row count.
 * - Device pointers are CUDA device addresses on the device that was current
 *   when the plan was created; host pointers are ordinary process memory.
 * - The caller owns the input tensor and every output buffer; the plan owns
 *   its workspace (allocated once in rcp_plan, freed in rcp_plan_destroy) and
 *   borrows the CUDA stream given to rcp_plan.  Work is enqueued on that
 *   stream and is asynchronous unless an entry point says it synchronises.
 *   The input tensor must stay valid until the enqueued work completes.
 * - Argument errors are returned synchronously and enqueue nothing.  Errors
 *   detected on the device (non-finite values, a singular Gram matrix that
 *   even the shifted fallback cannot factor, a bounded wait that ran out) are
 *   recorded in a device status word and returned by the next synchronising
 *   call (rcp_result, rcp_last_error, or an rcp_als call with host outputs).
 * - A plan is not thread-safe; use one plan per host thread.
 */
#ifndef RCP_H
#define RCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rcp_plan_s* rcp_plan_t;

typedef enum {
  RCP_OK = 0,
  RCP_EINVAL = 1,      /* invalid argument or configuration                       */
  RCP_ENOMEM = 2,      /* device or pinned-host allocation failed                  */
  RCP_ECUDA = 3,       /* a CUDA runtime call failed                               */
  RCP_ESINGULAR = 4,   /* a Gram matrix could not be factored even with a shift    */
  RCP_ENAN = 5,        /* a non-finite value reached a reduction                   */
  RCP_ETIMEOUT = 6,    /* a bounded device-side wait ran out                       */
  RCP_EORDER = 7,      /* entry points called out of the order of Algorithm 1      */
  RCP_ENOTCONV = 8     /* informational: ALS stopped at max_iters                  */
} rcp_status;

typedef enum {
  RCP_DTYPE_F64 = 0,
  RCP_DTYPE_F32 = 1
} rcp_dtype;

typedef enum {
  /* Every step in FP64 on the CUDA cores (the plain method). */
  RCP_PREC_F64 = 0,
  /* Tensor sweeps (sketch, power iterations, mode products) on the tensor
   * cores with FP32 accumulation; QR of each sketch and the R x R Gram solves
   * of ALS stay in FP64.  Working tensors T_2..T_N and B are FP32. */
  RCP_PREC_MIXED = 1
} rcp_precision;

/* Informational bits returned in rcp_result.info. */
enum {
  RCP_INFO_SHIFTED_QR = 1,     /* a sketch or power-iteration Gram needed the shifted fallback */
  RCP_INFO_ALS_REGULARISED = 2, /* an ALS Gram solve needed a diagonal shift                   */
  RCP_INFO_LEARNED_INIT = 4     /* ALS started from the warm-start network's factors          */
};

/* Flags for rcp_config.flags. */
enum {
  RCP_FLAG_HOST_STAGING = 1,   /* reserve device buffers so rcp_decompose_host can run  */
  RCP_FLAG_NO_SHIFT = 2,       /* no shifted-CholeskyQR fallback: a sketch whose Gram
                                  needs the shift (numerically rank-deficient Y) sets
                                  RCP_ESINGULAR instead of RCP_INFO_SHIFTED_QR        */
  RCP_FLAG_MODE_OVERSAMPLE = 4, /* use rcp_config.mode_oversample[n-1] as p for mode n
                                  (the remark after Algorithm 1)                       */
  RCP_FLAG_LU_NORM = 8,        /* normalise the power iterations with the pivoted LU
                                  factor of Algorithm 1 steps 8-9 (P L of Y = P L U)
                                  instead of CholeskyQR: the same spans, a different
                                  basis until the final QR of step 12                  */
  RCP_FLAG_INDEPENDENT = 16    /* the setting of Theorem 1: every mode's range finder
                                  (steps 5-12) reads the unfolding X_(n) of the input
                                  itself, not the partly compressed T_n, with
                                  l_n = min(R + p_n, I_n, prod of the other I_m);
                                  rcp_sketch then needs X for every mode, and the
                                  mode products of step 13 are unchanged            */
};

/* Initial factors of the stage-2 solver on B (Algorithm 2 step 2, Algorithm 3
 * step 2). */
typedef enum {
  RCP_INIT_RANDN = 0,   /* seeded N(0,1) factors for modes 2..N (the default)       */
  RCP_INIT_LEARNED = 1, /* the warm-start network's factors (rcp_set_warm_start; the
                           precision form, 3-way, l_n <= 24, R <= 16), else seeded   */
  RCP_INIT_EIG = 2      /* the leading R eigenvectors of B_(n) B_(n)^T, n = 2..N     */
} rcp_init;

/* Stage-2 solver on the compressed tensor B. */
typedef enum {
  RCP_SOLVER_ALS = 0,   /* CP-ALS, Algorithm 2                                       */
  RCP_SOLVER_BCD = 1    /* rank-one deflation by block coordinate descent, Algorithm 3 */
} rcp_solver;

#define RCP_MAX_NDIM 8
#define RCP_MAX_L 64      /* largest sketch width l_n = R + p supported */
#define RCP_MAX_RANK 64   /* largest target rank R supported            */

typedef struct {
  int32_t ndim;                  /* N, 2..RCP_MAX_NDIM                               */
  int64_t dims[RCP_MAX_NDIM];    /* I_1..I_N (each >= 1)                             */
  int32_t in_dtype;              /* rcp_dtype of the input tensor X                  */
  int32_t rank;                  /* target rank R, 1..RCP_MAX_RANK                   */
  int32_t oversample;            /* p >= 0; l_n = min(R + p, I_n, J_n) <= RCP_MAX_L   */
  int32_t power_iters;           /* q >= 0                                           */
  double tol;                    /* ALS stops when |rho_j - rho_{j-1}| < tol         */
  int32_t max_iters;             /* ALS sweep cap, >= 1                              */
  uint64_t seed;                 /* key of the counter-based random streams          */
  int32_t precision;             /* rcp_precision                                    */
  int32_t flags;                 /* RCP_FLAG_* bits                                  */
  int32_t init;                  /* rcp_init (0 = seeded N(0,1))                     */
  int32_t solver;                /* rcp_solver (0 = ALS)                             */
  int32_t skip_modes;            /* bit n-1 set: mode n is not compressed (Q_n = I,
                                    l_n = I_n <= RCP_MAX_L); the remark after
                                    Algorithm 1 lets the user choose the modes     */
  int32_t mode_oversample[RCP_MAX_NDIM]; /* p_n per mode with RCP_FLAG_MODE_OVERSAMPLE */
  int64_t wait_budget;           /* clock cycles each grid-barrier wait of the
                                    multi-CTA ALS kernel may spin before it records
                                    RCP_ETIMEOUT and the kernel leaves; 0 = the
                                    default (2^31 cycles, about one second)        */
} rcp_config;

/* Results of one decomposition, filled by rcp_result / rcp_decompose_host. */
typedef struct {
  double fit;             /* rho of Section 3.3 on the compressed tensor, last sweep    */
  int32_t iters;          /* ALS sweeps run                                             */
  int32_t info;           /* RCP_INFO_* bits                                            */
  double norm_x2;         /* |X|_F^2 (accumulated by the mode-1 sketch sweep)           */
  double norm_b2;         /* |B|_F^2                                                    */
  double rel_err;         /* |X - Xhat|_F / |X|_F = sqrt((|X|^2 - rho |B|^2) / |X|^2)   */
  int32_t device_status;  /* rcp_status recorded on the device                          */
  int32_t widths[RCP_MAX_NDIM]; /* l_1..l_N                                             */
} rcp_result;

/* Create a plan for one tensor shape and parameter set (Algorithm 2 "Require"
 * and "Optional" lines: tensor, target rank R, oversampling p, power
 * iterations q; plus the ALS tolerance and cap of Section 3.3).
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Allocates the whole workspace on the current device; returns RCP_EINVAL
 * for an unsupported configuration and RCP_ENOMEM when allocation fails.
 * *out is set only on success. */
rcp_status rcp_plan(const rcp_config* cfg, void* stream, rcp_plan_t* out);

/* Free the plan's workspace.  Synchronises the plan's stream first.
 * NULL is accepted and ignored. */
rcp_status rcp_plan_destroy(rcp_plan_t plan);

/* Sketch width l_n of 1-based mode n (Algorithm 1 step 3, capped as in
 * rcp_config.oversample), or -1 for an invalid plan or mode. */
int32_t rcp_width(rcp_plan_t plan, int32_t mode);

/* Algorithm 1 steps (4)-(12) for 1-based mode n: sketch the current tensor
 * T_n (X itself when n = 1), run q power iterations, orthonormalise, and keep
 * Q_n (I_n x l_n) in the plan.
 * X: device pointer to the input tensor (read when n = 1; ignored and may be
 *    NULL otherwise).
 * Q_out: optional device pointer receiving a copy of Q_n, I_n x l_n,
 *    column-major FP64; NULL skips the copy.
 * Order: n = 1 first, and n > 1 only after rcp_compress(n - 1); otherwise
 * RCP_EORDER.  Asynchronous. */
rcp_status rcp_sketch(rcp_plan_t plan, const void* X, int32_t mode, double* Q_out);

/* Algorithm 1 step (13): T_{n+1} = T_n x_n Q_n^T for 1-based mode n, after
 * rcp_sketch(n) (else RCP_EORDER).  X as in rcp_sketch.  After mode N the
 * plan holds the compressed tensor B (l_1 x ... x l_N).  Asynchronous. */
rcp_status rcp_compress(rcp_plan_t plan, const void* X, int32_t mode);

/* Replace the seeded N(0,1) initial factors of ALS (used when this is never
 * called) by caller-supplied ones.  At_dev[n-1] for n = 2..N: device pointer
 * to an l_n x R column-major FP64 matrix (At_dev[0] is ignored and may be
 * NULL).  The factors are copied on the stream; the pointers may be released
 * once that copy completes.  Applies to the next rcp_als call only. */
rcp_status rcp_als_init(rcp_plan_t plan, const double* const* At_dev);

/* The stage-2 solver on the compressed tensor B, from the initial factors that
 * rcp_config.init selects (seeded N(0,1), or Algorithm 2 step 2's eigenvectors
 * of B_(n) B_(n)^T; rcp_als_init overrides both for one call).
 * RCP_SOLVER_ALS -- Algorithm 2 steps (3)-(11): ALS sweeps over modes 1..N,
 *   each solving A_n = B_(n) (KR of the others) (Hadamard product of their
 *   Grams)^-1 and normalising columns (lambda from mode N), until the fit
 *   change falls below tol or max_iters sweeps have run.
 * RCP_SOLVER_BCD -- Algorithm 3 steps (3)-(15): for r = 1..R, rank-one sweeps
 *   a_n = Y_(n) (KR of the other a_m) / prod (a_m^T a_m) on the residual Y of
 *   the components already found (never formed: Section 3.2.2's residual-free
 *   MTTKRP), each component until its fit changes by less than tol or after
 *   max_iters sweeps; iters_host then counts the sweeps of all components.
 * Requires rcp_compress(N) (else RCP_EORDER).
 * lambda_host (R doubles), fit_host, iters_host: optional host outputs; when
 * any is non-NULL the call synchronises the stream and returns the device
 * status (RCP_ENOTCONV when the cap was reached without meeting tol). */
rcp_status rcp_als(rcp_plan_t plan, double* lambda_host, double* fit_host, int32_t* iters_host);

/* Algorithm 2 steps (12)-(13): A_n = Q_n Atilde_n for every mode, columns
 * re-normalised and lambda_r multiplied by the removed norms.
 * A_dev: host array of N device pointers, A_dev[n-1] -> I_n x R column-major
 * FP64 output.  lambda_dev: device pointer to R doubles (output).
 * Requires rcp_als (else RCP_EORDER).  Asynchronous. */
rcp_status rcp_project(rcp_plan_t plan, double* const* A_dev, double* lambda_dev);

/* All of the above in order for modes 1..N (asynchronous).  Arguments as in
 * rcp_sketch (X) and rcp_project (A_dev, lambda_dev). */
rcp_status rcp_decompose(rcp_plan_t plan, const void* X, double* const* A_dev, double* lambda_dev);

/* End-to-end call on host buffers: copies X_host (pinned or pageable host
 * memory, Kolda layout, cfg.in_dtype) to the device, runs rcp_decompose,
 * and copies the factors and lambda back.  A_host: host array of N host
 * pointers (I_n x R column-major FP64 each); lambda_host: R doubles;
 * res: optional result record.  Requires RCP_FLAG_HOST_STAGING in the plan's
 * flags (else RCP_EINVAL).  Synchronises. */
rcp_status rcp_decompose_host(rcp_plan_t plan, const void* X_host, double* const* A_host,
                              double* lambda_host, rcp_result* res);

/* Synchronise the plan's stream and fill *out (may be NULL to only check).
 * Returns the device status. */
rcp_status rcp_result_get(rcp_plan_t plan, rcp_result* out);

/* Copy the compressed tensor B (FP64, Kolda layout, l_1 x ... x l_N) to the
 * device buffer B_dev.  Requires rcp_compress(N).  Asynchronous. */
rcp_status rcp_get_core(rcp_plan_t plan, double* B_dev);

/* Copy the compressed-space factors Atilde_n (l_n x R column-major FP64, last
 * ALS state) to At_dev[n-1] (device pointers) and lambda (R doubles) to
 * lambda_dev (may be NULL).  Requires rcp_als.  Asynchronous. */
rcp_status rcp_get_compressed_factors(rcp_plan_t plan, double* const* At_dev, double* lambda_dev);

/* Synchronise and return the device status word (also stored in *device_status
 * when non-NULL). */
rcp_status rcp_last_error(rcp_plan_t plan, int32_t* device_status);

/* Static description of a status code. */
const char* rcp_status_str(rcp_status s);

/* Kernel classes timed by the profiling entry points. */
typedef enum {
  RCP_KT_SKETCH = 0,   /* Y = T_(n) Omega_n sweep (Algorithm 1 step 6)                */
  RCP_KT_APPLY = 1,    /* Y = T_(n) W sweep of a power iteration (step 10)            */
  RCP_KT_PROJECT = 2,  /* W = T_(n)^T Q sweep of a power iteration (step 9)           */
  RCP_KT_TTM = 3,      /* T_{n+1} = T_n x_n Q_n^T (step 13)                           */
  RCP_KT_ALS = 4,      /* every ALS kernel (Algorithm 2 steps 3-11)                   */
  RCP_KT_ALL = 5,      /* read-only: all kernels the library launched                 */
  RCP_KT_COUNT = 6
} rcp_kernel_kind;

/* Start (enable != 0) or stop recording CUDA events on the plan's stream
 * around every sweep launch; enabling clears earlier records.  Launches are
 * counted whether or not events are recorded.  Not a method step (the paper
 * has no counterpart): it exists to measure the kernels. */
rcp_status rcp_profile_enable(rcp_plan_t plan, int32_t enable);

/* Synchronise and report, for kernel class `kind` in 1-based mode `mode`
 * (0 = all modes), the number of launches and their summed device time in
 * milliseconds since the last rcp_profile_enable(plan, 1).  For RCP_KT_ALL
 * only `launches` is meaningful (total kernels launched by the library on
 * this plan).  Either output may be NULL. */
rcp_status rcp_profile_read(rcp_plan_t plan, int32_t kind, int32_t mode, int64_t* launches,
                            double* total_ms);

/* Test-matrix generator (Section 3.1: Gaussian entries for Omega_n), exposed
 * so that its counter-based stream can be checked against an independent
 * implementation.  Writes out_dev[k] for k < count: the element (first + k) of
 * the FP64 normal stream (seed, stream, purpose) -- Philox4x32-10 counter
 * (g mod 2^32, g div 2^32, stream, purpose), g = element div 2, key (seed lo,
 * seed hi), Box-Muller on 53-bit uniforms.  words_dev (optional, 4 uint32 per
 * counter for counters first/2 .. (first+count-1)/2) receives the raw Philox
 * output.  f32_out_dev (optional): the reduced-precision stream (four normals
 * per counter) evaluated on the device.  cuda_stream: cudaStream_t.
 * Asynchronous. */
rcp_status rcp_test_normals(uint64_t seed, uint32_t stream, uint32_t purpose, int64_t first,
                            int64_t count, double* out_dev, uint32_t* words_dev,
                            float* f32_out_dev, void* cuda_stream);

/* Test hook: the device arithmetic building blocks, elementwise on n inputs
 * (device arrays of doubles; n = 0 is a no-op).  op:
 *   RCP_ARITH_DW_ADD   x + y  in double word (two FP32 numbers hi + lo)
 *   RCP_ARITH_DW_MUL   x * y  in double word
 *   RCP_ARITH_DW_RCP   1 / x  in double word (x > 0, normal FP32 range)
 *   RCP_ARITH_DW_SQRT  sqrt x in double word (x > 0)
 *   RCP_ARITH_RSQRT64  1 / sqrt x in FP64 (x > 0)
 * The double-word ops first round each input to its nearest double word
 * (hi = the FP32 rounding of x, lo = the FP32 rounding of x - hi); the result's
 * components come back as doubles in out_hi_dev / out_lo_dev (out_lo_dev = 0
 * for RSQRT64).  These operations carry the Gram solves of Algorithm 2 and the
 * factorisations of the QR steps of Algorithm 1.  y_dev is read by the binary
 * ops only.  Errors: RCP_EINVAL for an unknown op, n < 0 or a missing array.
 * cuda_stream: cudaStream_t.  Asynchronous. */
enum rcp_arith_op {
  RCP_ARITH_DW_ADD = 0,
  RCP_ARITH_DW_MUL = 1,
  RCP_ARITH_DW_RCP = 2,
  RCP_ARITH_DW_SQRT = 3,
  RCP_ARITH_RSQRT64 = 4
};
rcp_status rcp_test_arith(int32_t op, const double* x_dev, const double* y_dev, int64_t n,
                          double* out_hi_dev, double* out_lo_dev, void* cuda_stream);

/* FP64 (fp64 = 1) or FP32 (fp64 = 0) FMA rate of the current device in TFLOP/s
 * (2 FLOP per FMA): 8 independent FMA chains per thread on 8 (FP64) or 16
 * (FP32) CTAs of 256 threads per SM, the second of two launches timed with CUDA
 * events on cuda_stream.  This is the arithmetic peak that the FP64 path's
 * sweeps are measured against (the paper has no counterpart: it is a
 * measurement aid).  Synchronises the stream.  Errors: RCP_EINVAL for a null
 * tflops or fp64 not 0/1; RCP_ECUDA. */
rcp_status rcp_measure_fma_rate(int32_t fp64, double* tflops, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched form: many tensors of uneven shapes decomposed together.  Every
 * step of Algorithm 1 (per mode), Algorithm 2 and the recovery of Eq. (qbs)
 * runs as one launch over all tensors (persistent kernels pulling
 * (tensor, tile) work items largest tensor first; one CTA per tensor for the
 * FP64 CholeskyQR2 of each sketch and for the ALS of each compressed tensor),
 * and the whole sequence is captured into one CUDA graph on the first run and
 * replayed afterwards.
 * ---------------------------------------------------------------------- */
typedef struct rcp_batched_s* rcp_batched_t;

/* Plan `count` decompositions.  cfgs[b] describes tensor b; all must have the
 * same ndim and power_iters, in_dtype RCP_DTYPE_F32, precision
 * RCP_PREC_MIXED, rank <= 32 and widths l_n <= 32.  Allocates one workspace
 * arena for the batch; stream as in rcp_plan.  RCP_EINVAL / RCP_ENOMEM. */
rcp_status rcp_plan_batched(const rcp_config* cfgs, int32_t count, void* stream,
                            rcp_batched_t* out);

/* Decompose every tensor: X_dev[b] is a device pointer to tensor b (Kolda
 * layout, FP32), valid until the run completes.  The first call captures the
 * launch sequence into a CUDA graph; later calls replay it (the pointers may
 * change between calls; each call waits for the previous run to finish before
 * updating them).  Asynchronous otherwise. */
rcp_status rcp_batched_run(rcp_batched_t plan, const void* const* X_dev);

/* Choose the launch and tile shapes of the batched sweeps by timing complete
 * batch runs on X_dev: a coordinate search, two passes, over
 *   choice[0]  persistent CTAs per SM of the row sweeps     (1, 2, 4, 8)
 *   choice[1]  persistent CTAs per SM of the column sweeps  (1, 2, 4, 8)
 *   choice[2]  loads in flight per thread in the row sweeps (4, 8)
 *   choice[3]  256-column blocks per column work item       (1, 2, 4, 8)
 * None of them changes the order of any sum, so every choice gives bit-identical
 * results.  Keeps the fastest for later runs and writes it to choice[0..3] when
 * choice is not NULL (4 int32).  Synchronises.  RCP_EINVAL / RCP_ECUDA. */
rcp_status rcp_batched_autotune(rcp_batched_t plan, const void* const* X_dev, int32_t* choice);

/* Results of tensor `index` after a run: factors A_n (A_dev[n-1], device,
 * I_n x R column-major FP64, entries may be NULL), lambda (device, R doubles,
 * may be NULL) and the result record.  Synchronises the stream; returns the
 * tensor's device status. */
rcp_status rcp_batched_result(rcp_batched_t plan, int32_t index, double* const* A_dev,
                              double* lambda_dev, rcp_result* res);

/* Intermediates of tensor `index` after a run, for checking each step of the
 * method: the bases Q_n of Algorithm 1 step 12 (Q_dev[n-1], I_n x l_n
 * column-major FP64), the compressed tensor B of step 13 (B_dev, FP64, Kolda
 * layout l_1 x ... x l_N), and the ALS factors Atilde_n of Algorithm 2 step 11
 * with their lambda (At_dev[n-1], l_n x R column-major FP64; lambda_t_dev, R
 * doubles).  Every pointer (and every array entry) may be NULL.  Asynchronous
 * on the plan's stream. */
rcp_status rcp_batched_intermediates(rcp_batched_t plan, int32_t index, double* const* Q_dev,
                                     double* B_dev, double* const* At_dev, double* lambda_t_dev);

/* Free the batch plan (synchronises first).  NULL is ignored. */
rcp_status rcp_batched_destroy(rcp_batched_t plan);

/* Allocation-free mode-1 range finder.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code
 * that runs where cudaMalloc is forbidden or unsafe (inside another
 * framework's memory budget that is fixed at start-up, inside a region whose
 * allocations the host application tracks and refuses, or on a teardown path),
 * and therefore cannot create an rcp_plan, which allocates its workspace.
 *
 * It computes what rcp_sketch(plan, X, 1, Q_out) computes for a plan with
 * power_iters = 0 and the FP64 path: Y = X_(1) Omega_1 with the Gaussian test
 * matrix of seed `seed`, then Q_1 = the thin QR factor of Y with a positive
 * diagonal of R (CholeskyQR2, shifted fallback).  X_dev: device tensor in the
 * Kolda layout (in_dtype RCP_DTYPE_F32 or RCP_DTYPE_F64), dims[0..ndim-1] =
 * I_1..I_N (host array).  Q_dev: device output, I_1 x l column-major FP64 with
 * l = min(rank + oversample, I_1, I_2 ... I_N).  status_dev: optional device
 * int32 that receives the device status (RCP_ENAN for non-finite input,
 * RCP_ESINGULAR for a sketch even the shift cannot factor).  stream:
 * cudaStream_t.  Asynchronous; calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Scratch: one file-scope device array of 4 MiB (2^19 doubles) per GPU that
 * loads the library, held until process exit, holding the split partials,
 * the sketch and the QR scratch.  Limit: I_1 * l <= 259052 (at least one
 * split must fit); larger sizes return RCP_EINVAL before any work.  The first
 * call on each device looks up the array's device address with
 * cudaGetSymbolAddress while that device is current; make that first call
 * outside any stream capture.  Every call on a device shares the same array
 * and leaves its contents behind (the status word is cleared at the start of
 * each call; partials and sketch are fully overwritten), so calls that
 * overlap on the GPU -- on different streams or host threads -- race and
 * must be serialised by the caller. */
rcp_status rcp_sketch_mode1_static(const void* X_dev, int32_t in_dtype, int32_t ndim,
                                   const int64_t* dims, int32_t rank, int32_t oversample,
                                   uint64_t seed, double* Q_dev, int32_t* status_dev,
                                   void* stream);

/* ------------------------------------------------------------------------
 * Learned warm start for CP-ALS (Algorithm 2 steps 1-2 choose the initial
 * factors; Section 3.2 names eigenvector or random initialisation).  This is
 * an addition to the paper: a 3-layer perceptron maps the compressed tensor
 * B (3-way, l_n <= 24, R <= 16) to initial factors.
 *
 * Input encoding: B in its canonical basis -- for each mode the eigenvectors
 * U_n of B_(n) B_(n)^T (descending eigenvalues, each vector's largest-
 * magnitude entry positive) -- i.e. G = B x_1 U_1^T x_2 U_2^T x_3 U_3^T / |B|_F,
 * zero-padded to 24 x 24 x 24, index i1 + 24 i2 + 576 i3 ("x rows", FP32,
 * RCP_MLP_IN floats per sample).  Output Y: 3 x 24 x 16, index
 * n * 384 + i * 16 + r ("y rows", RCP_MLP_OUT floats), read as a correction
 * in the canonical basis: initial A_n = U_n (E + Y_n) on l_n rows and R
 * columns, E = the first R unit vectors (Y = 0 gives the eigenvector
 * initialisation).  meta rows: int32 (l1, l2, l3, R) per sample; all zeros
 * marks a sample the network does not serve.
 *
 * Network: x -> relu(W1 x + b1) (512) -> relu(W2 h1 + b2) (512) -> W3 h2 + b3,
 * BF16 weights and activations as tensor-core operands, FP32 accumulation,
 * FP32 master parameters in the flat order W1 (512 x 13824, row-major), b1,
 * W2 (512 x 512), b2, W3 (1152 x 512), b3.  Adam updates the master copy.
 * ---------------------------------------------------------------------- */
#define RCP_WS_LPAD 24
#define RCP_WS_RPAD 16
#define RCP_MLP_IN 13824
#define RCP_MLP_HIDDEN 512
#define RCP_MLP_OUT 1152

typedef struct rcp_mlp_s* rcp_mlp_t;

/* Number of FP32 master parameters (7,930,032). */
int64_t rcp_mlp_param_count(void);

/* Create a network that processes up to `batch` samples per pass (multiple of
 * 128, <= 65536), with seeded initial weights W1, W2 ~ U(-1/sqrt(fan_in),
 * 1/sqrt(fan_in)), W3 and biases zero (the untrained network outputs Y = 0),
 * Adam moments zero.  stream: cudaStream_t borrowed for all
 * of the network's work.  RCP_EINVAL / RCP_ENOMEM / RCP_ECUDA. */
rcp_status rcp_mlp_create(int32_t batch, uint64_t seed, void* stream, rcp_mlp_t* out);
rcp_status rcp_mlp_destroy(rcp_mlp_t net);

/* Copy the master parameters, the Adam moments and the step count to host
 * buffers of rcp_mlp_param_count() floats (any pointer may be NULL), or load
 * them (checkpoint / resume).  Both synchronise the stream. */
rcp_status rcp_mlp_get_params(rcp_mlp_t net, float* params, float* adam_m, float* adam_v,
                              int64_t* step);
rcp_status rcp_mlp_set_params(rcp_mlp_t net, const float* params, const float* adam_m,
                              const float* adam_v, int64_t step);

/* Forward pass of `count` x rows (device, count <= batch); train != 0 keeps
 * what the backward pass needs.  y_dev: optional device output, count y rows.
 * Asynchronous. */
rcp_status rcp_mlp_forward(rcp_mlp_t net, const float* x_dev, int32_t count, int32_t train,
                           float* y_dev);

/* Backward pass of the last training forward: dy_dev holds batch y rows of
 * dLoss/dY (rows >= count zero).  Writes the gradients of every parameter
 * (flat order above) to grad_dev when not NULL.  RCP_EORDER without a
 * training forward.  Asynchronous. */
rcp_status rcp_mlp_backward(rcp_mlp_t net, const float* dy_dev, float* grad_dev);

/* One Adam step (Kingma & Ba) with the gradients of the last backward pass. */
rcp_status rcp_mlp_adam(rcp_mlp_t net, float lr, float beta1, float beta2, float eps);

/* Device status word of the network (RCP_ETIMEOUT if a tensor-core pipeline
 * wait gave up).  Synchronises. */
rcp_status rcp_mlp_status(rcp_mlp_t net);

/* x rows and canonical bases of `count` padded compressed tensors:
 * Bpad_dev count x 24^3 FP32 (index i1 + 24 i2 + 576 i3), meta_dev count x 4;
 * x_dev count x 24^3; U_dev count x 3 x 24 x 24 (U_n[i][j] at
 * ((b * 3 + n) * 24 + i) * 24 + j, column j = eigenvector j).  Asynchronous. */
rcp_status rcp_ws_canonicalize(const float* Bpad_dev, const int32_t* meta_dev, int32_t count,
                               float* x_dev, float* U_dev, void* stream);

/* Training loss of `count` y rows against targets t_dev (y-row layout: the
 * converged factors in the canonical basis, unit columns): after the
 * minimum-cost one-to-one matching of the R components (Hungarian method),
 * loss_b = (1/R) sum_r sum_n (1 - cos^2(E + Y_n column r, target column
 * match(r))).  Writes loss_dev[b] and dy_dev = scale * dloss_b/dY.  Async. */
rcp_status rcp_ws_loss(const float* y_dev, const float* t_dev, const int32_t* meta_dev,
                       int32_t count, float scale, float* dy_dev, float* loss_dev, void* stream);

/* forward (train), loss with scale 1/count, backward, Adam(lr, 0.9, 0.999,
 * 1e-8).  loss_dev: optional device output of the per-sample losses. */
rcp_status rcp_mlp_train_step(rcp_mlp_t net, const float* x_dev, const float* t_dev,
                              const int32_t* meta_dev, int32_t count, float lr, float* loss_dev);

/* Training data from a batch plan after a run: per tensor b the padded
 * compressed tensor (Bpad_dev, count x 24^3), meta (count x 4), x row
 * (count x 24^3), canonical bases (count x 3 x 24 x 24) and the converged
 * factors in the canonical basis with unit columns (t_dev, count x 1152).
 * Tensors the network does not serve (ndim != 3, l_n > 24, R > 16) get zero
 * meta.  Asynchronous on the plan's stream. */
rcp_status rcp_batched_export(rcp_batched_t plan, float* Bpad_dev, int32_t* meta_dev,
                              float* x_dev, float* U_dev, float* t_dev);

/* Start the ALS of every eligible tensor from the network's factors in later
 * runs (the captured graph gains the canonicalisation, the forward pass and
 * the factor construction); net = NULL restores the random initialisation.
 * Tensors the network does not serve, or whose predicted factors have a
 * non-finite or zero column, keep the random initialisation; the others set
 * RCP_INFO_LEARNED_INIT.  The network's batch must be >= the plan's count and
 * its stream is not used by the plan.  Synchronises. */
rcp_status rcp_batched_set_warm_start(rcp_batched_t plan, rcp_mlp_t net);

/* Start the stage-2 solver of a plan whose rcp_config.init is RCP_INIT_LEARNED
 * from the warm-start network's factors (the batched form's data path for the
 * plan's one compressed tensor: canonical basis, a forward pass of `net`,
 * A_n = U_n (E + Y_n)); a prediction with a non-finite or zero column falls back
 * to the seeded start.  The plan must be of the precision form, 3-way, with
 * l_n <= 24 and R <= 16 (else RCP_EINVAL); net = NULL detaches the network
 * (seeded start).  The network runs on the plan's stream and must stay alive
 * while the plan uses it.  The first call allocates the plan's warm-start
 * buffers and synchronises. */
rcp_status rcp_set_warm_start(rcp_plan_t plan, rcp_mlp_t net);

/* Synthetic CP tensor for training and benchmarking (no counterpart in the
 * method): X[i_1..i_N] = sum_r lambda_r prod_n A_n[i_n, r] + sigma z, z ~ N(0, 1)
 * from the counter-based stream (key = seed, counter = linear index,
 * purpose 3), written in the Kolda layout (FP32).  factors: host array of N
 * device pointers (A_n: I_n x R column-major FP32); lambda_dev: R FP32.
 * Asynchronous. */
rcp_status rcp_synth_cp(int32_t ndim, const int64_t* dims, int32_t rank,
                        const float* const* factors, const float* lambda_dev, float sigma,
                        uint64_t seed, float* X_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RCP_H */
