/*
 * sqsm.h -- C ABI of the GB300 parallel square-root smoothers.
 *
 * Implements the data-parallel hot path of "Parallel square-root statistical
 * linear regression for inference in nonlinear state space models"
 * (Yaghoobi, Corenflos, Hassan, Saerkkae; arXiv 2207.00426):
 *   - the square-root parallel Kalman filter (Sec. 3.1, Lemmas 1-2,
 *     Tables 1-3, Alg. 1) and RTS smoother (Sec. 3.2, Lemmas 3-4,
 *     Tables 4-5, Alg. 2) as associative scans whose operator uses Tria;
 *   - Taylor (Sec. 4.2) and cubature sigma-point (Sec. 4.3) statistical
 *     linear regression inside iterated posterior linearisation (Alg. 3);
 *   - the pseudo log-likelihood (Sec. 5.1) and its gradient through the
 *     fixed point of Alg. 3 (Sec. 5.2, eq. implicity_function_theorem,
 *     Alg. 4) by a reverse-mode adjoint.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - All array arguments are DEVICE pointers unless stated otherwise, in
 *   row-major order; matrices of one time step are contiguous.
 * - dtype selects the element type of every floating-point array argument:
 *   SQSM_F32 (float) or SQSM_F64 (double).  Log-likelihoods, gradients and
 *   model parameters are always double.
 * - "Lower factor" arguments are full nx x nx (or ny x ny) matrices whose
 *   strictly upper part is ignored on input and written as zero on output.
 * - Time indexing follows eq. linear-model: for t = 0..n-1, row t of the
 *   transition arrays holds (F_t, c_t, S_Lambda_t) of
 *   x_{t+1} = F_t x_t + c_t + q_t, and row t of the observation arrays holds
 *   (H_{t+1}, d_{t+1}, S_Omega_{t+1}, y_{t+1}).  State outputs have n+1 rows,
 *   k = 0..n (row 0 is the prior).
 * - Ownership: the caller owns every argument buffer.  The library never
 *   frees or retains caller memory beyond the call, and never synchronises
 *   the stream except where stated.  Work is enqueued on `stream`
 *   (a cudaStream_t passed as void*; NULL = legacy default stream).
 * - Alignment: every array pointer must be a multiple of its element size
 *   (4 bytes for float, 8 for double and for the double outputs, 4 for
 *   int); a misaligned pointer is an argument error.
 * - Errors: every call returns an sqsm_status.  Argument errors are detected
 *   on the host before anything is enqueued.  Conditions detected on the
 *   device (a non-finite output, a prior covariance that is not positive
 *   definite, an unsettled fixed point) are OR-ed into a device status word
 *   that sqsm_get_status() reads.  sqsm_last_error() gives the text of the
 *   last host-side error of a context.
 * - A context is not thread-safe; use one context per host thread.
 */
#ifndef SQSM_H
#define SQSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SQSM_OK = 0,
  SQSM_ERR_INVALID_ARG = 1,      /* null or misaligned pointer, bad
                                    size/stride/offsets/enum              */
  SQSM_ERR_UNSUPPORTED = 2,      /* (nx, ny) pair not compiled in            */
  SQSM_ERR_NOT_PD = 4,           /* device: a prior covariance given with
                                    sqsm_options.prior_covariance is not
                                    positive definite (its FP64 Cholesky
                                    met a non-positive pivot; the factor and
                                    the outputs it feeds are NaN)          */
  SQSM_ERR_NONFINITE = 8,        /* device: NaN/Inf in an output             */
  SQSM_ERR_CUDA = 16,            /* a CUDA runtime call failed               */
  SQSM_ERR_NO_MEMORY = 32,       /* workspace allocation failed              */
  SQSM_ERR_TOO_LARGE = 64,       /* problem exceeds a fixed-size buffer      */
  SQSM_ERR_NOT_CONVERGED = 128   /* device: sqsm_ipls_nll_grad's trajectory or
                                    adjoint had not settled to its tol      */
} sqsm_status;

typedef enum { SQSM_F32 = 0, SQSM_F64 = 1 } sqsm_dtype;

/* Linearisation rule of the SLR step (Sec. 4.2 / 4.3). */
typedef enum {
  SQSM_CUBATURE = 0,   /* third-degree spherical-radial rule, 2 nx points */
  SQSM_EXTENDED = 1,   /* first-order Taylor expansion at the mean         */
  SQSM_UNSCENTED = 2,  /* unscented transform, alpha = 1, beta = 0,
                          kappa = 1: 2 nx + 1 points, positive weights     */
  SQSM_GAUSS_HERMITE = 3   /* three-point Gauss-Hermite rule per dimension,
                              3^nx points (243 at nx = 5), two passes     */
} sqsm_linearization;

/* Compiled-in model families (a C ABI cannot carry device functions). */
typedef enum {
  SQSM_MODEL_CT_BEARINGS = 1,  /* coordinated turn, two bearing sensors:
                                  nx = 5, ny = 2, theta = (log sigma,
                                  log q_c, log q_omega)                   */
  SQSM_MODEL_POPULATION = 2,   /* stochastic Ricker model, Poisson counts
                                  (state-dependent observation noise):
                                  nx = ny = 1, theta = (log a, log b,
                                  log Q); dt and sensors unused; cubature
                                  or extended SLR; sqsm_ipls_smooth and
                                  sqsm_ipls_smooth_tol only               */
  SQSM_MODEL_CT_BEARINGS_R = 3 /* the coordinated-turn bearings model with
                                  one noise standard deviation per sensor
                                  (Sec. 6.4 estimates the first one,
                                  sqrt(R_11)): theta = (log sqrt(R_11),
                                  log q_c, log q_omega, log sqrt(R_22)),
                                  host double[4]; gradients double[4].
                                  Accepted wherever SQSM_MODEL_CT_BEARINGS
                                  is, which is the case R_11 = R_22       */
} sqsm_model_kind;

/* Coordinated-turn bearings-only model (Sec. 6.2): state
 * (p_x, p_y, v_x, v_y, omega), nx = 5; two bearings atan2(p_y - s_y,
 * p_x - s_x), ny = 2; additive process noise with covariance
 * q_c [[dt^3/3 I, dt^2/2 I], [dt^2/2 I, dt I]] on (p, v) and q_omega dt on
 * omega; bearing noise sigma^2 I.  theta = (log sigma, log q_c,
 * log q_omega) is passed separately (host double[3]); with
 * SQSM_MODEL_CT_BEARINGS_R the noise is diag(R_11, R_22) and theta has
 * four entries (see there). */
typedef struct {
  int kind;             /* sqsm_model_kind                          */
  double dt;            /* time step                                */
  double sensors[4];    /* s_x^1, s_y^1, s_x^2, s_y^2               */
} sqsm_model;

/* Scan shape.  Zero fields take defaults: leaf_chunk 3 when all leaf chunks
 * of a call fit one wave of 256 threads per SM, else 4; radix 0 folds upper
 * levels of more than 160000 items 4 per thread and scans smaller levels in
 * one-warp chunks of 32.
 *
 * autotune = 1 (with leaf_chunk = radix = 0): the first sqsm_ipls_smooth or
 * sqsm_ipls_nll_grad call of each workload shape (dtype, linearisation,
 * batch size, log2 of the total and of the longest sequence length) times
 * one IPLS iteration for each candidate scan shape on the caller's inputs
 * and stream, keeps the fastest for the context, then runs the call.  That
 * first call synchronises the stream and overwrites the outputs before
 * writing the final ones; later calls of the shape use the stored choice. */
typedef struct {
  int leaf_chunk;       /* time steps folded by one thread at the leaf  */
  int radix;            /* items folded by one thread at upper levels   */
  int use_graph;        /* 1: replay the IPLS iterations as a CUDA graph */
  int autotune;         /* 1: measure and keep the fastest scan shape   */
  int absolute;         /* 1: IPLS smooths each linearisation in the
                           printed absolute coordinates (c = z_bar - F m)
                           instead of deviations from the nominal
                           trajectory (default 0)                        */
  int prior_covariance; /* 1: the N0 argument of sqsm_lgssm_smooth,
                           sqsm_ipls_smooth, sqsm_ipls_smooth_tol and
                           sqsm_ipls_nll_grad holds prior covariances P0
                           (full nx x nx per sequence, lower triangle
                           read) instead of lower factors; each call
                           factors them on the GPU with an FP64 Cholesky
                           (N0 = chol(P0), written in the call's dtype)
                           before its scans.  A P0 that is not positive
                           definite sets SQSM_ERR_NOT_PD in the device
                           status word.  Default 0.                     */
  int refine;           /* mixed-precision refinement passes (0..2) of
                           every IPLS iteration's linear smoother: after
                           the smoother, the residual model about its
                           result is formed beyond the working precision
                           (its offsets c' = F dx + c - dx_k,
                           d' = d + H dx_k: in FP32 by compensated
                           TwoSum / Dot2 arithmetic, in FP64 in FP64;
                           rounded once) and smoothed again in the call's dtype,
                           the correction added to the trajectory.  Each
                           pass costs one more filter scan and a smoother
                           scan of the means alone (the factors do not
                           change; in FP32 with at most 64 sequences and
                           n_x >= 3 the filter scan's top levels too,
                           replayed from what
                           the first pass stores: about 3.4 MB at
                           n = 1e5); it removes most of the FP32 error of the linear
                           solve, which a non-converging Alg. 3 amplifies
                           from iteration to iteration.  Deviation
                           coordinates only (ignored with absolute).
                           Default 0.                                    */
  int textbook_slr;     /* 1: the cubature SLR of sqsm_ipls_smooth,
                           sqsm_ipls_smooth_tol and sqsm_ipls_smooth_std
                           evaluates each sigma point's function value in
                           absolute coordinates and subtracts the value at
                           the mean, as the regression formulas are
                           printed, instead of the cancellation-free
                           differences (bearings from atan2 of absolute
                           positions).  Less accurate in FP32 by design: a
                           comparator for the robustness experiment of
                           Sec. 6.  Default 0.                           */
  int max_group_steps;  /* > 0: sqsm_ipls_nll_grad evaluates a batch whose
                           total number of time steps exceeds this bound
                           in groups of consecutive sequences of at most
                           this many steps each, one group after another
                           (the sequences are independent, so the NLL and
                           the gradient are sums over the groups and the
                           changes maxima), and frees each group's
                           workspace before the next group's is made: the
                           call's device memory is then that of one
                           group, about 3.4 KB per time step in FP32 and
                           6.6 KB in FP64.  A grouped call runs without
                           graphs and synchronises the device between
                           groups; a sequence longer than the bound
                           returns SQSM_ERR_TOO_LARGE.  0 (default): the
                           whole batch at once.                          */
} sqsm_options;

typedef struct sqsm_ctx sqsm_ctx;

/* The scan shape (leaf_chunk, radix; radix 0 = the adaptive upper levels)
 * that IPLS calls on this context use for a batch of sequences with the
 * given host offsets (batch + 1 values) and dtype: the options', the
 * autotuned choice if one is stored, else the default.  No GPU work. */
int sqsm_scan_shape(sqsm_ctx* ctx, int dtype, int linearization, int64_t batch,
                    const int64_t* offsets, int* leaf_chunk, int* radix);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * The context owns scan workspaces, cached plans and captured graphs; they
 * are freed by sqsm_destroy.  Returns SQSM_ERR_CUDA if the device cannot be
 * used. */
int sqsm_create(sqsm_ctx** out, int device, const sqsm_options* opt);

/* Free a context and everything it owns (synchronises the device first).
 * NULL is accepted. */
int sqsm_destroy(sqsm_ctx* ctx);

/* Text of the last host-side error of ctx ("" if none).  The pointer stays
 * valid until the next call on ctx. */
const char* sqsm_last_error(const sqsm_ctx* ctx);

/* Synchronise ctx's device, read and clear the device status word: the OR
 * of the device-detected conditions since the last read -- SQSM_ERR_NONFINITE
 * (a kernel produced a non-finite filtered or smoothed mean or
 * log-likelihood), SQSM_ERR_NOT_PD (a prior covariance was not positive
 * definite), SQSM_ERR_NOT_CONVERGED (sqsm_ipls_nll_grad's fixed points had
 * not settled) -- or 0.  *status is host memory. */
int sqsm_get_status(sqsm_ctx* ctx, int* status);

/* Parallel square-root Kalman filter and RTS smoother on one linear-Gaussian
 * model (Alg. 1 then Alg. 2) plus its log-likelihood (Sec. 5.1).
 *
 *   nx, ny   state / observation dimensions (1 <= nx, ny <= 8; the
 *            compiled-in pairs are listed by sqsm_supported_shape).
 *   n        number of observations (n >= 1).
 *   F  [n][nx][nx], c [n][nx], SQ [n][nx][nx] lower: transition model;
 *   H  [n][ny][nx], d [n][ny], SR [n][ny][ny] lower: observation model;
 *            each with a per-step stride in elements (sF, sc, ...); a
 *            stride of 0 means the same matrix for every step.
 *   m0 [nx], N0 [nx][nx] lower: prior x_0 ~ N(m0, N0 N0^T).
 *   y  [n][ny] observations.
 *   mf, Nf   [n+1][nx], [n+1][nx][nx]: filtering means / lower factors
 *            (either may be NULL if not wanted).
 *   ms, Ns   [n+1][nx], [n+1][nx][nx]: smoothing means / lower factors.
 *   loglik   device double[1]: sum_k log N(y_k; H m^-_k + d, S_k), or NULL.
 * Arrays must not overlap outputs.  Uses ctx workspace (allocated on first
 * use of a shape). */
int sqsm_lgssm_smooth(sqsm_ctx* ctx, int dtype, int nx, int ny, int64_t n,
                      const void* F, int64_t sF, const void* c, int64_t sc,
                      const void* SQ, int64_t sSQ, const void* H, int64_t sH,
                      const void* d, int64_t sd, const void* SR, int64_t sSR,
                      const void* m0, const void* N0, const void* y,
                      void* mf, void* Nf, void* ms, void* Ns, double* loglik,
                      void* stream);

/* Iterated posterior linearisation smoother (Alg. 3) on `batch`
 * independent sequences of a compiled-in model, in one set of launches.
 *
 *   model, theta   model description and host parameters (double[3];
 *                  double[4] for SQSM_MODEL_CT_BEARINGS_R).
 *   linearization  sqsm_linearization.
 *   M              number of iterations (>= 1).
 *   batch          number of sequences (>= 1).
 *   offsets        HOST int64[batch+1], offsets[0] = 0, increasing:
 *                  sequence b has n_b = offsets[b+1]-offsets[b] >= 1
 *                  observations, rows offsets[b].. of y.  Its states are
 *                  rows offsets[b]+b .. offsets[b+1]+b of the state arrays
 *                  (n_b + 1 rows).
 *   y              [offsets[batch]][ny].
 *   m0, N0         [batch][nx], [batch][nx][nx] lower: priors.
 *   init_ms, init_Ns  initial nominal trajectory in state layout, or both
 *                  NULL for the prior broadcast to every step.
 *   ms, Ns         outputs, state layout: smoothing means / lower factors
 *                  after iteration M.
 *   loglik         device double[batch]: pseudo log-likelihood of each
 *                  sequence (filter of iteration M, Sec. 5.1), or NULL.
 * The plan and graph for an (offsets, pointers, M) combination are cached in
 * ctx; the first call for a combination builds them. */
int sqsm_ipls_smooth(sqsm_ctx* ctx, int dtype, const sqsm_model* model,
                     const double* theta, int linearization, int M,
                     int64_t batch, const int64_t* offsets, const void* y,
                     const void* m0, const void* N0, const void* init_ms,
                     const void* init_Ns, void* ms, void* Ns, double* loglik,
                     void* stream);

/* Alg. 3 in the standard (covariance) form: the left columns of Tables
 * 1-5 for the parallel filter and smoother and the covariance form of the
 * cubature SLR (Sec. 4.1), otherwise as sqsm_ipls_smooth (same batch layout,
 * deviation coordinates, prior broadcast as the initial trajectory).  It is
 * the comparator of the square-root form's numerical stability (Sec. 6): in
 * FP32 its covariances can lose positive definiteness, which shows as NaN in
 * ms / loglik and SQSM_ERR_NONFINITE in the status word.
 *   P0  [batch][nx][nx]: prior covariances (full, symmetric).
 *   Ps  output covariances P^s_k (full, symmetric), state layout.
 * Cubature or extended SLR; the context's `absolute` option selects the
 * printed absolute coordinates; scan levels fold 4 items per thread; no
 * graph capture. */
int sqsm_ipls_smooth_std(sqsm_ctx* ctx, int dtype, const sqsm_model* model,
                         const double* theta, int linearization, int M,
                         int64_t batch, const int64_t* offsets, const void* y,
                         const void* m0, const void* P0, void* ms, void* Ps,
                         double* loglik, void* stream);

/* sqsm_ipls_smooth run until convergence (Alg. 3 "until convergence"):
 * iterations continue while the largest change of any smoothing mean
 * component between consecutive iterations, max_k |m^(i)_k - m^(i-1)_k|,
 * is >= tol, at most max_iters times (>= 1; the change after iteration 1 is
 * measured from the initial trajectory).  iters_done: device int, the
 * number of iterations run.  ms, Ns, loglik: as sqsm_ipls_smooth after the
 * last iteration.  With use_graph the whole loop is one CUDA graph whose
 * iterations are the body of a conditional WHILE node, so the host never
 * waits; without it the host reads a continue flag after every iteration
 * (one stream synchronisation per iteration).  The change is compared in
 * FP32.  Errors as sqsm_ipls_smooth; SQSM_ERR_INVALID_ARG also for tol < 0
 * or a null iters_done. */
int sqsm_ipls_smooth_tol(sqsm_ctx* ctx, int dtype, const sqsm_model* model,
                         const double* theta, int linearization, int max_iters,
                         double tol, int64_t batch, const int64_t* offsets,
                         const void* y, const void* m0, const void* N0,
                         const void* init_ms, const void* init_Ns, void* ms,
                         void* Ns, double* loglik, int* iters_done, void* stream);

/* Negative pseudo log-likelihood and its gradient with respect to theta
 * through the fixed point of Alg. 3 (Sec. 5.2: eq. implicity_function_theorem
 * and Alg. 4, in reverse / vector-Jacobian form), summed over the batch.
 *
 * Runs M iterations of Alg. 3 (as sqsm_ipls_smooth; M = 0 takes
 * init_ms/init_Ns as the trajectory), linearises once more at the result
 * n* and filters/smooths that model (Sec. 5.1: nll = -sum_b l_b of this
 * last filter), then iterates the adjoint fixed point
 *   lambda <- (dKS/dn)^T lambda + d nll/dn      (adj_iters times, from 0)
 * and returns grad = d nll/d theta + (dKS/d theta)^T lambda.  The adjoint
 * pass is hand-written: reverse recurrences of the smoother and the filter
 * (as parallel scans), the Cholesky adjoint of the smoother factors and the
 * adjoint of the linearisation -- any sqsm_linearization: the sigma-point
 * regressions (cubature, unscented, Gauss-Hermite) through every point,
 * the Taylor linearisation through the second derivatives of the model
 * functions (Sec. 4.2, 4.3).
 *
 *   adj_iters   adjoint iterations (>= 0); always all of them (a fixed
 *               amount of work per evaluation, replayable as one graph).
 *               Iteration i takes the trajectory cotangent lambda of
 *               iteration i - 1 (0 in the first), so adj_iters = 1 gives
 *               the partial derivative of nll with respect to theta at the
 *               fixed trajectory n* (with M = 0: at init_ms/init_Ns);
 *               adj_iters = 0 computes nll only and writes grad = 0.
 *   tol         fixed-point tolerance (relative, max-norm): when > 0 the
 *               call sets SQSM_ERR_NOT_CONVERGED in the device status word
 *               if ipls_change >= tol or adj_change >= tol (or either is
 *               not finite), i.e. if n* is not a fixed point of Alg. 3 or
 *               lambda has not converged, so that grad is not the
 *               derivative Sec. 5.2 defines.  tol <= 0: no check.
 *   ms, Ns      outputs: the trajectory n* (state layout), as
 *               sqsm_ipls_smooth with the same M.
 *   nll         device double[1]; grad device double[3] (double[4] for
 *               SQSM_MODEL_CT_BEARINGS_R), theta order.
 *   adj_change  device double[1] or NULL: max-norm change of lambda in the
 *               last adjoint iteration relative to its max-norm (0 when
 *               adj_iters = 0).
 *   ipls_change device double[1] or NULL: max-norm change of the smoothing
 *               means from n* to the smoother of its linearisation (one
 *               more iteration of Alg. 3), relative to their max-norm.
 * With sqsm_options.max_group_steps a large batch is evaluated in groups of
 * sequences with a bounded workspace (see there); adj_change and
 * ipls_change are then the largest over the groups.
 * Other arguments as sqsm_ipls_smooth. */
int sqsm_ipls_nll_grad(sqsm_ctx* ctx, int dtype, const sqsm_model* model,
                       const double* theta, int linearization, int M,
                       int adj_iters, double tol, int64_t batch,
                       const int64_t* offsets, const void* y, const void* m0,
                       const void* N0, const void* init_ms,
                       const void* init_Ns, void* ms, void* Ns, double* nll,
                       double* grad, double* adj_change, double* ipls_change,
                       void* stream);

/* Statistical linear regression of a compiled-in model about a nominal
 * trajectory (one application of Sec. 4.2 / 4.3 to every step, the first
 * half of one iteration of Alg. 3).  Same batch layout as
 * sqsm_ipls_smooth; ms, Ns (state layout) are the nominal means / lower
 * factors.  Writes, for every observation row t of sequence b, the
 * linearised model of eq. Gamma-s: F[t] (nx x nx), c[t], SQ[t] (lower)
 * about state row t + b (k - 1), and H[t] (ny x nx), d[t], SR[t] (lower)
 * about state row t + b + 1 (k); d includes the 2 pi multiple that puts
 * y[t] on the branch of the bearings nearest h(m).  The outputs can be
 * passed to sqsm_lgssm_smooth with strides nx*nx, nx, nx*nx, ny*nx, ny,
 * ny*ny. */
int sqsm_ct_linearize(sqsm_ctx* ctx, int dtype, const sqsm_model* model,
                      const double* theta, int linearization, int64_t batch,
                      const int64_t* offsets, const void* y, const void* ms,
                      const void* Ns, void* F, void* c, void* SQ, void* H,
                      void* d, void* SR, void* stream);

/* Per-kernel timing (tracing aid; not part of the method).  While enabled,
 * sqsm_lgssm_smooth and sqsm_ipls_smooth bracket every kernel launch with a
 * pair of CUDA events on the launch stream; IPLS calls then replay a
 * separately captured, instrumented graph.  Enabling does not change any
 * result. */
int sqsm_profile_enable(sqsm_ctx* ctx, int on);

/* Synchronise ctx's device and sum the event-timed durations of the kernels
 * launched by the most recent profiled call, per kernel family:
 * ms[k] (milliseconds) and launches[k] for k = 0..nkinds-1 (host arrays;
 * families beyond the library's count are set to zero).  Returns the number
 * of families through *nfamilies if it is not NULL. */
int sqsm_profile_read(sqsm_ctx* ctx, int nkinds, double* ms, int* launches,
                      int* nfamilies);

/* Name of kernel family k ("" if out of range). */
const char* sqsm_kernel_name(int k);

/* Measurement aid, not part of the method (the paper has no counterpart):
 * enqueues on `stream` one kernel of `blocks` x `threads` threads (threads a
 * multiple of 32, at most 1024) whose only work is independent chains of
 * FP32 fused multiply-adds, `iters` loop trips of 128 FMAs per thread, and
 * writes one float per thread to the device buffer `out` (blocks * threads
 * floats, caller-owned).  *flops (host) receives the floating-point
 * operations it performs (an FMA counts 2).  Timing it with CUDA events on
 * `stream` gives the FP32 pipe's measured peak, the roof of the ALU-bound
 * scan and SLR kernels.  Returns SQSM_ERR_INVALID_ARG for bad sizes or null
 * pointers, SQSM_ERR_CUDA if the launch fails. */
int sqsm_fp32_fma_probe(int iters, int blocks, int threads, void* out, double* flops,
                        void* stream);

/* The linear smoother of sqsm_lgssm_smooth for callers that cannot
 * allocate device memory.  The paper has no counterpart of this call; it
 * exists for code running where cudaMalloc is unavailable or forbidden (an
 * allocator or memory-pool callback, a process whose device memory a
 * framework reserved up front, a real-time loop that cannot afford the
 * device synchronisation of an allocation).  Such callers cannot create an
 * sqsm_ctx, so this call takes none and allocates nothing: its scratch
 * buffers live in one fixed array of 32 MiB per device, part of the loaded
 * library, held until the process exits.
 *
 * Arguments and results are those of sqsm_lgssm_smooth, except:
 * - mf and Nf must not be NULL.
 * - Scan shape: leaf chunks of 4 steps and radix-4 folds on every upper
 *   level, the shape of a context created with leaf_chunk = 4 and radix = 4;
 *   on such a context sqsm_lgssm_smooth gives bit-identical results.  A
 *   context with the default shape brackets the scan differently, so its
 *   results agree with this call's to rounding only.
 * - There is no device status word: a non-finite result (a diverging
 *   filter) is not reported and the call still returns SQSM_OK; callers who
 *   need to know check the outputs (for example isfinite(*loglik)).
 * - The current CUDA device is used; `stream` must belong to it.
 * - Limit: n is bounded by the scratch size (about 280 bytes per step at
 *   FP32 and nx = 5, i.e. n up to roughly 1.2e5; half that at FP64).
 *   Larger problems return SQSM_ERR_TOO_LARGE before any GPU work.
 * - Set-up: the first call on a device (and the first after the device's
 *   context was reset, e.g. by cudaDeviceReset) initialises the device's
 *   primary context if needed and looks up the scratch array's device
 *   address, which loads the library's device code on that device; make
 *   that first call before any stream capture.
 * - All calls on a device share the scratch and its contents persist
 *   between calls; each call rewrites or clears what it reads.  Calls whose
 *   GPU work overlaps (different streams, different host threads) race on
 *   the scratch and must be serialised by the caller.
 * - If the calling thread has a CUDA error pending (cudaPeekAtLastError),
 *   the call enqueues nothing, leaves that error in place and returns
 *   SQSM_ERR_CUDA.
 * Returns SQSM_ERR_INVALID_ARG / SQSM_ERR_UNSUPPORTED as sqsm_lgssm_smooth,
 * SQSM_ERR_TOO_LARGE, or SQSM_ERR_CUDA. */
int sqsm_lgssm_smooth_noalloc(int dtype, int nx, int ny, int64_t n,
                              const void* F, int64_t sF, const void* c,
                              int64_t sc, const void* SQ, int64_t sSQ,
                              const void* H, int64_t sH, const void* d,
                              int64_t sd, const void* SR, int64_t sSR,
                              const void* m0, const void* N0, const void* y,
                              void* mf, void* Nf, void* ms, void* Ns,
                              double* loglik, void* stream);

/* 1 if the (nx, ny) pair is compiled into sqsm_lgssm_smooth, else 0. */
int sqsm_supported_shape(int nx, int ny);

#ifdef __cplusplus
}
#endif

#endif /* SQSM_H */
