/*
 * ihs.h -- C ABI of the GB300 Iterative Hessian Sketch library (libihs.so).
 *
 * The method is the Iterative Hessian Sketch with sparse embeddings of
 * Cormode & Dickens, "Iterative Hessian Sketch in Input Sparsity Time"
 * (arXiv 1910.14166).  For a problem (A, b, C) of Eq. 1,
 *     x_OPT = argmin_{x in C} f(x),  f(x) = 1/2 ||A x - b||_2^2,
 * each iteration draws a fresh CountSketch / SJLT S (Sec. 2), forms S A,
 * the approximate Hessian (SA)^T SA (Sec. 1), the exact gradient
 * A^T (b - A x^t), and solves the quadratic program of Eq. 2:
 *     x^{t+1} = argmin_{x in C} 1/2 ||S A (x - x^t)||^2 - <A^T (b - A x^t), x - x^t>.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers unless a comment says HOST.
 *     Matrices are row-major.  Nothing is copied: A and b are borrowed and
 *     must stay valid and unchanged for the life of the context.
 *   - Work is issued on the context's CUDA stream (or the stream argument of
 *     the stateless calls) and is asynchronous unless the comment says the
 *     call synchronises.  A context is not thread-safe.
 *   - Every call returns an ihs_status; nothing throws across the ABI.  A
 *     failure detected on the device (Hessian not positive definite, a QP
 *     that did not converge, a bounded wait that ran out) is written to a
 *     device status word and returned by the next call that synchronises
 *     (ihs_solve, ihs_sync, ihs_adjoint).
 *   - Sizes: n < 2^31 rows, 1 <= d <= 1024 columns, s divides m, m >= d.
 *     Dense A: m <= 51200 (the bucket sort counts in 200 KB of shared
 *     memory) and s * n < 2^31.  CSR A: nnz < 2^31, m / s <= 51200 with FP32
 *     accumulators, <= 25600 with FP64 (a block's buckets in 200 KB of
 *     shared memory).
 */
#ifndef IHS_H_
#define IHS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ihs_ctx ihs_ctx;

typedef enum {
  IHS_OK = 0,
  IHS_ERR_ARG = 1,            /* invalid argument or shape                      */
  IHS_ERR_CUDA = 2,           /* a CUDA runtime call failed                     */
  IHS_ERR_OOM = 3,            /* device allocation failed                       */
  IHS_ERR_NOT_SPD = 4,        /* sketched Hessian not positive definite         */
  IHS_ERR_NOT_CONVERGED = 5,  /* the inner QP / PCG did not reach its tolerance */
  IHS_ERR_NONFINITE = 6,      /* NaN or Inf met in the data or the iterate      */
  IHS_ERR_TIMEOUT = 7,        /* a bounded device wait gave up                  */
  IHS_ERR_UNSUPPORTED = 8     /* valid request outside this build's limits      */
} ihs_status;

/* Matrix storage (Eq. 1's A).  DENSE: val is n x d row-major with leading
 * dimension ld >= d (elements).  CSR: rowptr[n+1] (int32 or int64, see
 * rowptr_i64), col[nnz] int32 in [0, d), val[nnz]; columns within a row
 * must be distinct. */
enum { IHS_DENSE = 0, IHS_CSR = 1 };
enum { IHS_F64 = 0, IHS_F32 = 1 };

typedef struct {
  int kind;            /* IHS_DENSE or IHS_CSR                         */
  int dtype;           /* IHS_F64 or IHS_F32 (values)                  */
  int64_t n, d;        /* rows, columns                                */
  int64_t ld;          /* DENSE: leading dimension in elements          */
  const void* val;     /* values                                        */
  const int32_t* col;  /* CSR column indices (NULL for DENSE)           */
  const void* rowptr;  /* CSR row pointers (NULL for DENSE)             */
  int rowptr_i64;      /* CSR: 1 if rowptr is int64, 0 if int32         */
  int64_t nnz;         /* CSR: number of stored entries                 */
} ihs_matrix;

/* Constraint set C of Eq. 1 (Sec. 1 lists OLS and the p-norm balls).
 *   IHS_OLS        C = R^d                                param unused
 *   IHS_L1_BALL    C = {x : ||x||_1 <= param}  (LASSO)     param = radius > 0
 *   IHS_RIDGE      f(x) + (param/2) ||x||^2, C = R^d       param = lambda >= 0
 *   IHS_L1_PENALTY f(x) + param ||x||_1, C = R^d            param = lambda > 0
 *   IHS_L2_BALL    C = {x : ||x||_2 <= param}               param = radius > 0
 * Ridge is not in the paper; it is the squared-l2 penalty beside the p = 2
 * ball, with the penalty kept exact (not sketched).  IHS_L1_PENALTY is the
 * penalised LASSO of the experiments (Sec. 5, lambda = 5): each step solves
 * argmin_x 1/2 ||S A (x - x^t)||^2 - <A^T (b - A x^t), x - x^t> + lambda ||x||_1
 * exactly, the penalty unsketched.
 * IHS_L2_BALL (Sec. 1's p = 2 ball) solves each step exactly through the
 * secular equation ||(H + mu I)^{-1} (H x^t + g)|| = R (Newton's method on mu,
 * one factorisation of H + mu I per Newton step, FP64-refined solves); the
 * host reads two scalars per Newton step, so ihs_step / ihs_solve wait on
 * the GPU inside each such step. */
enum { IHS_OLS = 0, IHS_L1_BALL = 1, IHS_RIDGE = 2, IHS_L1_PENALTY = 3, IHS_L2_BALL = 4 };

typedef struct {
  int kind;
  double param;
} ihs_constraint;

/* Arithmetic of the sketch and Hessian (the residual and gradient are
 * FP64-class in every mode).
 *   IHS_PREC_FP64  plain: SA accumulated in FP64, FP64 Gram, FP64 Cholesky.
 *   IHS_PREC_TF32  mixed: SA accumulated in FP32, Gram on the tensor cores
 *                  from TF32 inputs with FP32 accumulation, FP32 factor.
 *   IHS_PREC_BF16  mixed: as TF32 with BF16 Gram inputs. */
enum { IHS_PREC_FP64 = 0, IHS_PREC_TF32 = 1, IHS_PREC_BF16 = 2 };

typedef struct {
  int64_t m;          /* sketch rows (projection dimension, Sec. 2)          */
  int s;              /* nonzeros per column of S: 1 = CountSketch, >1 = SJLT */
  uint64_t seed;      /* sketch seed; iteration t uses counter t             */
  int precision;      /* IHS_PREC_*                                          */
  int qp_max_iter;    /* l1 ball: FISTA iteration cap per QP (0 = default)   */
  double qp_tol;      /* l1 ball: KKT acceptance tolerance (0 = default)     */
  int flags;          /* IHS_FLAG_* (0 = default)                           */
  int sketch;         /* IHS_SKETCH_* (0 = the sparse embedding)             */
} ihs_options;

/* Sketch family (Sec. 2).
 *   IHS_SKETCH_SPARSE  CountSketch (s = 1) or SJLT (s > 1): the method's sketch.
 *   IHS_SKETCH_SRHT    S = m^{-1/2} P H D, the paper's dense comparison: D the
 *                      +-1 signs of the sparse draw's block 0, H the Sylvester
 *                      Hadamard transform of order n2 = the least power of two
 *                      >= n (A padded with zero rows), P m rows sampled
 *                      uniformly with replacement (block 1's words).  Dense A
 *                      only (IHS_ERR_UNSUPPORTED for CSR), s must be 1; the
 *                      context holds an n2 x d work buffer (FP64 in the plain
 *                      form, FP32 in the mixed form).
 *   IHS_SKETCH_GAUSSIAN S = G / sqrt(m) with G_ij iid N(0, 1) (Box-Muller of
 *                      the counter words of block 2), the dense comparison
 *                      whose cost is an O(m n d) product.  G is never stored:
 *                      the sketch kernel generates each tile of G in shared
 *                      memory and multiplies it into SA there (tcgen05 tensor
 *                      cores with TF32 inputs and FP32 accumulation in the
 *                      mixed form, FP64 SIMT in the plain form); the context
 *                      holds the split-K partials of SA.  Dense A only, s = 1. */
enum { IHS_SKETCH_SPARSE = 0, IHS_SKETCH_SRHT = 1, IHS_SKETCH_GAUSSIAN = 2 };

/* Option flags (a bit not listed here makes ihs_create return IHS_ERR_ARG).
 * IHS_FLAG_NO_FUSE: in ihs_solve, form SA and the gradient in
 * two separate passes over A even where the single fused pass applies (dense
 * FP32 data, mixed precision, CountSketch, d <= 512); results agree to
 * rounding, the fused pass reads A once instead of twice. */
enum {
  IHS_FLAG_NO_FUSE = 1,
  IHS_FLAG_SERIAL = 2,
  IHS_FLAG_CLUSTER = 4,
  IHS_FLAG_NO_LOOKAHEAD = 8,
  IHS_FLAG_FP64_FACTOR = 16,
  IHS_FLAG_NO_GRAPH = 32
};
/* IHS_FLAG_SERIAL: issue the sketch chain (draw, sort, SA, Gram, factor) on
 * the caller's stream too, instead of overlapping it with the gradient and
 * step on an internal stream.  Same results; useful for timing stages.
 * IHS_FLAG_CLUSTER: factor the sketched Hessian with the 16-CTA cluster
 * kernel (the whole factor resident in the cluster's shared memory, hardware
 * cluster barriers between steps) where it fits (FP32 up to d = 1024, FP64
 * up to d = 768), instead of the cooperative grid kernel.  The two give
 * identical factors; the grid kernel, spread over every SM, is the faster
 * one at the sizes measured so far.
 * IHS_FLAG_NO_LOOKAHEAD: with the fused pass, form SA of iteration t and the
 * gradient of iteration t in the same pass and factor before the step.  By
 * default the pass of iteration t forms the gradient of t and SA of t + 1,
 * so the Gram and factor of t + 1 (on a 16-CTA share of the GPU) run beside
 * the step of t and the pass of t + 1 instead of between them; SA of the
 * first iteration then takes one sketch-only pass.  Same sketches, same
 * iterates to rounding.
 * IHS_FLAG_FP64_FACTOR: in the mixed forms, factor the (TF32/BF16) sketched
 * Hessian and apply the factor in FP64, as the plain form does, instead of
 * in FP32.  The factor only preconditions the step (the residual, gradient
 * and update that set the attainable accuracy are FP64-class either way), so
 * both reach the same accuracy in the same iterations.  The FP64 factor costs
 * more on this GPU's FP64 units: with the look-ahead pipeline the pass of
 * iteration t then forms SA of iteration t + 2 (not t + 1), so each factor
 * has two passes' time beside them; the context keeps three factors.
 * IHS_FLAG_NO_GRAPH: a context whose A takes at most 128 MB (where a solve
 * is bound by launches, not by the data) replays each ihs_solve as a CUDA
 * graph: captured on the first call with a given (t0, iters), on an internal
 * copy of the iterate, and launched as one unit afterwards (the p = 2 ball,
 * whose step reads scalars on the host, the l1 penalty, whose one-CTA step
 * kernels must be issued ahead of the sketch chain's full-width kernels to
 * get an SM, and IHS_FLAG_SERIAL never are).
 * Same kernels in the same order, so the same results.  This flag turns it
 * off.  ihs_report.graph tells whether a solve ran as a graph; if a capture
 * fails, the context falls back to issuing on its streams for good. */

typedef struct {
  int iters;            /* iterations taken                                */
  int qp_fista_iters;   /* l1 steps: FISTA iterations spent, summed         */
  int status;           /* ihs_status of the device status word             */
  double step_norm;     /* ||x^{t+1} - x^t||_inf of the last step            */
  int qp_active_rounds; /* penalised l1: active-set rounds spent, summed     */
  int graph;            /* ihs_solve: 1 if it ran as a replayed CUDA graph   */
} ihs_report;

/* ihs_create -- validate (A, b, C, options) and allocate every workspace:
 * the problem (A, b, C) of Eq. 1 with the sketch of Sec. 2 (m rows, s
 * blocks, seed).
 * A: matrix descriptor (HOST struct; its arrays are DEVICE, borrowed).
 * b: DEVICE, n doubles, borrowed.  C, opt: HOST structs, copied.
 * stream: a cudaStream_t (NULL = legacy default stream).  For CSR input a
 * column-major (CSC) copy of A is built once here and owned by the context.
 * Workspaces come from a library-owned device memory pool (see
 * ihs_trim_memory).
 * Synchronises.  Errors: IHS_ERR_ARG for shapes (m % s != 0, m < d,
 * n >= 2^31, bad kind/dtype/flags), IHS_ERR_UNSUPPORTED for d > 1024 and
 * the m, s * n and nnz limits above, IHS_ERR_OOM, IHS_ERR_CUDA. */
ihs_status ihs_create(ihs_ctx** out, const ihs_matrix* A, const double* b,
                      const ihs_constraint* C, const ihs_options* opt,
                      void* stream);

/* ihs_sketch -- draw S for counter t (Sec. 2) and form SA and the
 * approximate Hessian H = (1/s) (SA)^T SA (+ lambda I for ridge) inside the
 * context (Sec. 1; Eq. 2's quadratic term).  Asynchronous. */
ihs_status ihs_sketch(ihs_ctx* ctx, int64_t t);

/* ihs_gradient -- g = A^T (b - A x) (minus lambda x for ridge), the linear
 * term of Eq. 2, and optionally r = b - A x.  x: DEVICE d doubles (in);
 * g: DEVICE d doubles (out); r: DEVICE n doubles or NULL.  Asynchronous. */
ihs_status ihs_gradient(ihs_ctx* ctx, const double* x, double* g, double* r);

/* ihs_sketch_gradient -- both halves of Eq. 2's subproblem, with one read
 * of A where the fused pass applies: draw S for counter t and form SA, the
 * Hessian (1/s) (SA)^T SA (+ lambda I) and its factor, as ihs_sketch does,
 * and the gradient g = A^T (b - A x) (minus lambda x for ridge) at x, as
 * ihs_gradient does.  SA is the sum over the rows of each bucket (Sec. 2's
 * streaming update) and the gradient is O(nnz(A)); both stream A, so the
 * fused pass (dense FP32 A, a mixed precision, CountSketch, d <= 512, ld and
 * d multiples of 4, IHS_FLAG_NO_FUSE unset) uses each row of A three times
 * while it is in registers: for SA, for the residual and for the gradient.
 * It is the kernel ihs_solve runs every iteration, in the same row-chunk
 * plan.  Other contexts run the sketch chain and then the gradient pass.
 * x: DEVICE d doubles (in); g: DEVICE d doubles (out), may not alias x.
 * Afterwards ihs_get_sketch returns this SA and Hessian and ihs_step uses
 * this factor.  Asynchronous, on the context's stream.  Errors: IHS_ERR_ARG
 * (NULL, t < 0), IHS_ERR_CUDA. */
ihs_status ihs_sketch_gradient(ihs_ctx* ctx, int64_t t, const double* x, double* g);

/* ihs_step -- one step of Eq. 2 with the Hessian of the last ihs_sketch:
 * x (DEVICE, d doubles) holds x^t on entry and x^{t+1} on return.  OLS and
 * ridge: Cholesky solve of H delta = g.  l1 ball: the exact QP over the ball.
 * Asynchronous; device failures surface at the next synchronising call. */
ihs_status ihs_step(ihs_ctx* ctx, double* x);

/* ihs_solve -- iterations t = t0 .. t0+iters-1 of Eq. 2 (ihs_sketch + ihs_step) from
 * the x given (DEVICE, d doubles; in: x^{t0}, out: x^{t0+iters}).  The run
 * is a pure function of (A, b, C, options, x, t0), so stopping after k
 * iterations and resuming with t0 + k reproduces it exactly.  rep: HOST,
 * nullable.  Synchronises and returns the device status. */
ihs_status ihs_solve(ihs_ctx* ctx, double* x, int64_t t0, int iters,
                     ihs_report* rep);

/* ihs_sync -- wait for the context's stream and return the device status
 * word (then clear it).  A service of the library (no counterpart in the
 * paper). */
ihs_status ihs_sync(ihs_ctx* ctx);

/* ihs_get_sketch -- copy the last sketch out, for inspection and tests: SA of
 * Sec. 2 and the approximate Hessian of Sec. 1.
 * SA_out: DEVICE buffer for the m x d row-major raw sketch SA (entries +-1,
 * SJLT normalisation not applied), FP64 for precision FP64 and FP32 for the
 * mixed modes (*SA_dtype, HOST, gets IHS_F64 or IHS_F32).  H_out: DEVICE
 * d x d doubles, the Hessian actually used ((1/s) SA^T SA + lambda I).
 * scale: HOST, gets 1/s.  Every output may be NULL.  Stream-ordered copies;
 * IHS_ERR_ARG if no sketch has been formed yet. */
ihs_status ihs_get_sketch(ihs_ctx* ctx, void* SA_out, int* SA_dtype, double* H_out,
                          double* scale);

/* ihs_trim_memory -- a service of the library (no counterpart in the
 * paper).  Contexts take their device workspaces from a
 * library-owned memory pool per device that keeps what ihs_destroy frees, so
 * that creating the next context does not map new device memory.  This call
 * returns every pool's unused memory to the device.  Call it with no context
 * operation in flight (it does not synchronise streams).  Errors:
 * IHS_ERR_CUDA. */
ihs_status ihs_trim_memory(void);

/* ihs_selftest_wait -- a self-test of the library (no counterpart in the
 * paper): exercises the bounded device wait used by the
 * library's grid barriers without faulting or hanging the GPU: two CTAs wait
 * at a barrier that expects three (nothing ever completes it), each gives up
 * after 4096 polls (well under a millisecond) and records the timeout in a
 * device status word, which is read back.  Returns IHS_ERR_TIMEOUT when the
 * wait gave up as designed, IHS_OK if the barrier wrongly passed,
 * IHS_ERR_CUDA / IHS_ERR_OOM on a runtime failure.  stream: a cudaStream_t
 * (NULL = legacy default stream); synchronises it. */
ihs_status ihs_selftest_wait(void* stream);

/* ihs_selftest_rsqrt -- evaluates, for each of the n doubles p[i] (DEVICE),
 * the reciprocal square root the FP64 Cholesky factor uses for its pivots
 * (Newton-Raphson from an FP32 seed; the pivots of the factor of Eq. 2's
 * sketched Hessian) into out[i], and CUDA's rsqrt(p[i]) into ref[i] (both
 * DEVICE, n doubles), so that tests can bound the first against the second.
 * Positive finite p only (the factor records a non-positive pivot as
 * IHS_ERR_NOT_SPD before it takes the root).  n <= 0 does nothing.  stream:
 * a cudaStream_t (NULL = legacy default stream); not synchronised.  Errors:
 * IHS_ERR_ARG (null pointer with n > 0), IHS_ERR_CUDA. */
ihs_status ihs_selftest_rsqrt(const double* p, double* out, double* ref, int64_t n, void* stream);

/* ihs_exact_gram -- G = A^T A in FP64 (DEVICE, d x d doubles, row-major,
 * both triangles), the reference of the sketch-quality experiment (App. B:
 * the empirical error ||A^T S^T S A - A^T A||_F / ||A^T A||_F).  Dense A: an
 * FP64 Gram over the n rows (FP32 entries promoted exactly), deterministic.
 * CSR A: each row's outer product added with FP64 atomics, so the rounding
 * order varies from run to run.  Stream-ordered on the context's stream
 * (does not synchronise); the dense form allocates its split partials on
 * first use.  Errors: IHS_ERR_ARG (null), IHS_ERR_OOM, IHS_ERR_CUDA. */
ihs_status ihs_exact_gram(ihs_ctx* ctx, double* G);

/* ihs_sketch_error -- App. B's empirical sketch error: form the sketch of
 * counter t as ihs_sketch does, then
 * err (HOST) = ||H_t - G||_F / ||G||_F with H_t = (1/s) (S_t A)^T (S_t A)
 * (+ lambda I for ridge) and G (DEVICE, d x d) normally from
 * ihs_exact_gram.  Synchronises; returns the device status. */
ihs_status ihs_sketch_error(ihs_ctx* ctx, int64_t t, const double* G, double* err);

/* ihs_adjoint -- reverse-mode derivative of a loss L(x) of the ridge / OLS
 * solution x = (A^T A + lambda I)^{-1} A^T b (not in the paper).
 * v = (A^T A + lambda I)^{-1} dLdx is solved by conjugate gradients
 * preconditioned with the Cholesky factor of the last sketched Hessian; then
 *   dL/db = A v                  (DEVICE, n doubles, nullable)
 *   dL/dA = r v^T - (A v) x^T    (DEVICE, n x d row-major in A's dtype, nullable)
 * with r = b - A x.  x, dLdx: DEVICE d doubles.  Requires an earlier
 * ihs_sketch.  rep (HOST, nullable) gets the CG iteration count in iters.
 * Synchronises.  IHS_ERR_NOT_CONVERGED if CG misses 1e-13 relative. */
ihs_status ihs_adjoint(ihs_ctx* ctx, const double* x, const double* dLdx,
                       double* dLdb, void* dLdA, ihs_report* rep);

/* Stage timing (CUDA events recorded on the stream that runs each stage,
 * around each stage of every iteration while enabled) and a count of the
 * library's kernel launches.  Stages, in order: IHS_ST_SORT (sketch draw and
 * bucket sort), IHS_ST_SKETCH (the SA kernel; in the in-order fused form the
 * one pass that forms SA and the gradient; in the look-ahead fused form the
 * sketch-only pass that starts each ihs_solve), IHS_ST_SKETCH_FIX
 * (straddling and empty buckets), IHS_ST_GRAM, IHS_ST_FACTOR, IHS_ST_GRAD
 * (the gradient pass; in the look-ahead fused form the pass that forms the
 * gradient and the next iteration's SA), IHS_ST_STEP. */
enum { IHS_ST_SORT = 0, IHS_ST_SKETCH, IHS_ST_SKETCH_FIX, IHS_ST_GRAM, IHS_ST_FACTOR,
       IHS_ST_GRAD, IHS_ST_STEP, IHS_NSTAGES };

/* ihs_profile -- enable (1) or disable (0) stage timing; enabling clears
 * the totals and the launch count.  A service of the library (no
 * counterpart in the paper), like ihs_profile_read. */
ihs_status ihs_profile(ihs_ctx* ctx, int enable);

/* ihs_profile_read -- synchronise and report, per stage, the summed event
 * time in ms (ms[IHS_NSTAGES], HOST) and the number of timed instances
 * (count[IHS_NSTAGES], HOST, nullable), and the kernel launches issued by the
 * library since ihs_profile(ctx, 1) (launches, HOST, nullable).  A service of
 * the library (no counterpart in the paper). */
ihs_status ihs_profile_read(ihs_ctx* ctx, double* ms, int* count, int64_t* launches);

/* ihs_destroy -- free every workspace (NULL is a no-op).  Synchronises.
 * A service of the library (no counterpart in the paper). */
void ihs_destroy(ihs_ctx* ctx);

/* ihs_status_str -- static text for a status code (a service of the
 * library). */
const char* ihs_status_str(ihs_status st);

/* ---------------------------------------------------------------------
 * Stateless kernels (no context).  Same conventions; stream may be NULL.
 * --------------------------------------------------------------------- */

/* ihs_hash -- the sketch draw of Sec. 2 for counter t: for block k < s and
 * row i < n, bucket[k*n + i] = k*(m/s) + h_k(i) (global row of S, int32)
 * and sign[k*n + i] in {+1, -1} (int8).  The generator is SplitMix64
 * (Steele, Lea & Flood 2014) used counter-style:
 *   key_seed = F(seed, 0), key_t = F(key_seed, t), key_tk = F(key_t, k),
 *   w = F(key_tk, i),  F(x, j) = mix(x + (j + 1) * 0x9E3779B97F4A7C15),
 * with the SplitMix64 finaliser mix; h_k(i) = (hi32(w) * (m/s)) >> 32 and the
 * sign is -1 iff bit 0 of w is set.  Errors: IHS_ERR_ARG if m % s != 0. */
ihs_status ihs_hash(uint64_t seed, int64_t t, int s, int64_t m, int64_t n,
                    int32_t* bucket, int8_t* sign, void* stream);

/* ihs_sketch_adjoint -- S^T G for the sketch of counter t with entries
 * sign/sqrt(s): out[i, :] = sum_k sign_k(i) G[bucket_k(i), :] / sqrt(s).
 * G: DEVICE m x d doubles (row-major), out: DEVICE n x d doubles.  A
 * gather, one row of out per row of A (the adjoint of Sec. 2's map). */
ihs_status ihs_sketch_adjoint(uint64_t seed, int64_t t, int s, int64_t m,
                              int64_t n, int64_t d, const double* G,
                              double* out, void* stream);

/* ihs_gradient_noalloc -- g = A^T (b - A x) - lambda x for a DENSE A (the
 * linear term of Eq. 2), the same quantity as ihs_gradient, for callers that cannot allocate device
 * memory when they call: code whose device memory is all handed to its own
 * pool allocator, or latency-critical loops that cannot afford the implicit
 * device-wide synchronisation of cudaMalloc.  It needs no context and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 * The paper has no counterpart; this is a service of the library.
 *   A: HOST descriptor of a DENSE matrix (IHS_F32 or IHS_F64, DEVICE values,
 *      d <= 1024; n = 0 is allowed, with A->val and b then unused and
 *      possibly NULL, and gives g = -lambda x); b: DEVICE n doubles;
 *   x: DEVICE d doubles; g: DEVICE d doubles (out); stream: cudaStream_t or
 *   NULL.  The types and lengths behind these pointers cannot be checked
 *   here: a b shorter than n or of another type is read out of bounds.
 * Scratch: a fixed 4 MiB array of per-warp partial gradients inside the
 * library (512 Ki doubles), held by every GPU that loads the library until
 * the process exits; the number of warps is chosen so that warps * d fits.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current, together with its SM count, which sets
 * the number of warps); make the first call on each device before any stream
 * capture.  The address belongs to the device's current context: if that
 * context is destroyed and re-created (cudaDeviceReset), the next call sees
 * a new context id and looks the address up again.  Every call overwrites
 * the slots it uses, so no clearing is needed, but calls that overlap on the
 * GPU (in flight at the same time, e.g. on two streams) race on the shared
 * array.
 * Errors: IHS_ERR_ARG (not dense, bad shape or NULL pointer),
 * IHS_ERR_UNSUPPORTED (d > 1024), IHS_ERR_CUDA.  Asynchronous. */
ihs_status ihs_gradient_noalloc(const ihs_matrix* A, const double* b, const double* x,
                                double lambda, double* g, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IHS_H_ */
