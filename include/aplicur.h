/*
 * aplicur.h -- C ABI of the GB300 (sm_103a) APLICUR solver.
 *
 * APLICUR solves the regularized linear least-squares problem
 *     min_x ||A x - b||_2^2 + mu ||x||_2^2,   A in R^{m x n}, m >= n,
 * (Huh, Cartis, Nakatsukasa, "Adaptive LSQR Preconditioning from One Small
 * Sketch", Eq. regularizedLLS) by LSQR on the augmented matrix
 * [A; delta I], delta = sqrt(mu) (Eq. augLLS), right-preconditioned by the
 * CUR-based spectral preconditioner of Eq. preconditioner2, which is refined
 * between warm-started LSQR phases from one sparse-sign sketch S A
 * (Algorithm "APLICUR: detailed implementation").
 *
 * Conventions for every entry point:
 *  - Device pointers are CUDA device addresses on the current device; host
 *    pointers are ordinary process memory.  Each argument says which.
 *  - Dense matrices passed in are row-major with leading dimension `ld`
 *    (elements); small dense outputs are column-major unless stated.
 *  - Borrowed inputs (A, b) must stay alive and unmodified until
 *    aplicur_destroy.  The library never frees caller memory.
 *  - All work is issued on the stream given at creation (a cudaStream_t
 *    passed as void*; NULL: a non-blocking stream the handle creates and owns, so
 *    that graph captures on it never meet work on the legacy default stream of
 *    other threads).  Calls that return host results synchronise that stream.
 *  - No C++ exception crosses this boundary.  Every call returns an
 *    aplicur_status; on failure aplicur_last_error(h) holds a message.
 *  - Calls on one handle are not thread-safe; distinct handles are.
 */
#ifndef APLICUR_H_
#define APLICUR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  APLICUR_OK = 0,
  APLICUR_EINVAL = 1,      /* invalid argument (shape, pointer, option) */
  APLICUR_ENOMEM = 2,      /* device or host allocation failed */
  APLICUR_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  APLICUR_ENOTCONV = 4,    /* maxit reached before tol; x_out holds the best iterate */
  APLICUR_EBREAKDOWN = 5,  /* a Cholesky factorisation met a non-positive pivot */
  APLICUR_ETIMEOUT = 6     /* a bounded device wait gave up */
} aplicur_status;

enum { APLICUR_DENSE_ROWMAJOR = 0, APLICUR_CSR = 1 };
enum { APLICUR_F64 = 0, APLICUR_F32 = 1 };
/* Arithmetic of the products with an FP32-stored A (FP64-stored A always uses FP64):
 *  FP64  products and sums in FP64 (values promoted exactly);
 *  MIXED FP32 products with FP32 sums per thread, FP64 across threads; each LSQR phase
 *        is an inner solve of an FP64 iterative refinement in correction form: it
 *        starts from g = A^T (b - A x) - mu x formed with FP64 products, solves
 *        [A; delta I] dx ~ [0; g / delta] (the normal equations of the paper's warm
 *        start) and adds dx to x in FP64; it ends once its estimate of ||Abar^T rbar||
 *        fell by 1e-4, or when an explicit residual check (formed as the statistic
 *        ne_res is) shows the residual no longer falling.
 *        The stopping tests use the paper's residual estimate.  (mu = 0: the phase
 *        starts from the FP64 residual [b - A x; 0] instead.)
 *  DF32  compensated FP32: operand vectors split into FP32 hi + lo parts, exact
 *        products by FMA residuals and two-term sums, i.e. FP64-level accuracy from
 *        FP32 instructions only.
 * In every mode the preconditioner basis, all LSQR scalars and the CUR core
 * factorisations are FP64. */
enum { APLICUR_PREC_FP64 = 0, APLICUR_PREC_MIXED = 1, APLICUR_PREC_DF32 = 2 };

/* The matrix A (borrowed, device memory).
 *  format = APLICUR_DENSE_ROWMAJOR: values -> m x n row-major, leading dim ld >= n.
 *  format = APLICUR_CSR: rowptr (m+1 int32), colidx (nnz int32, column indices
 *  of each row in increasing order), values (nnz).  dtype selects F64 or F32
 *  values.  The library builds its own transposed (CSC) copy at creation. */
typedef struct {
  int32_t format;
  int32_t dtype;
  int64_t m, n, ld, nnz;
  const void* values;
  const int32_t* rowptr;
  const int32_t* colidx;
} aplicur_matrix;

/* Solver options; fill with aplicur_options_default() then override.
 * Defaults follow the paper's Section 7 settings: eps_cur = 30 delta,
 * nu_prec = 10, nu_lsqr = 100, eps_lsqr = 1e-10, xi = 8, r = 10. */
typedef struct {
  uint64_t seed;             /* drives S and W when they are not supplied */
  double eps_cur_factor;     /* eps_cur = eps_cur_factor * sqrt(mu) */
  double nu_prec;            /* re-preconditioning tolerance (Section 5.3.2) */
  double nu_lsqr;            /* dynamic LSQR stopping tolerance (Section 5.3.2) */
  double eps_lsqr;           /* Paige-Saunders stopping tolerance of each phase */
  int32_t xi;                /* nonzeros per sketch column (capped at s) */
  int32_t normest_r;         /* Gaussian vectors of Eq. 2normestimate */
  int32_t check_gap;         /* LSQR iterations between explicit residual checks */
  int32_t max_extra_phases;  /* warm restarts of the final phase */
  int32_t precision;         /* APLICUR_PREC_FP64, _MIXED or _DF32 */
  int32_t graph_iters;       /* LSQR iterations per captured CUDA graph (>=1) */
  /* Optional host arrays that replace the seeded draws (parity testing):
   * sketch_rows/sketch_signs: m*xi row indices in [0,s) and +-1 signs of the
   * sparse sign embedding, row-major by column of S; normest_w: n*r Gaussian
   * matrix, column-major.  Copied at creation. */
  const int32_t* sketch_rows;
  const int8_t* sketch_signs;
  const double* normest_w;
  /* Optional replay schedule (host arrays, copied at creation; see also
   * aplicur_set_replay): phase k runs exactly replay_phases[k] LSQR iterations
   * and rank step k rebuilds the preconditioner iff replay_rebuild[k] != 0.
   * Used to run the exact schedule of another run (e.g. of a reference solve)
   * so that iterates can be compared; explicit residual checks are off then. */
  int32_t replay_nphases;
  const int32_t* replay_phases;
  int32_t replay_nsteps;
  const int8_t* replay_rebuild;
  /* Non-zero: record CUDA events around the hot-loop kernels inside every LSQR
   * iteration and accumulate their device times (aplicur_get_profile). */
  int32_t profile;
  /* > 0: cap the CUR rank; reaching it ends rank growth like reaching min(m, n)
   * (the last block is truncated to fit).  0: no cap. */
  int32_t max_rank;
  /* Non-zero: the dense products of the rank steps and preconditioner builds (GEMMs of
   * augmentQR, E_col, E_row, Cholesky and triangular-solve updates, the Jacobi rotation
   * transfer) run on the FP64 units.  0 (default): compensated FP32 (hi + lo operands,
   * exact hi products, TwoSum accumulation; about 2^-46 relative), several times faster
   * on GB300, whose FP64 rate is 1/64 of its FP32 rate. */
  int32_t fp64_dense;
  /* APLICUR_VARIANT_SVD (0, default): the SVD-based preconditioner (Algorithm
   * CURPreconditioner).  APLICUR_VARIANT_SVDFREE (1): the SVD-free preconditioner of the
   * paper's "SVD-free variant" (Eq. preconditioner_svdfree).  With mu = 0 the CUR is of A;
   * with mu > 0 it is of the regularised matrix A_mu = [A; sqrt(mu) I] ((m + n) x n, the
   * appended rows stored with sqrt(mu) rounded to A's value type), as the paper prescribes
   * for regularised problems: the sketch then has m + n columns (user-supplied sketch
   * draws hold (m + n) xi entries), row indices >= m (aplicur_get_indices) name the row
   * m + j of A_mu, sqrt(mu) e_j^T, and C, R and the cross are those of A_mu.  Its inverse
   * sighat Q_R M^{-1} Q_R^T + (I - Q_R Q_R^T) uses
   * M^{-1} = T_R^{-T} A(I,J) T_C^{-1}, formed once per build by two triangular solves.  The
   * target level sighat is sigma_min(M) = 1 / ||M^{-1}||_2 from 50 power-iteration steps
   * on M^{-T} M^{-1} (the smallest CUR singular value, which the SVD-based form uses; the
   * paper's choice, the estimate rho, overstates it by up to the estimate's safety factor
   * and can leave A P^{-1} worse conditioned than A); the dynamic stopping rule uses it as
   * the smallest CUR singular value.  Not available for batched solves. */
  int32_t variant;
  /* APLICUR_SCHEDULE_ADAPTIVE (0, default): fully adaptive (rank growth interleaved with
   * preconditioner builds and warm-started LSQR phases).  APLICUR_SCHEDULE_SINGLE_SHOT (1):
   * the paper's rank-adaptive single-shot variant (Section "Levels of adaptivity"): the rank
   * grows as usual, but the preconditioner is built once, when growth ends, and a single
   * LSQR phase (with its warm restarts) follows.  With max_rank = sketch_dim the one rank
   * step selects all indices at once, which is the fixed-rank single-shot variant
   * (Algorithm "Sketched CUR with cross approximation using LUPP"). */
  int32_t schedule;
  /* Dense FP32 A with FP32 or compensated products (precision MIXED or DF32): how the
   * LSQR iterations read A.  The fused pass reads A once per iteration: thread-block
   * clusters stream row tiles through shared memory and form u' = A z - alpha u and the
   * column partial sums of A^T u' from the same tile (it needs n and ld multiples of 4
   * and a 16-byte aligned A; otherwise the two-pass form runs).  The two-pass form reads
   * A twice (A z, then A^T u).  Both give the same result up to rounding.
   *  APLICUR_DENSE_PASS_AUTO (0, default): fused with FP32 products (MIXED), where the
   *    pass is bound by HBM; two-pass with compensated products (DF32), where about
   *    eleven FP32 instructions per product make either form bound by instruction issue
   *    and the two-pass form issues them faster;
   *  APLICUR_DENSE_PASS_TWO (1): always two-pass;
   *  APLICUR_DENSE_PASS_FUSED (2): fused wherever it applies. */
  int32_t dense_pass;
  /* Optional caller-supplied device allocator.  When alloc is set, every device buffer of
   * the handle (workspace, factors, LSQR vectors) is allocated by
   * alloc(bytes, stream, alloc_ctx) and released by free_(ptr, bytes, stream, alloc_ctx),
   * with `stream` the stream the buffer is used on (stream-ordered semantics, as
   * cudaMallocAsync / cudaFreeAsync); the library then allocates no device memory itself.
   * alloc returning NULL fails the call with ENOMEM.  Set both or neither (EINVAL).  The
   * callbacks may be called from worker threads of batched solves and from
   * aplicur_destroy.  NULL (default): stream-ordered cudaMallocAsync / cudaFreeAsync. */
  void* (*alloc)(size_t bytes, void* stream, void* alloc_ctx);
  void (*free_)(void* ptr, size_t bytes, void* stream, void* alloc_ctx);
  void* alloc_ctx;
  /* The sketching operator S of Y = S A (appendix "Sketch comparison"):
   *  APLICUR_SKETCH_SPARSE_SIGN (0, default): the sparse sign embedding of Section 5.1
   *    (xi nonzeros per column, Y summed in a fixed FP64 order);
   *  APLICUR_SKETCH_GAUSSIAN (1): G / sqrt(s) with G i.i.d. N(0, 1);
   *  APLICUR_SKETCH_SRHT (2): the subsampled randomized Hadamard transform
   *    (1 / sqrt(s)) R H D (random column signs D, s distinct sampled rows R of the
   *    Walsh-Hadamard matrix of the padded length).
   * The dense operators are drawn on the host from the project generator (seed) and
   * applied as a product with A: FP64 products for CSR A, the dense routines' products
   * (compensated FP32 by default) for dense A. */
  int32_t sketch_kind;
  /* 1, 2 or 3 (dense A and a dense operator only; 0 = off): Y on the tensor cores
   * (tcgen05, FP32 accumulation), s <= 512.  S is rounded to bfloat16 (the rounded matrix
   * is the sketching operator) and A, after rounding to FP32, is represented by the first
   * sketch_tc terms of its bfloat16 expansion A_0 + A_1 + A_2 (A_0 = bf16(A), A_1 =
   * bf16(A - A_0), ...; three terms hold an FP32 value exactly).  One term leaves a noise
   * floor of about 2^-9 |A| entrywise in the sketch, which the adaptive rank cannot see
   * through when delta is below it; two terms lower it to 2^-17; three leave the FP32
   * accumulation only.  The CUR indices can differ from those of the FP64 sketch. */
  int32_t sketch_tc;
} aplicur_options;

enum { APLICUR_SKETCH_SPARSE_SIGN = 0, APLICUR_SKETCH_GAUSSIAN = 1, APLICUR_SKETCH_SRHT = 2 };

enum { APLICUR_DENSE_PASS_AUTO = 0, APLICUR_DENSE_PASS_TWO = 1, APLICUR_DENSE_PASS_FUSED = 2 };

enum { APLICUR_VARIANT_SVD = 0, APLICUR_VARIANT_SVDFREE = 1 };
enum { APLICUR_SCHEDULE_ADAPTIVE = 0, APLICUR_SCHEDULE_SINGLE_SHOT = 1 };

/* Device time by kernel family, accumulated over the solves since creation or the
 * last aplicur_reset_profile (requires options.profile).  Families:
 *  0 the A z pass, 1 the A^T u pass, 2 the preconditioner passes (LSQR hot loop;
 *    timed by events inside the captured iteration graphs);
 *  3 dense products (GEMMs, including those inside triangular solves and Cholesky;
 *    compensated FP32 by default, FP64 with fp64_dense),
 *  4 the second Jacobi stage of the preconditioner SVD (compensated FP32 by default,
 *    FP64 with fp64_dense), 5 LUPP index selection,
 *  6 the first, FP32 Jacobi stage of the SVD.
 * work[k] is algorithmic bytes for families 0, 1, 2, 5, FP64-equivalent flops for 3, 4
 * and FP32 flops for 6. */
typedef struct {
  double ms[7];              /* summed event-to-event device time */
  int64_t launches[7];       /* timed regions (kernel launches, sweeps, selections) */
  double work[7];            /* summed algorithmic bytes or flops */
  int64_t kernel_launches;   /* all kernels this process launched through the library */
} aplicur_profile;

typedef struct aplicur_ctx* aplicur_handle;

typedef struct {
  int64_t iters;        /* LSQR iterations over all phases */
  int32_t ell;          /* final CUR rank */
  int32_t nphases;      /* LSQR phases run */
  int32_t nsteps;       /* rank steps taken */
  int32_t converged;    /* explicit relative residual <= tol */
  double ne_res;        /* ||A^T(b - A x) - mu x|| / ||A^T b|| at exit, formed with FP64
                         * products; with FP32 values in the MIXED and DF32 forms a value
                         * above 100 tol may come from compensated FP32 products (about 44
                         * significant bits per sum), which decide no comparison with tol */
  double rho;           /* last norm estimate */
  double time_setup_ms; /* sketch and creation work (device time) */
  double time_solve_ms; /* aplicur_solve wall time */
  double time_rank_ms;  /* of which: CUR rank steps (Parts 1 and 2) */
  double time_build_ms; /*           preconditioner builds */
  double time_lsqr_ms;  /*           LSQR phases and residual checks */
  int32_t fused_pass;   /* 1: LSQR iterations read dense A once (fused A pass) */
  int32_t cluster_size; /* CTAs per thread-block cluster of the fused pass (0: not used) */
  int32_t rank_breakdown; /* 1: a rank step met a non-positive Cholesky pivot (the new
                           * columns or rows were numerically dependent on the selected
                           * ones); rank growth ended there and the solve finished with
                           * the last preconditioner built (the batched driver does the
                           * same per problem) */
} aplicur_stats;

/* Fill `opt` with the defaults above. */
void aplicur_options_default(aplicur_options* opt);

/* Create a solver for (A, b, mu) with block size b = sketch_dim and sketch
 * rows s = ceil(1.1 b) (Algorithm "APLICUR: detailed implementation",
 * Initialise), and compute the sketch Y = S A once (Section 5.1).
 *  out        host: receives the handle.
 *  A          host struct describing borrowed device memory (see above).
 *  b          device: m doubles (borrowed).
 *  mu         >= 0, coefficient of ||x||^2.
 *  sketch_dim block size b, 1 <= b <= min(m, n).
 *  opt        host, nullable (defaults).
 *  stream     cudaStream_t as void*.
 * Errors: EINVAL (m < n, bad pointers, sizes), ENOMEM, ECUDA. */
aplicur_status aplicur_create(aplicur_handle* out, const aplicur_matrix* A, const double* b,
                              double mu, int32_t sketch_dim, const aplicur_options* opt,
                              void* stream);

/* Run the adaptive solve (CUR rank steps, preconditioner updates, warm-started
 * LSQR phases) until the relative normal-equation residual
 * ||A^T(b - A x) - mu x|| / ||A^T b|| <= tol (checked in FP64) or maxit LSQR
 * iterations.  Restarts from x = 0 and I = J = {} on every call.
 *  x_out device: n doubles (caller-owned).
 * Returns OK, ENOTCONV (x_out still written), EBREAKDOWN, ETIMEOUT, ECUDA. */
aplicur_status aplicur_solve(aplicur_handle h, double tol, int64_t maxit, double* x_out);

/* Replace the replay schedule (host arrays, copied).  nphases = nsteps = 0
 * turns replay off. */
aplicur_status aplicur_set_replay(aplicur_handle h, int32_t nphases, const int32_t* phases,
                                  int32_t nsteps, const int8_t* rebuild);

/* Plain (unpreconditioned) LSQR on [A; delta I] with the same kernels and the
 * same stopping test: the comparison baseline.  x_out device n doubles.  Clears the CUR
 * state of the handle, so that a following aplicur_backward is the unpreconditioned
 * adjoint solve of this baseline. */
aplicur_status aplicur_plain_lsqr(aplicur_handle h, double tol, int64_t maxit, double* x_out);

/* Adjoint of the last solve (not in the paper).  With g = dL/dx (device, n),
 * solves (A^T A + mu I) lambda = g by preconditioned LSQR on
 * min ||[A; delta I] lambda - [0; g/delta]|| with the final preconditioner, then
 *   grad_b  = A lambda                    (device, m doubles, may be NULL)
 *   grad_mu = -lambda^T x                 (host, 1 double, may be NULL)
 *   grad_A  = r lambda^T - (A lambda) x^T (device, m x n row-major in A's dtype,
 *             leading dim n; dense A only; may be NULL), r = b - A x.
 * Requires mu > 0 and a previous aplicur_solve (or aplicur_plain_lsqr: then P = I). */
aplicur_status aplicur_backward(aplicur_handle h, const double* grad_x, double tol,
                                int64_t maxit, double* grad_b, double* grad_mu, void* grad_A);

/* Copy the CUR row and column indices (selection order) to host arrays of
 * capacity min(m, n); *ell receives their count.  I or J may be NULL. */
aplicur_status aplicur_get_indices(aplicur_handle h, int32_t* I, int32_t* J, int32_t* ell);

/* Copy the sketch Y = S A (s x n, column-major, FP64) to device memory y_out;
 * *s_out (host) receives s. */
aplicur_status aplicur_get_sketch(aplicur_handle h, double* y_out, int32_t* s_out);

/* Summary of the last solve (host struct). */
aplicur_status aplicur_get_stats(aplicur_handle h, aplicur_stats* st);

/* Per-phase record k of the last solve: CUR rank, LSQR iterations, stop reason
 * (0 none, 1 exact, 2 replay, 3 Paige-Saunders test 2, 4 test 1, 5 dynamic,
 * 6 tol, 7 maxit, 9 drift: the recurrence estimate passed tol but the FP64
 * residual did not, so the phase ends and the next one restarts from an
 * exactly formed residual; 10 inner: FP32-sum inner solve reduced its residual
 * estimate by 1e-4), relative normal-equation residual at the phase end (evaluated as
 * the statistic ne_res is). */
aplicur_status aplicur_get_phase(aplicur_handle h, int32_t k, int32_t* ell, int64_t* iters,
                                 int32_t* reason, double* ne_res);

/* Per-rank-step record k of the last solve: rank after the step, norm estimate
 * rho (Eq. 2normestimate), whether the preconditioner was rebuilt, and the
 * smallest relative LUPP pivot margin of the step (near-tie indicator). */
aplicur_status aplicur_get_step(aplicur_handle h, int32_t k, int32_t* ell, double* rho,
                                int32_t* rebuilt, double* margin);

/* The current preconditioner: rank ell (host) and, when the pointers are not
 * NULL, sigma (device ell doubles, singular values of the CUR approximation,
 * descending) and its target level sigma-hat (host). */
aplicur_status aplicur_get_preconditioner(aplicur_handle h, int32_t* ell, double* sigma,
                                          double* sighat);

/* Apply the current preconditioner: out = P^{-1} w (Eq. preconditioner2 inverted),
 * w and out device n doubles.  ell = 0 gives the identity. */
aplicur_status aplicur_apply_preconditioner(aplicur_handle h, const double* w, double* out);

/* y = A x (trans = 0, x: n, y: m) or y = A^T x (trans = 1, x: m, y: n), device
 * doubles, with the solver's kernels in its precision mode. */
aplicur_status aplicur_matvec(aplicur_handle h, int32_t trans, const double* x, double* y);

/* Hot-loop kernel times and the launch count (host struct). */
aplicur_status aplicur_get_profile(aplicur_handle h, aplicur_profile* out);

/* Zero the accumulated kernel times of h. */
aplicur_status aplicur_reset_profile(aplicur_handle h);

/* Kernels this process has launched through the library (every handle). */
int64_t aplicur_launch_count(void);

/* Device allocations this process made through the library's own stream-ordered
 * allocator (cudaMallocAsync), i.e. without a caller allocator (every handle). */
int64_t aplicur_internal_alloc_count(void);

/* y = A^T x for a dense row-major A (FP64 or FP32 values, FP64 products and sums)
 * without allocating any device or host memory.  The paper has no counterpart; it
 * is for callers that cannot allocate: code running inside a fixed memory budget
 * or a pre-allocated arena (an inference server's pool, an embedding application
 * that owns all device memory) and code paths where an allocation would
 * synchronise or fail.
 *  A   host struct: format APLICUR_DENSE_ROWMAJOR, dtype F64 or F32, values on the
 *      device, m, n >= 1, ld >= n, n <= 524288.
 *  x   device, m doubles; y device, n doubles (overwritten).
 *  stream  cudaStream_t as void*, a stream of the current device.
 * A, x and y must live on the current device: the scratch address is that device's
 * copy of the array, so a call made with another device current would hand the
 * kernels the wrong device's scratch.
 * The only scratch, 4 MiB of row-chunk partial sums, is a static device array that
 * every GPU loading the library keeps until the process exits.  All calls share it:
 * calls that may overlap on the GPU (different streams, threads) race and must be
 * serialised by the caller.  Each call overwrites the part it reads, so no state
 * carries over.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Errors: EINVAL (null pointer, not dense, n above the limit; message through
 * aplicur_last_error(NULL)), ECUDA.  The call does not synchronise. */
aplicur_status aplicur_dense_atx_noalloc(const aplicur_matrix* A, const double* x, double* y,
                                         void* stream);

/* ---- Batched solves ------------------------------------------------------------------
 * nprob independent problems  min ||A_p x - b_{p,r}||^2 + mu ||x||^2,  r < nrhs, with
 * FP32 matrices of uneven sizes.  APLICUR (Algorithm "APLICUR: detailed implementation")
 * runs per problem: each problem gets its own sparse sign sketch (seed opt.seed + p), CUR
 * rank steps and preconditioner builds, and its right-hand sides share them; each pair
 * (p, r) runs its own LSQR recurrences (warm-started phases, Paige-Saunders and dynamic
 * stopping tests of Section 5.3.2) and leaves the solve when its own normal-equation
 * residual reaches tol, so a pair's result is that of a single-right-hand-side solve of
 * (A_p, b_{p,r}).  The rank steps and builds of different problems run concurrently on
 * their own streams; the LSQR iterations of all pairs run as grouped kernels (one launch
 * per step of the iteration covers every problem, products with A are SpMM / tall-skinny
 * GEMM over the nrhs block), captured in CUDA graphs.  Products use FP32 values and FP32
 * sums; every phase starts from the normal-equation residual g = A^T (b - A x) - mu x
 * formed with compensated FP32 products (about 2^-44 relative) and solves for the
 * correction with right-hand side [0; g / sqrt(mu)], whose normal equations are those of
 * the paper's warm start; the stopping tests use the paper's residual estimate.  Dense
 * tile shapes are picked by timing candidates at creation. */
typedef struct aplicur_batch_ctx* aplicur_batch_handle;

typedef struct {
  int32_t pairs;              /* nprob * nrhs */
  int32_t converged;          /* pairs with normal-equation residual <= tol */
  int64_t iters_max;          /* largest LSQR iteration count of a pair */
  int64_t iters_sum;          /* LSQR iterations of all pairs */
  double ne_max;              /* largest relative normal-equation residual */
  double time_setup_ms;       /* creation: sketches, ||A^T b||, tuning (host clock) */
  double time_rank_ms, time_build_ms, time_lsqr_ms, time_check_ms;  /* last solve */
  int32_t rows_per_warp;      /* tuned dense A-pass tile */
  int32_t cols_per_lane;      /* tuned dense A^T-pass tile */
  int64_t launches_per_iter;  /* kernel launches of one grouped LSQR iteration */
} aplicur_batch_stats;

/* Create a batch.
 *  A      host array of nprob matrices: format dense row-major (any ld >= n) or CSR, dtype
 *         F32, values on the device, m_p >= n_p >= sketch_dim; borrowed until destroy.
 *  b      host array of nprob device pointers, each m_p x nrhs FP64 column-major; borrowed.
 *  nrhs   1..16.   mu > 0 (the refinement solves for corrections through the damping rows).
 *  opt    as for aplicur_create (precision, replay and profile are ignored).
 *  stream the stream of the grouped LSQR kernels (NULL: a private stream).
 * Requires n_p * (nrhs rounded up to 4 or 16) * 4 bytes <= 200 KiB (n_p <= 3200 at 16
 * right-hand sides).  Errors: EINVAL, ENOMEM, ECUDA; message via aplicur_batch_last_error. */
aplicur_status aplicur_batch_create(aplicur_batch_handle* out, int32_t nprob,
                                    const aplicur_matrix* A, const double* const* b,
                                    int32_t nrhs, double mu, int32_t sketch_dim,
                                    const aplicur_options* opt, void* stream);

/* Solve every pair to the relative normal-equation residual tol (as aplicur_solve), at
 * most maxit LSQR iterations per pair.  Unlike aplicur_solve, a breakdown in one problem
 * does not fail the batch (see aplicur_batch_get_problem).  After the rank steps, phases without the dynamic
 * test continue until tol, the budget, 4 * max_extra_phases phases, or a phase that gains
 * less than 10%.  x_out: host array of nprob device pointers, each
 * n_p x nrhs FP64 column-major (overwritten).  ENOTCONV when a pair missed tol (x still
 * written). */
aplicur_status aplicur_batch_solve(aplicur_batch_handle h, double tol, int64_t maxit,
                                   double* const* x_out);

/* The same batch by unpreconditioned LSQR with the same grouped kernels (P = I). */
aplicur_status aplicur_batch_plain_lsqr(aplicur_batch_handle h, double tol, int64_t maxit,
                                        double* const* x_out);

/* Adjoint of the last aplicur_batch_solve / aplicur_batch_plain_lsqr (Section "adjoint"
 * of the single-problem entry, per pair): with the incoming gradients g_{p,r} = dL/dx_{p,r}
 * (grad_x: nprob device pointers, each n_p x nrhs FP64 column-major; borrowed), solves
 * (A_p^T A_p + mu I) lambda = g with the preconditioners the solve built (batched
 * correction-form phases to the normal-equation residual tol relative to ||g||), then
 * writes, for every output that is not NULL:
 *   grad_b[p]  (m_p x nrhs FP64 column-major, device)  dL/db = A_p lambda;
 *   grad_mu    (nprob * nrhs FP64, device, index p * nrhs + r)  dL/dmu = -lambda^T x;
 *   grad_A[p]  (m_p x n_p FP32 row-major, device; dense problems only)  dL/dA_p =
 *              sum_r r_r lambda_r^T - (A_p lambda_r) x_r^T,  r_r = b_r - A_p x_r.
 * The forward solutions stay in place (aplicur_batch_get_pair and the statistics then
 * report the adjoint solves).  ENOTCONV when a pair missed tol (outputs still written);
 * EINVAL without a prior solve or for grad_A of a CSR problem. */
aplicur_status aplicur_batch_backward(aplicur_batch_handle h, const double* const* grad_x,
                                     double tol, int64_t maxit, double* const* grad_b,
                                     double* grad_mu, float* const* grad_A);

/* Result of pair (p, r) of the last solve (or adjoint); any output may be NULL. */
aplicur_status aplicur_batch_get_pair(aplicur_batch_handle h, int32_t p, int32_t r,
                                      int64_t* iters, double* ne_res, int32_t* converged);

/* CUR state of problem p after the last solve: rank, rank steps, phases, whether a
 * factorisation broke down (1: the Cholesky of C^T C or of the Q_R update met a non-positive
 * pivot even with FP64 products; the problem's rank growth stopped there and its right-hand
 * sides finished with the last preconditioner it had), and the row and column indices in
 * selection order (I, J: host, >= ell entries, or NULL).  Any output may be NULL. */
aplicur_status aplicur_batch_get_problem(aplicur_batch_handle h, int32_t p, int32_t* ell,
                                         int32_t* nsteps, int32_t* nphases, int32_t* broke,
                                         int32_t* I, int32_t* J);

aplicur_status aplicur_batch_get_stats(aplicur_batch_handle h, aplicur_batch_stats* st);

/* Message of the last failed call on h (never NULL); NULL: last failed create. */
const char* aplicur_batch_last_error(aplicur_batch_handle h);

void aplicur_batch_destroy(aplicur_batch_handle h);

/* Message of the last failed call on h (never NULL); with h = NULL, the last
 * failed aplicur_create or aplicur_dense_atx_noalloc of this thread. */
const char* aplicur_last_error(aplicur_handle h);

/* Static description of a status code (never NULL). */
const char* aplicur_status_string(aplicur_status st);

/* Free everything the handle owns.  NULL is ignored. */
void aplicur_destroy(aplicur_handle h);

#ifdef __cplusplus
}
#endif

#endif /* APLICUR_H_ */
