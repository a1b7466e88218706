/*
 * h2ulv.h -- C ABI of the GB300 (sm_103a) dependency-free H^2-ULV solver.
 *
 * The method is the one of Ma, Deshmukh and Yokota, "Scalable Linear Time
 * Dense Direct Solver for 3-D Problems Without Trailing Sub-Matrix
 * Dependencies" (arXiv 2208.10907): a dense kernel matrix A_ij = K(x_i, x_j)
 * over a point cloud is compressed as an H^2 matrix with strong
 * admissibility (Sec. I), the fill-ins of the dense-block factorization are
 * pre-computed and folded into the shared bases (Sec. III-B/C, eq. fillu and
 * eq. fillv), and every level is then factored box by box without trailing
 * sub-matrix dependencies (eq. rs, eq. ss, eq. lu ... eq. BLR2final).
 *
 * Conventions for every entry point:
 *   - All functions return an h2_status; nothing throws across the ABI.  On
 *     error, h2_last_error() returns a thread-local message.
 *   - Array arguments are plain pointers that may point to host memory or
 *     to device memory of the current CUDA device; the library detects which
 *     (cudaPointerGetAttributes) and copies host buffers itself.
 *   - The caller owns every array it passes; the library copies what it
 *     keeps.  The library owns all factor storage through the handle until
 *     h2_destroy().
 *   - Work is issued on the stream given to h2_construct (NULL = legacy
 *     default stream).  Calls that return values to host memory synchronise
 *     that stream.
 *   - Vectors are in the caller's point order (the tree permutation is
 *     internal); multiple right-hand sides are column-major with leading
 *     dimension ld >= N.
 */
#ifndef H2ULV_H
#define H2ULV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  H2_OK = 0,
  H2_ERR_ARG = 1,           /* invalid argument (null pointer, size, tolerance) */
  H2_ERR_NONFINITE = 2,     /* NaN or Inf in the points or the right-hand side  */
  H2_ERR_OOM = 3,           /* device allocation failed                         */
  H2_ERR_BUDGET = 4,        /* the memory plan exceeds hbm_budget_bytes         */
  H2_ERR_SINGULAR = 5,      /* zero pivot in a redundant-block or root LU       */
  H2_ERR_RANK_CAP = 6,      /* reserved: rank cap violated by a predicted size  */
  H2_ERR_NOT_CONVERGED = 7, /* refinement stopped at max_iter above the target  */
  H2_ERR_DEVICE = 8,        /* CUDA error (message in h2_last_error)            */
  H2_ERR_STATE = 9,         /* call out of order (e.g. solve before factor)     */
  H2_ERR_NOT_SPD = 10,      /* Cholesky pivot <= 0 in the SPD path              */
  H2_ERR_TIMEOUT = 11       /* a bounded device-side wait gave up               */
} h2_status;

/* Kernel functions (Sec. IV: Laplace Green's function; Sec. V: Yukawa).
 * The point singularity of 1/(4 pi r) is regularised:
 *   H2_K_LAPLACE : K = 1 / (r + delta)
 *   H2_K_YUKAWA  : K = exp(-kappa r) / (r + delta)
 *   H2_K_MATERN32: K = (1 + sqrt(3) r / ell) exp(-sqrt(3) r / ell), plus
 *                  nugget on the diagonal (r == 0). */
typedef enum { H2_K_LAPLACE = 0, H2_K_YUKAWA = 1, H2_K_MATERN32 = 2 } h2_kernel_kind;

typedef struct {
  int32_t kind;    /* h2_kernel_kind */
  double delta;    /* regulariser of 1/r, e.g. 1e-3 */
  double kappa;    /* Yukawa decay, e.g. 1 */
  double ell;      /* Matern length scale, e.g. 0.1 */
  double nugget;   /* Matern diagonal shift, e.g. 1e-4 */
} h2_kernel;

/* Construction options (Sec. I admissibility, Sec. II-A rank tolerance,
 * Sec. IV-C leaf size).  far_s0 / far_smin set the deterministic far-field
 * sample of each box's block row: the far boxes of the box's own level give
 * far_s0 points each, one level up far_s0/2, ... never fewer than far_smin;
 * far_s0 = 0 takes every far point (exact block row, small N only). */
typedef struct {
  double eta;          /* strong admissibility: far iff max(diam) <= eta*dist */
  int32_t leaf;        /* maximum points per leaf box (<= 256) */
  double tol;          /* relative rank tolerance of the pivoted QR / ID */
  int32_t max_rank;    /* rank cap (<= 256; a parent box then has up to 512 skeletons) */
  int32_t far_s0;      /* far-field sample per far box at the box's level */
  int32_t far_smin;    /* minimum sample per far box */
  int64_t hbm_budget_bytes; /* 0 = no budget check */
  int32_t partition;   /* cluster tree: 0 = coordinate bisection (split along the
                          longest side at the median), 1 = balanced 2-means
                          (Sec. V's k-means partition with a power-of-two number of
                          leaves: every box split into its floor(n/2) points nearest
                          one Lloyd centroid and the rest) */
} h2_options;

/* Precision of the factorization.  The rank decisions (pivoted QR/ID), the
 * redundant-block LU/Cholesky pivots and the refinement residual are FP64
 * in every mode.  H2_MIXED runs the dense products (fill-ins, projections,
 * Schur updates, far-field Gram) in split 3xTF32 on the tensor cores: each
 * FP32 operand is split into two TF32 parts and three products accumulate
 * in FP32.  There is no split-BF16 mode: three BF16 parts need six
 * products for the same accuracy, at twice the TF32 rate, i.e. the same
 * tensor-core time. */
typedef enum { H2_FP64 = 0, H2_MIXED = 1 } h2_precision;

typedef struct h2_handle_* h2_handle;

/* Build the cluster tree (coordinate bisection), the strong-admissibility
 * near/far lists and the H^2 operator used as the refinement residual:
 * nested interpolative bases from the far-field block rows (eq. u,
 * Sec. II-D: dense blocks never enter the basis) and the dense leaf near
 * blocks.
 *   points : N x 3 row-major doubles (host or device), caller order
 *   N      : number of points, >= 1
 *   kern   : kernel description (host pointer)
 *   opt    : options (host pointer); leaf in [1,256], max_rank in [1,256],
 *            tol >= 0, eta > 0
 *   stream : cudaStream_t to issue work on (NULL = default stream)
 *   out    : receives the handle
 * Errors: H2_ERR_ARG, H2_ERR_NONFINITE (non-finite coordinate),
 * H2_ERR_BUDGET, H2_ERR_OOM, H2_ERR_DEVICE. */
h2_status h2_construct(const double* points, int64_t N, const h2_kernel* kern,
                       const h2_options* opt, void* stream, h2_handle* out);

/* Batched construct over P independent problems (each its own tree); the
 * factor and solve then run every box of every problem at the same height
 * above the leaves in one launch per step.
 *   points[p] : N[p] x 3 row-major doubles of problem p
 * Right-hand sides of a batched handle are stacked problem after problem
 * (rows offset by the prefix sum of N). */
h2_status h2_construct_batched(int32_t P, const double* const* points, const int64_t* N,
                               const h2_kernel* kern, const h2_options* opt, void* stream,
                               h2_handle* out);

/* Dependency-free H^2-ULV factorization, level by level from the leaves
 * (Sec. III-B fill-in pre-computation, Sec. III-C shared basis with
 * fill-ins, eq. rs / eq. ss projection, eq. lu partial LU, merge, and the
 * dense LU of eq. BLR2final at the top).
 *   precision : H2_FP64 or H2_MIXED
 *   spd       : nonzero = Cholesky instead of LU (symmetric positive
 *               definite kernels only)
 * Basis of each box (eq. fillu), by one of two routes:
 *   "qr"   : Householder QR of the block row [fill-ins | far field] (the
 *            fill-ins sharing a box K enter as A_IK A_KK^-1 R_K^T, R_K the
 *            QR triangle of [A_KJ]_J^T), then column-pivoted QR; resolves
 *            the block row to FP64 rounding.  H2_FP64 with tol < 2^-20.
 *   "gram" : the Gram matrix of the same block row and pivoted Cholesky
 *            (same pivots in exact arithmetic); it resolves the block row
 *            only to about sqrt(eps) of its norm in FP64 and 2^-10 in FP32.
 *            H2_FP64 with tol >= 2^-20 (tol used as given) and H2_MIXED
 *            (FP32 on the tensor cores, rank tolerance max(tol, 2^-10);
 *            the factors precondition the FP64 refinement).
 * h2_stats reports the route ("basis_route": "qr" or "gram") and the
 * tolerance the bases used ("tol_basis").
 * Errors: H2_ERR_SINGULAR, H2_ERR_NOT_SPD, H2_ERR_NONFINITE (non-finite
 * value in a block row), H2_ERR_OOM, H2_ERR_DEVICE, H2_ERR_TIMEOUT. */
h2_status h2_factor(h2_handle h, int32_t precision, int32_t spd);

/* Solve A x = b with the ULV factors (Sec. II-B: L z = U^T b, U y = z,
 * x = V^T y) and FP64 iterative refinement whose residual is the H^2
 * matvec, until ||b - A_H2 x|| / ||b|| <= target for every right-hand side
 * or max_iter corrections were applied.  With nrhs <= 8 the correction
 * equation is solved by GMRES(30) preconditioned by the ULV factors (each
 * Arnoldi step = one ULV solve + one H^2 matvec, counted as one
 * correction); otherwise x <- x + ULV^-1 (b - A_H2 x).
 *   b, x   : N x nrhs column-major, leading dimension ld (host or device)
 *   achieved_rel_residual : host array of nrhs (may be NULL)
 *   iters  : host int, corrections applied (may be NULL)
 * Errors: H2_ERR_STATE (not factored), H2_ERR_ARG, H2_ERR_NOT_CONVERGED
 * (x still holds the last iterate). */
h2_status h2_solve(h2_handle h, const double* b, double* x, int32_t nrhs, int64_t ld,
                   double target_rel_residual, int32_t max_iter,
                   double* achieved_rel_residual, int32_t* iters);

/* Solve every problem of a batched handle with its own right-hand sides
 * (Sec. II-B solve and the FP64 refinement of h2_solve), all problems in the
 * same launches.
 *   b[p], x[p] : N[p] x nrhs[p] column-major, leading dimension ld[p] >= N[p]
 *                (host or device), in problem p's caller order
 *   nrhs[p]    : right-hand sides of problem p (>= 1)
 *   achieved_rel_residual : host array of P (may be NULL): per problem, the
 *                largest ||b - A_H2 x|| / ||b|| over its columns
 *   iters      : host int, corrections applied (may be NULL)
 * The columns are stacked and padded with zero columns to the largest
 * nrhs[p], so the cost is that of max_p nrhs[p] columns over all problems.
 * The refinement is the stationary one (x <- x + ULV^-1 (b - A_H2 x)), which
 * acts on each problem separately, and every column of every problem must
 * reach the target on its own norm.  Stacked work buffers are kept by the
 * handle between calls.
 * Errors: H2_ERR_STATE (not factored), H2_ERR_ARG, H2_ERR_NONFINITE,
 * H2_ERR_NOT_CONVERGED (x still holds the last iterate). */
h2_status h2_solve_batched(h2_handle h, const double* const* b, double* const* x, const int32_t* nrhs,
                           const int64_t* ld, double target_rel_residual, int32_t max_iter,
                           double* achieved_rel_residual, int32_t* iters);

/* y = A_H2 x, the H^2 operator used as the refinement residual (near blocks
 * exact, far blocks through the nested bases, eq. transfer).
 *   x, y : N x nrhs column-major, leading dimension ld (host or device)
 * With nrhs = 1 the near-field products run in double-float arithmetic
 * (FP64 entries split exactly into FP32 pairs; about 2^-46 relative per
 * product); the far field and all sums are FP64. */
h2_status h2_matvec(h2_handle h, const double* x, double* y, int32_t nrhs, int64_t ld);

/* log|det A| and its sign from the factorization: the sum over every level
 * and box of log|det S^RR_II| plus the root's (|det Q_I| = 1).  For a
 * batched handle, problem p's value is written to log_abs_det[p] (host
 * arrays of length P). */
h2_status h2_logdet(h2_handle h, double* log_abs_det, int32_t* sign);

/* Allocation-free variant of h2_logdet, for callers that cannot call
 * cudaMalloc when they need the value (their device memory is fully reserved
 * or owned by another allocator, or they must not trigger an allocation
 * between latency-critical launches).  The paper has no counterpart: it is
 * an interface addition of this library.  Same result as h2_logdet (host
 * arrays of length P for a batched handle).
 *   - Scratch: a fixed 1 MB device array inside the library (task
 *     descriptors and per-block partials), held by every device that loads
 *     the library until the process exits; nothing is allocated per call.
 *   - Limit: at most 16384 factored blocks per tree height; larger handles
 *     are rejected with H2_ERR_ARG.
 *   - The array used is the one on the device that was current when the
 *     handle was constructed (the call makes that device current and
 *     restores the caller's current device before returning).
 *   - The first call on a device looks up the array's device address (once
 *     per device); make that first call before any stream capture.
 *   - Every call shares the array and it keeps the last call's contents;
 *     calls that overlap on the GPU (several host threads or handles at
 *     once) race on it and must be serialised by the caller. */
h2_status h2_logdet_noalloc(h2_handle h, double* log_abs_det, int32_t* sign);

/* JSON statistics: per-level ranks, flops, bytes, times (ms), the basis
 * route and effective rank tolerance of the last factorization; cap = size
 * of the host buffer json.  Truncated output is still NUL-terminated. */
h2_status h2_stats(h2_handle h, char* json, size_t cap);

/* Per-kernel instrumentation shared by all handles of the process.  Every
 * launch is counted; with enable = 1 each launch is also bracketed by CUDA
 * events on the stream it runs on, and h2_stats reports, per kernel, its
 * launches, summed event time (ms) and the algorithmic flops and bytes its
 * callers declared.  reset = 1 clears the counters first. */
h2_status h2_profile(int32_t enable, int32_t reset);

/* ---------------------------------------------------------------------
 * Rank predictor (an interface addition; the paper has no learned part).
 * A 3-layer MLP (8 box features -> 64 -> 64 -> 1, tanh, FP32) trained on the
 * GPU by the library's own forward / backward / Adam kernels on
 * (box features -> rank of the pivoted QR of the block row) pairs.  Given
 * to a handle, it predicts every box's rank before the basis pass so that
 * the next level's block storage is sized and allocated while the basis
 * kernels run; the pivoted QR still decides every rank, and a box whose
 * rank exceeds its prediction plus the margin falls back to exact sizing.
 * Parameter layout: W1 (64 x 8, row-major), b1 (64), W2 (64 x 64), b2 (64),
 * w3 (64), b3 (1).  Arrays may be host or device pointers. */
typedef struct h2_mlp_* h2_mlp;

/* Number of parameters for n_features inputs (4801 for 8). */
int32_t h2_mlp_param_count(int32_t n_features);

/* Create a predictor from initial parameters (caller-drawn, length
 * h2_mlp_param_count(8)); n_features must be 8. */
h2_status h2_mlp_create(int32_t n_features, const float* init_params, void* stream, h2_mlp* out);

/* steps full-batch Adam steps on mean((f(X) - T)^2); X is B x 8 row-major,
 * T has B targets; final_loss (host, may be NULL) receives the loss after
 * training. */
h2_status h2_mlp_train(h2_mlp m, const float* X, const float* T, int32_t B, int32_t steps, float lr,
                       float* final_loss);

/* Y = f(X) for B samples. */
h2_status h2_mlp_forward(h2_mlp m, const float* X, int32_t B, float* Y);

/* Gradient of mean((f(X) - T)^2) with respect to the parameters (length
 * h2_mlp_param_count) and the loss; parameters are not changed. */
h2_status h2_mlp_gradient(h2_mlp m, const float* X, const float* T, int32_t B, float* grad, float* loss);

/* Copy the current parameters out. */
h2_status h2_mlp_params(h2_mlp m, float* out);

const char* h2_mlp_last_error(void);
void h2_mlp_destroy(h2_mlp m);

/* Features of every box at one height (8 floats per box, row-major) and,
 * after h2_factor, the rank the pivoted QR chose for each box (training
 * targets).  features or ranks may be NULL; *nboxes receives the count. */
h2_status h2_box_features(h2_handle h, int32_t height, float* features, int32_t* ranks, int32_t* nboxes);

/* Use m (kept by reference; NULL detaches) to size each level's storage
 * before its basis pass; a box is covered when its rank is at most
 * (1 + margin) times its predicted rank plus 4.  h2_stats reports hits,
 * misses and the bytes sized up front. */
h2_status h2_set_rank_predictor(h2_handle h, h2_mlp m, double margin);

/* Thread-local message of the last failed call on this thread. */
const char* h2_last_error(void);

/* Free every device buffer owned by the handle, and the library's cache of
 * released scratch buffers (kept between calls for reuse on the same
 * stream). */
void h2_destroy(h2_handle h);

#ifdef __cplusplus
}
#endif
#endif /* H2ULV_H */
