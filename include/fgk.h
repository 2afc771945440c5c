/*
 * libfgk — exact fast Matérn-kernel matrix-vector products and GP solves on
 * one NVIDIA GB300 (sm_103a).
 *
 * The library computes, exactly up to rounding,
 *
 *     Y = K V,   K_ij = s2 * K(x_i - x_j),                  (Sec. 2, eq. Ky)
 *
 * for the half-integer Matérn kernels nu = 1/2, 3/2, 5/2, 7/2, 9/2 (App. C.1,
 * eqs. matern_1_2 ... matern_9_2, eq. matern_explicit) combined over d <= 3
 * coordinates
 * either through the L1 norm, K(u) = k(sum_k |u_k| / ell_k) (eq. L1_kernel),
 * or as a product, K(u) = prod_k k(|u_k| / ell_k) (eq. product_kernel), with
 * one lengthscale per dimension (eq. scaled_kernel read per dimension).  It
 * does so by the paper's decomposition of the kernel sum into weighted
 * empirical CDFs (Propositions 1 and 2, eqs. L1_decomposition and
 * product_decomposition), evaluated over a dominance structure whose sorted
 * subsets are computed once per point set and kept on the device (Sec. 2.2.3).
 * On top of the product it solves (K + sigma^2 I) alpha = y by conjugate
 * gradients (App. A.1, Algorithm 2 with the identity or the pivoted-Cholesky
 * preconditioner of App. A.3), with an optional generalised-least-squares
 * fixed-effects mean (Sec. 3.2, Algorithm 1's GLS step), and provides the
 * pieces of the likelihood and its gradient (eqs. gp_log_likelihood and
 * gp_log_likelihood_derivative): products with the lengthscale derivatives of
 * K (App. C.1), log det(K + sigma^2 I) by stochastic Lanczos quadrature
 * (App. A.2), the gradient with Hutchinson probes, and the posterior mean at
 * new points (eq. gp_mean).
 *
 * Conventions for every entry point:
 *  - Pointers documented "device" must be device memory of the current CUDA
 *    device; "host" means ordinary host memory.  The caller owns every
 *    pointer it passes; the library never frees or keeps them past the call
 *    (fgk_build copies what it needs).
 *  - Arrays of points and vectors are row-major: X is N x d, V and Y are
 *    N x nrhs (the nrhs values of one point are contiguous), in the caller's
 *    original point order.
 *  - Work is enqueued on the given stream (NULL = legacy default stream);
 *    calls on one handle must be ordered on one stream (a handle owns one
 *    workspace).  fgk_build, the solves (fgk_cg_solve, fgk_cg_solve_pc,
 *    fgk_slq_logdet, fgk_loglik_grad) and fgk_precond_build synchronise that
 *    stream before returning; the products (fgk_matvec, fgk_matvec_q,
 *    fgk_matvec_dlogell) do not.
 *  - Return value: FGK_OK (0) on success, a negative FGK_ERR_* code on
 *    failure (nothing is thrown across the ABI); fgk_last_error() then gives
 *    a message for the calling thread.  FGK_NOT_CONVERGED (1) is a soft
 *    result of fgk_cg_solve.
 *  - Error codes, where an entry lists none of its own: FGK_ERR_INVALID for
 *    a NULL handle or required pointer or a count outside its documented
 *    range (checked before any device work is enqueued); FGK_ERR_OOM when a
 *    device allocation fails; FGK_ERR_CUDA when a CUDA call or a kernel
 *    launch fails; FGK_ERR_TIMEOUT when a bounded device-side wait expires;
 *    FGK_ERR_INTERNAL when a device-side consistency check fails.  The sizes
 *    of caller buffers cannot be checked: they must match the documented
 *    shapes.  An asynchronous call reports what it sees at enqueue time.
 */
#ifndef FGK_H
#define FGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t, spelled without the CUDA headers (same underlying type). */
typedef struct CUstream_st *fgk_stream_t;

typedef struct fgk_plan *fgk_handle;

enum fgk_status {
    FGK_OK = 0,
    FGK_NOT_CONVERGED = 1,  /* CG stopped at maxit above tol; outputs hold the best iterate */
    FGK_ERR_INVALID = -1,   /* an argument is out of range */
    FGK_ERR_NONFINITE = -2, /* NaN or Inf in an input */
    FGK_ERR_OOM = -3,       /* device allocation failed */
    FGK_ERR_CUDA = -4,      /* a CUDA call failed; the message names it */
    FGK_ERR_BREAKDOWN = -5, /* CG met p^T A p <= 0: the system is not positive definite */
    FGK_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
    FGK_ERR_INTERNAL = -7   /* a device-side consistency check failed */
};

enum fgk_kind { FGK_L1 = 0, FGK_PRODUCT = 1 };
enum fgk_precision { FGK_F64 = 0, FGK_F32 = 1, FGK_MIXED = 2 };

/* Device allocator used for the handle's memory and workspace.  alloc must
 * return device memory usable on `stream` (NULL on failure); free releases
 * it.  Default (or after passing NULL, NULL): cudaMallocAsync/cudaFreeAsync.
 * The setting is process-wide and applies to allocations made after it. */
typedef void *(*fgk_alloc_fn)(size_t bytes, fgk_stream_t stream, void *ctx);
typedef void (*fgk_free_fn)(void *ptr, fgk_stream_t stream, void *ctx);
int fgk_set_allocator(fgk_alloc_fn alloc, fgk_free_fn free_fn, void *ctx);

/* Build the cached sort and dominance structure of a point set
 * (Sec. 2.1: sorting then fast sum updating; Sec. 2.2.3: the sorted subsets
 * of the divide and conquer stored in a data structure; eq. scaled_kernel
 * for ell and outscale2).
 *   X          device, N x d FP64 row-major; finite (else FGK_ERR_NONFINITE).
 *   N          1 <= N <= 2^30.
 *   d          1, 2 or 3.
 *   two_nu     2 nu: 1, 3, 5, 7 or 9 (9 only with d <= 2).  nu = 7/2 and
 *              9/2 (eqs. matern_7_2, matern_9_2) run the scans with four and
 *              five moments and run-time coefficients; the batch calls take
 *              nu <= 5/2, the lengthscale-derivative products nu <= 7/2
 *              (nu <= 5/2 at d = 3).
 *   ell        host, d lengthscales, finite and > 0.
 *   outscale2  varsigma^2 > 0 (1 when the kernel has no outputscale).
 *   kind       FGK_L1 or FGK_PRODUCT (identical when two_nu == 1 or d == 1).
 *   out        host; receives the handle (NULL on failure).
 * The handle owns device memory of about fgk_bytes_estimate(...) bytes and
 * must be released with fgk_destroy. */
int fgk_build(const double *X, int64_t N, int d, int two_nu, const double *ell, double outscale2,
              int kind, fgk_stream_t stream, fgk_handle *out);

/* Y = K V (eq. Ky for nrhs columns at once; the kernel sum of eq. kde for
 * every z in the point set).
 *   V, Y       device, N x nrhs row-major, original point order; FP64 when
 *              precision == FGK_F64, FP32 when precision == FGK_F32.  V must
 *              be finite; V and Y must not overlap.
 *   nrhs       >= 1.
 *   precision  FGK_F64 (FP64 scans) or FGK_F32 (FP32 scans, FP32 in/out).
 * Asynchronous on `stream`. */
int fgk_matvec(fgk_handle h, const void *V, int nrhs, void *Y, int precision, fgk_stream_t stream);

/* Y = (dK / d log ell_dim) V: the product with the lengthscale derivative of
 * K that the trace term of the likelihood gradient needs
 * (eq. gp_log_likelihood_derivative, tr((K + sigma^2 I)^{-1} dK/dtheta) by
 * Hutchinson probes, App. A.2), from the gradient formulas of App. C.1.  The
 * derivative is taken with respect to log ell (ell times the paper's
 * d/d ell): divide column-wise by ell_dim for d/d ell_dim.
 *   dim        0 <= dim < d: the lengthscale of coordinate dim; product
 *              kernel (or d == 1).
 *              -1: every lengthscale scaled together (ell_k -> t ell_k,
 *              derivative at t = 1, i.e. the sum of the d per-coordinate
 *              derivatives); for one isotropic lengthscale this is
 *              ell dK/d ell, the paper's gradient formulas.  Any kernel.
 *              The L1 kernel with d > 1 takes only -1 (its per-coordinate
 *              derivative is not a function of the L1 distance alone):
 *              other values give FGK_ERR_INVALID.
 *   V, Y, nrhs, precision as fgk_matvec.  The diagonal of the derivative is
 *   zero (self-pairs have distance 0).  Allocates a workspace (cudaMallocAsync
 *   or the installed allocator).  Asynchronous on `stream`. */
int fgk_matvec_dlogell(fgk_handle h, const void *V, int nrhs, void *Y, int dim, int precision,
                       fgk_stream_t stream);

/* Y = K V with V and Y in the plan's internal point order: row q holds the
 * point perm_1[q] (fgk_get_permutation(h, 0, ...)), i.e. the points sorted
 * by their first scaled coordinate.  Iterative methods that keep their
 * vectors in this order (as fgk_cg_solve does) skip the two permutations of
 * fgk_matvec.  Arguments otherwise as fgk_matvec.  Asynchronous. */
int fgk_matvec_q(fgk_handle h, const void *Vq, int nrhs, void *Yq, int precision, fgk_stream_t stream);

/* The product of fgk_matvec_q for callers that must not allocate device
 * memory during the call (their device memory is planned before they start:
 * a serving loop whose budget is already handed out, an engine whose memory
 * plan is fixed, a latency-critical path that cannot afford an allocator
 * call or an out-of-memory error in the middle of its work).  The paper has
 * no counterpart; this is an interface choice.
 * It calls no cudaMalloc, cudaFree or allocating library routine: the
 * scratch of the product (one output row per level, N x nrhs values each,
 * and the tile aggregates of segments longer than a tile) lives in one
 * 64 MiB __device__ array compiled into the library.  The CUDA runtime
 * loads code and such arrays lazily, so the first fgk_build on each device
 * reserves the array there (and looks up its device address), and every
 * fgk_build has the runtime load the product kernels of its plan: build
 * plans while allocation is still allowed.  The array is then held until
 * the process exits.  All calls on a device share the array and it keeps
 * the last call's contents: calls whose work overlaps on the GPU race and
 * must be ordered by the caller.  FGK_ERR_INVALID, without launching
 * anything: a product needing more scratch than the array holds (the need
 * grows with nrhs and with the number of levels), or a call made while
 * another device than the plan's is current.
 * Arguments, layout and precision as fgk_matvec_q; the handle comes from an
 * earlier fgk_build.  Asynchronous. */
int fgk_matvec_q_noalloc(fgk_handle h, const void *Vq, int nrhs, void *Yq, int precision, fgk_stream_t stream);

/* Per-solve report of fgk_cg_solve (host memory, filled on return). */
typedef struct {
    int32_t iterations;     /* CG iterations (the most any column took) */
    int32_t refinements;    /* FP64 true-residual evaluations (residual replacements) */
    int32_t mvm_f32;        /* products taken with FP32 scans */
    int32_t mvm_f64;        /* products taken with FP64 scans */
    double max_true_resid;  /* max over solved columns of ||b - A x|| / ||b||, FP64 */
    double *true_resid;     /* optional host array of nrhs + L doubles (columns
                               [y, H]); written when not NULL */
    int32_t restarts;       /* mixed mode: restarts (p = r on the affected
                               columns) after an FP32 p^T A p <= 0 that FP64
                               scans did not confirm */
    int32_t fp64_switch;    /* fgk_cg_solve, mixed mode: 1 if too many such
                               restarts moved the remaining iterations to FP64 scans */
} fgk_cg_info;

/* Solve (K + sigma2 I) alpha = y (eq. gp_mean_system) for nrhs columns by
 * conjugate gradients (Algorithm 2, identity preconditioner, zero start),
 * optionally with a linear fixed-effects mean m(x) = H beta estimated by
 * generalised least squares, beta = (H^T A^{-1} H)^{-1} H^T A^{-1} y
 * (Sec. 3.2), in which case alpha = A^{-1} (y - H beta) (eq. gp_mean).
 *   y          device, N x nrhs FP64 row-major, original point order.
 *   sigma2     noise variance >= 0.
 *   H, L       fixed effects: H == NULL && L == 0: none; H == NULL && L == -1:
 *              the default H = [1, x_1, ..., x_d] (L = 1 + d, unscaled x);
 *              H != NULL: device N x L FP64 row-major, 1 <= L <= 8.
 *   tol        stop when every column's true relative residual
 *              ||b - A x||_2 / ||b||_2 (recomputed in FP64) is <= tol.
 *   maxit      cap on CG iterations.
 *   mode       FGK_F64: FP64 scans throughout; FGK_MIXED: FP32 scans inside
 *              CG with FP64 inner products and vectors, the residual
 *              recomputed with FP64 scans whenever the
 *              recursive residual has dropped by a factor (env
 *              FGK_MIXED_DELTA, default 0.5) and substituted for it, the
 *              FP64 solution being corrected in place (iterative refinement
 *              without restarting the Krylov space).  An FP32 p^T A p <= 0 is
 *              re-evaluated with FP64 scans: confirmed, it is a breakdown;
 *              otherwise the column restarts from p = r, and after 4 such
 *              restarts the solve continues with FP64 scans.
 *   alpha      device, N x nrhs FP64 (output).
 *   beta       device, L x nrhs FP64 (output) or NULL; ignored without H.
 *   info       host, may be NULL.
 * Returns FGK_OK, FGK_NOT_CONVERGED, FGK_ERR_BREAKDOWN (p^T A p <= 0, e.g.
 * the indefinite L1 kernel at nu >= 3/2, d >= 2) or an error.  Synchronises
 * `stream`. */
int fgk_cg_solve(fgk_handle h, const double *y, int nrhs, double sigma2, const double *H, int L, double tol,
                 int maxit, int mode, double *alpha, double *beta, fgk_cg_info *info, fgk_stream_t stream);

/* The posterior mean at M evaluation points (eq. gp_mean; eq. gp_mean_2 once
 * alpha is known): out[j] = sum_i K(z_j, x_i) alpha_i + h(z_j)^T beta.
 *   h          the plan of the data X (kernel, nu, lengthscales, outscale2).
 *   alpha      device, N x nrhs FP64 row-major, original point order (as
 *              fgk_cg_solve returns it).
 *   Z, M       device, M x d FP64 row-major, unscaled coordinates; M >= 1.
 *   HZ, L      fixed effects at the new points: HZ == NULL && L == 0: none;
 *              HZ == NULL && L == -1: the default h(z) = [1, z_1..z_d];
 *              HZ != NULL: device M x L FP64 row-major, 1 <= L <= 8.
 *   beta       device, L x nrhs FP64 (from fgk_cg_solve), required when L != 0.
 *   precision  FGK_F64 or FGK_F32: the scans of the product.
 *   out        device, M x nrhs FP64 (output).
 * Method: one product over the union of the data and the new points with
 * weights [alpha; 0], read at the new points -- exact (the definition of
 * k_z^T alpha), at the cost of building the union's structure (N + M points).
 * Errors: FGK_ERR_INVALID, FGK_ERR_NONFINITE (alpha or Z), FGK_ERR_OOM.
 * Synchronises `stream`. */
int fgk_predict(fgk_handle h, const double *alpha, int nrhs, const double *Z, int64_t M, const double *HZ, int L,
                const double *beta, int precision, double *out, fgk_stream_t stream);

/* ---- the pivoted-Cholesky preconditioner (App. A.3) ---- */

typedef struct fgk_precond_s *fgk_precond;

typedef struct {
    int32_t rank_requested; /* min(rank, N) as passed to fgk_precond_build */
    int32_t rank;           /* realised rank k (smaller once the largest residual
                               diagonal entry of K - L L^T is at most 1e-12 s2) */
    double sigma2;          /* the noise variance P was built for */
    double trace_resid;     /* trace(K - L L^T): the approximation error */
    double logdet;          /* log det P = N log sigma2 + log det(I_k + L^T L / sigma2)
                               (Sylvester's determinant theorem, App. A.3) */
    size_t device_bytes;    /* device memory held by the preconditioner */
} fgk_precond_report;

/* Build P = L L^T + sigma2 I, where L (N x k) is the rank-k pivoted Cholesky
 * factor of the plan's K (App. A.3, after Harbrecht et al.): at each step the
 * pivot is the point with the largest remaining diagonal of K - L L^T (ties:
 * the smallest original point index), and L gains the column of K at the
 * pivot minus what the earlier columns explain, divided by the square root of
 * that diagonal entry.  The factor is stored in FP32 and each new column is
 * rounded to FP32 before the later columns and the residual diagonal use it,
 * so the factor is the exact pivoted-Cholesky recurrence of its own stored
 * columns (the next columns take up each rounding); its sums are float pairs
 * of exact products (about 48 bits), the divisions and the residual diagonal
 * FP64.  The Woodbury matrix I + L^T L / sigma2 is formed from the stored
 * values, so P is exactly L L^T + sigma2 I for the stored L.
 *   h       a built plan; it must outlive the preconditioner.
 *   rank    0 <= rank <= 1024 (the paper uses 100); rank 0 gives P = sigma2 I.
 *   sigma2  > 0, the noise variance of the systems it will precondition.
 * Device memory: about N x rank x 4 bytes plus O(rank^2) held, and 8 x N bytes
 * per column the applies have taken (the float pairs of R's rows); during the
 * build also 16 x d x N bytes of exponential tables and the Gram partials.  Synchronises
 * `stream`.  Errors: FGK_ERR_INVALID (arguments), FGK_ERR_OOM. */
int fgk_precond_build(fgk_handle h, int rank, double sigma2, fgk_stream_t stream, fgk_precond *out);

/* The report of a built preconditioner; pivots (host, may be NULL) receives
 * the k pivots as original point indices in the order chosen. */
int fgk_precond_info(fgk_precond pc, fgk_precond_report *rep, int64_t *pivots);

/* L (device, N x k FP64 row-major, the caller's point order: row i holds the
 * k factor values of point i).  Asynchronous. */
int fgk_precond_factor(fgk_precond pc, double *L, fgk_stream_t stream);

/* Z = P^{-1} R by the Woodbury formula of App. A.3,
 * P^{-1} R = R / sigma2 - L (I_k + L^T L / sigma2)^{-1} L^T R / sigma2^2.
 * R, Z: device, N x ncols FP64 row-major, original point order,
 * 1 <= ncols <= 64.  Asynchronous (allocates scratch on `stream`).  The
 * scratch belongs to pc, as a plan's workspace belongs to its handle: the
 * calls that use one preconditioner (its applies and the solves it
 * preconditions) must be ordered on one stream. */
int fgk_precond_apply(fgk_precond pc, const double *R, int ncols, double *Z, fgk_stream_t stream);

int fgk_precond_destroy(fgk_precond pc);

/* fgk_cg_solve preconditioned by pc (Algorithm 2 with s_P = P^{-1}): every
 * argument as fgk_cg_solve; pc == NULL is fgk_cg_solve.  pc must come from
 * the same plan and be built for the same sigma2 (else FGK_ERR_INVALID), and
 * the columns solved together, nrhs plus the L fixed-effect columns, must
 * number at most 64 (else FGK_ERR_INVALID, before any device work).  The
 * stop test stays on the unpreconditioned true residual ||b - A x|| / ||b||;
 * in mixed mode the FP32 iterations run until the recursive residual has
 * dropped by FGK_MIXED_DELTA (default 1e-3 here), then the FP64 true
 * residual replaces it and every column restarts from p = P^{-1} r. */
int fgk_cg_solve_pc(fgk_handle h, fgk_precond pc, const double *y, int nrhs, double sigma2, const double *H, int L,
                    double tol, int maxit, int mode, double *alpha, double *beta, fgk_cg_info *info,
                    fgk_stream_t stream);

/* Solve (K + sigma2 I) alpha = y when K + sigma2 I is symmetric but need not
 * be positive definite, by MINRES (Paige and Saunders): the L1 kernel at
 * nu >= 3/2 and d >= 2, which App. B (Prop. 4) shows is not positive
 * definite, so that fgk_cg_solve can stop with FGK_ERR_BREAKDOWN on it.
 * Lanczos vectors from each column b of y, the tridiagonal reduced by Givens
 * rotations, alpha the minimiser of ||b - A x|| over the Krylov space; FP64
 * scans, zero start.  A column stops when its recursive residual is at most
 * tol ||b||; its true residual is then recomputed with FP64 scans and the
 * process restarts on it from the current alpha until that meets tol too.
 *   y, alpha   device, N x nrhs FP64 row-major, original point order
 *              (alpha: output).  1 <= nrhs <= 64.
 *   sigma2     >= 0;  tol > 0;  maxit >= 1 (iterations over all restarts).
 *   info       host, may be NULL: iterations, restarts (in refinements and
 *              restarts), FP64 products, true residuals (true_resid if set).
 * FGK_NOT_CONVERGED when a column misses tol after maxit iterations (alpha
 * holds the best iterate); FGK_ERR_NONFINITE for NaN or Inf in y.
 * Synchronises the stream once per iteration.  Allocates a workspace of
 * 8 N nrhs doubles plus the product's. */
int fgk_minres_solve(fgk_handle h, const double *y, int nrhs, double sigma2, double tol, int maxit, double *alpha,
                     fgk_cg_info *info, fgk_stream_t stream);

/* One d = 1 problem over several devices (the d = 1 product split by point
 * ranges): each device holds a shard, a contiguous range of the points in
 * sorted order, and a plan of its own points; the plan's product covers the
 * pairs inside the shard, and the pairs between shards act through P
 * moments per shard and direction (Sec. 2.1, the fast sum updating of
 * eq. fast_exact_decomposition_1d with the running sums relative to an
 * anchor point):
 *   M_q = sum_j v_j delta_j^q exp(-delta_j),  q < P = nu + 1/2,
 * delta_j = x'_last - x'_j (forward: this shard's sources seen from after
 * it) or x'_j - x'_first (backward), x' the scaled coordinates.
 *
 * fgk_shard_moments: V device N x nrhs FP64, original point order, 1 <= nrhs
 * <= 64; out host, 2 + 2 nrhs P doubles: x'_first, x'_last, then M indexed
 * [(r * 2 + dir) * P + q] (dir 0 forward, 1 backward).  FP64, fixed-order
 * sums.  Synchronises the stream.  d = 1 plans only (FGK_ERR_INVALID).
 *
 * fgk_shard_fixup: Y += the contributions of the other shards' points, given
 * carry (host, 2 nrhs P doubles, the same indexing): dir 0 the moments of
 * every point before this shard anchored at its x'_first, dir 1 those after
 * it anchored at x'_last (the caller composes them from all shards'
 * fgk_shard_moments by the binomial step M'_q = exp(-g) sum_{t<=q} C(q,t)
 * g^{q-t} M_t over each gap g).  Y device N x nrhs FP64, original order.
 * Asynchronous. */
int fgk_shard_moments(fgk_handle h, const double *V, int nrhs, double *out, fgk_stream_t stream);
int fgk_shard_fixup(fgk_handle h, const double *carry, int nrhs, double *Y, fgk_stream_t stream);

/* ---- log-determinant by stochastic Lanczos quadrature (App. A.2) ---- */

/* Probe vectors distributed as N(0, P) for the preconditioned log-determinant
 * estimate: B = L_hi E_r + sigma E_n, where L_hi is the FP32 factor the
 * preconditioner applies (P = L_hi L_hi^T + sigma2 I exactly).  The caller
 * draws the standard normal numbers:
 *   E_r  device, k x nprobe FP64 row-major (k: fgk_precond_info's rank),
 *   E_n  device, N x nprobe FP64 row-major (original point order),
 *   B    device, N x nprobe FP64 row-major (original point order),
 *   1 <= nprobe <= 64.  Asynchronous.  Errors: FGK_ERR_INVALID (a NULL
 * argument, E_r NULL with k > 0 (it may be NULL at k = 0), nprobe outside
 * the range). */
int fgk_precond_sample(fgk_precond pc, const double *E_r, const double *E_n, int nprobe, double *B,
                       fgk_stream_t stream);

typedef struct {
    double logdet;          /* the estimate of log det(K + sigma2 I) */
    double logdet_precond;  /* log det P added to it (0 without a preconditioner) */
    int steps_max;          /* the longest Lanczos process of the probes */
    int solve_status;       /* the CG solve's own return code (FGK_OK or FGK_NOT_CONVERGED) */
    double max_true_resid;  /* of the solves X */
} fgk_slq_report;

/* log det(K + sigma2 I) by stochastic Lanczos quadrature: the trace of the
 * matrix logarithm (eq. approximationLogDet) estimated with the probes B by
 * Hutchinson's estimator, each quadratic form b^T log(.) b taken from the
 * tridiagonal Lanczos matrix T_b that CG with a zero initial guess produces
 * (Algorithm 2: T[k][k] = 1/alpha_k + beta_{k-1}/alpha_{k-1},
 * T[k+1][k] = sqrt(beta_k)/alpha_k) as gamma_b e_1^T log(T_b) e_1, with
 * gamma_b = b^T P^{-1} b the squared norm of the Lanczos start vector (the
 * paper approximates it by N).  With a preconditioner the quadrature is of
 * P^{-1/2}(K + sigma2 I)P^{-1/2} and log det P (Sylvester, App. A.3) is added;
 * the probes must then be N(0, P) samples (fgk_precond_sample), else N(0, I).
 *   pc      NULL (no preconditioner) or built on h for this sigma2.
 *   B       device, N x nprobe FP64 row-major, original point order;
 *           1 <= nprobe <= 64.
 *   m       the most CG (Lanczos) steps per probe; tol the CG stop test
 *           (relative FP64 true residual, as fgk_cg_solve).  A column's
 *           Lanczos process ends at its first residual replacement.
 *   X       device N x nprobe or NULL: the solves (K + sigma2 I)^{-1} B (for
 *           the Hutchinson trace term of eq. gp_log_likelihood_derivative).
 *   quad    host nprobe or NULL: gamma_b e_1^T log(T_b) e_1 per probe.
 *   steps   host nprobe or NULL: Lanczos steps per probe.
 *   rep     host: the estimate and diagnostics.
 * The solve runs with FP64 scans.  Allocates a workspace of 16 m nprobe
 * bytes (the coefficient log), plus 8 N nprobe when X is NULL.  Synchronises
 * `stream`.  A probe whose solve stops at m steps is not an error (its
 * partial Lanczos process is used; rep->solve_status is FGK_NOT_CONVERGED).
 * Errors: FGK_ERR_INVALID (arguments, or pc built on another plan or for
 * another sigma2), FGK_ERR_OOM, FGK_ERR_NONFINITE (B), FGK_ERR_BREAKDOWN (a
 * Ritz value <= 0: the system is not positive definite), or any other error
 * of the CG solve. */
int fgk_slq_logdet(fgk_handle h, fgk_precond pc, double sigma2, const double *B, int nprobe, int m, double tol,
                   double *X, double *quad, int *steps, fgk_slq_report *rep, fgk_stream_t stream);

/* e_1^T log(T) e_1 for the Lanczos matrix T of m CG steps with coefficients
 * alpha[0..m) and beta[0..m-1) (Algorithm 2's formulas above): the Gauss
 * quadrature of log with T's eigenvalues as nodes and the squared first
 * components of its eigenvectors as weights.  Host arrays; no GPU work.
 * FGK_ERR_INVALID for m < 1, alpha <= 0 or beta < 0; FGK_ERR_BREAKDOWN if a
 * Ritz value is <= 0. */
int fgk_lanczos_logquad(const double *alpha, const double *beta, int m, double *out);

/* ---- the likelihood gradient (eq. gp_log_likelihood_derivative) ---- */

typedef struct {
    double yAy;            /* y^T (K + sigma2 I)^{-1} y (Algorithm 1's sigma update uses it) */
    double alpha_sq;       /* alpha^T alpha, alpha = (K + sigma2 I)^{-1} y */
    double max_true_resid; /* of the solve of [y, B] */
    int iterations;        /* CG iterations of that solve */
    int solve_status;      /* its return code (FGK_OK or FGK_NOT_CONVERGED) */
    int n_grad;            /* entries written to grad */
} fgk_grad_report;

/* The gradient of the log marginal likelihood log p(y | x, theta)
 * (eq. gp_log_likelihood_derivative) with respect to the log-parameters:
 *   d/dtheta = 1/2 a^T dK/dtheta a - 1/2 tr((K + sigma2 I)^{-1} dK/dtheta),
 *   a = (K + sigma2 I)^{-1} y, the trace by Hutchinson's estimator
 *   (App. A.2) mean_i ((K + sigma2 I)^{-1} b_i)^T dK/dtheta (P^{-1} b_i) over
 *   the probe columns b_i of B (N(0, P) draws with a preconditioner,
 *   fgk_precond_sample; N(0, I) without).
 *   grad   host: first the lengthscales, d/d log ell_k for k < d with the
 *          product kernel (d > 1), else one entry for all lengthscales
 *          scaled together (fgk_matvec_dlogell's dim = -1); then
 *          d/d log varsigma^2 (the outputscale of the plan) and
 *          d/d log sigma^2; rep->n_grad entries.
 *   y      device, N FP64, original point order; B device, N x nprobe FP64
 *          row-major, 0 <= nprobe <= 63.  nprobe = 0 solves y alone: rep
 *          holds y^T A^{-1} y and alpha^T alpha, grad only the terms in a
 *          (the quadratic halves, no trace).
 *   tol, maxit, mode  of the CG solve of [y, B] (as fgk_cg_solve).
 *   pc     NULL or built on h for this sigma2.
 * Allocates a workspace of about 8 N (4 nprobe + 3) bytes; synchronises
 * `stream`.  A solve that stops at maxit is not an error (rep->solve_status
 * is FGK_NOT_CONVERGED and the gradient uses its iterate).  Errors:
 * FGK_ERR_INVALID (arguments, or pc built on another plan or for another
 * sigma2), FGK_ERR_OOM, FGK_ERR_NONFINITE (y or B), FGK_ERR_BREAKDOWN, or any
 * other error of the solve, the preconditioner or the gradient products. */
int fgk_loglik_grad(fgk_handle h, fgk_precond pc, double sigma2, const double *y, const double *B, int nprobe,
                    double tol, int maxit, int mode, double *grad, fgk_grad_report *rep, fgk_stream_t stream);

/* ---- batches: many problems advanced together (d <= 2) ---- */

typedef struct fgk_batch_s *fgk_batch;

/* Group n built plans (all d <= 2) for products and solves with nrhs columns
 * per problem (1 <= nrhs <= 64).  The vectors of a batch are packed: problem
 * i occupies rows [off_i, off_i + N_i) (fgk_batch_layout), each row its nrhs
 * values, in that problem's internal order (as fgk_matvec_q).  One launch
 * per phase of the product covers every problem; rhs_per_cta (1..nrhs, or 0
 * for all) sets how many right-hand sides one CTA scans.  The plans must
 * outlive the batch.  Synchronises `stream`. */
int fgk_batch_create(const fgk_handle *handles, int n, int nrhs, int rhs_per_cta, fgk_stream_t stream,
                     fgk_batch *out);

/* row_offsets: host, n + 1 values: the first packed row of each problem and
 * the total row count. */
int fgk_batch_layout(fgk_batch b, int64_t *row_offsets);

/* Y = K_i V_i for every problem i at once, FP32 scans; Vq, Yq device,
 * packed (total rows x nrhs) FP32.  Asynchronous. */
int fgk_batch_matvec_q(fgk_batch b, const float *Vq, float *Yq, fgk_stream_t stream);

/* Solve (K_i + sigma2[i] I) alpha_i = y_i for every problem and column at
 * once: mixed-precision CG as fgk_cg_solve (FP32 scans, FP64 vectors, inner
 * products and residual replacements), no fixed effects.
 *   y, alpha   host arrays of n device pointers, each N_i x nrhs FP64,
 *              row-major, the problem's original point order.
 *   sigma2     host, n values >= 0.
 *   info       host array of n reports, or NULL.
 * Returns as fgk_cg_solve.  Synchronises `stream`. */
int fgk_batch_cg_solve(fgk_batch b, const double *const *y, const double *sigma2, double tol, int maxit,
                       double *const *alpha, fgk_cg_info *info, fgk_stream_t stream);

/* fgk_batch_cg_solve with one preconditioner per problem (pcs[i] built with
 * fgk_precond_build on problem i's plan for sigma2[i]): every iteration
 * applies each active problem's P^{-1} inside the captured graph; the mixed
 * refinement then replaces at a drop by FGK_MIXED_DELTA (default 1e-3) and
 * restarts every replaced column from p = P^{-1} r (as fgk_cg_solve_pc).
 * The preconditioners must outlive the call. */
int fgk_batch_cg_solve_pc(fgk_batch b, const fgk_precond *pcs, const double *const *y, const double *sigma2,
                          double tol, int maxit, double *const *alpha, fgk_cg_info *info, fgk_stream_t stream);

int fgk_batch_destroy(fgk_batch b);

/* Upper estimate, in bytes, of the device memory a handle for these sizes
 * holds after fgk_build plus the workspace of fgk_cg_solve with nrhs
 * columns (used for admission against a memory budget).  0 if invalid. */
size_t fgk_bytes_estimate(int64_t N, int d, int two_nu, int kind, int nrhs);

/* Release a handle and its device memory (stream-ordered on the stream of
 * its last call).  NULL is ignored. */
int fgk_destroy(fgk_handle h);

/* Message for the last failing call on this thread ("" if none). */
const char *fgk_last_error(void);

/* ---- instrumentation (tools) ---- */

/* Number of CUDA kernels the library has launched in this process (each
 * replay of a captured CG iteration counts its kernels). */
uint64_t fgk_kernel_launches(void);

/* CUDA-event timing of the main scan kernel (the output pass of the level
 * scans).  enable = 1 clears the totals and starts bracketing every launch
 * of that kernel made outside graph capture with events on its stream;
 * enable = 0 stops; enable = -1 only reads.  total_ms and launches (either
 * may be NULL) receive the accumulated elapsed time and launch count, after
 * waiting for the recorded events. */
int fgk_scan_timing(int enable, double *total_ms, int64_t *launches);

/* The same CUDA-event timing for any of these kernels (fgk_scan_timing is
 * kernel FGK_TIMED_SCAN_OUT): the output pass of the level scans, and the
 * two passes over L of the preconditioner apply (t = L^T R and
 * Z = R / sigma2 - L c).  FGK_ERR_INVALID for an unknown id. */
enum { FGK_TIMED_SCAN_OUT = 0, FGK_TIMED_PC_LTR = 1, FGK_TIMED_PC_APPLY = 2 };
int fgk_kernel_timing(int kernel, int enable, double *total_ms, int64_t *launches);

/* Measured fused multiply-add throughput of the current device, the
 * denominator of the ALU roofline of the FP64 scans and of the FP32 scans
 * with many moments (the paper has no counterpart; instrumentation).  A
 * kernel of independent FMA chains (16 per thread, 8 resident CTAs of 256
 * threads per SM) is launched once to warm up and `reps` times timed by CUDA
 * events on `stream`; *flops receives 2 x FMAs / second of the fastest
 * launch.  precision FGK_F32 or FGK_F64; reps >= 1.  Synchronises. */
int fgk_fma_rate(int precision, int reps, double *flops, fgk_stream_t stream);

/* ---- inspection (tests and tools): copies of the cached structure ---- */

typedef struct {
    int64_t N;
    int32_t d, two_nu, kind;
    int32_t L;          /* ceil(log2 N) */
    int32_t n_levels;   /* 1 (d=1), L (d=2), L(L+1)/2 (d=3) */
    double outscale2;
    double ell[3];
    size_t device_bytes; /* held by the handle now */
} fgk_plan_info;

int fgk_get_info(fgk_handle h, fgk_plan_info *out);

/* perm: host, N int32: the stable ascending order of the scaled coordinate
 * x'_dim = x_dim * sqrt(2 nu) / ell_dim (ties by original index). */
int fgk_get_permutation(fgk_handle h, int dim, int32_t *perm);

/* Copy level `level` of the structure to host arrays (any may be NULL):
 *   q     N uint32: point index in x'_1 order, per entry;
 *   roles N uint8: bit 0 = role in the first split dimension, bit 1 = role
 *         in the second (d = 3);
 *   dl64, dl32  N gaps of the sweep coordinate to the previous entry of the
 *         same segment (0 at a segment start);
 *   off64, off32  N x (d-1) row-major offsets |x' - split| per split dim;
 *   seg_size  the level's segment size (power of two).
 * Synchronous. */
int fgk_get_level(fgk_handle h, int level, uint32_t *q, uint8_t *roles, double *dl64, float *dl32,
                  double *off64, float *off32, int64_t *seg_size);

#ifdef __cplusplus
}
#endif

#endif /* FGK_H */
