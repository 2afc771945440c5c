/*
 * Oracle for the exact fast Matérn kernel matrix-vector product.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The product path
 * (libfgk) never links, calls or includes anything from here, and nothing
 * here is shared with the CUDA sources.
 *
 * Everything is FP64 and deliberately plain:
 *
 *  orc_kernel      closed-form half-integer Matérn kernels, eqs. matern_1_2,
 *                  matern_3_2, matern_5_2, matern_7_2, matern_9_2 (App. C.1),
 *                  unit lengthscale.  The definition-based entries below
 *                  (O1, K, columns, cross-covariance, gradient products)
 *                  take nu = 1/2 .. 9/2; the decompositions (O2 and its
 *                  relatives) are printed for nu <= 5/2 and take only those.
 *  orc_mvm_brute   O1: the definition of the product, eqs. covariance_matrix
 *                  and Ky (Sec. 2), with the L1 kernel (eq. L1_kernel) or the
 *                  product kernel (eq. product_kernel), scaled as in
 *                  eq. scaled_kernel.  O(N^2), Neumaier-compensated sums,
 *                  OpenMP over output rows.
 *  orc_kmat        the dense matrix K itself (small N), same definition.
 *  orc_kcols       selected columns K[:, idx] (the pivoted Cholesky of the
 *                  preconditioner needs one column per step), same definition.
 *  orc_kcross      the cross-covariance [K(z_j, x_i)] between evaluation
 *                  points Z and the data X (the vector k_z of eq. gp_mean),
 *                  same definition.
 *  orc_kernel_dlog  the lengthscale derivatives of the closed forms
 *                  (App. C.1, the gradient formulas beside each Matérn
 *                  decomposition): l d/dl k(|x|/l) = -u k'(u) and -k'(u).
 *  orc_mvm_dlogell_brute  Y = (dK/d log l_m) V from the definition: the
 *                  gradient product of the trace term of
 *                  eq. gp_log_likelihood_derivative, per lengthscale or for
 *                  all lengthscales scaled together.
 *  orc_mvm_dc_cross  the kernel sums at new points (k_z of eq. gp_mean)
 *                  by the same decomposition, sources and queries apart.
 *  orc_mvm_dc_dlogell_l1  the L1 kernel's lengthscale gradient by the
 *                  paper's printed ECDF decompositions, on O2's machinery.
 *  orc_mvm_dc_dlogell_product  the product kernel's lengthscale gradient
 *                  through Proposition 2 with one factor differentiated.
 *  orc_mvm_dc      O2: the paper's own algorithm, written in its order and
 *                  notation: weighted ECDFs with the generalised inequality
 *                  (eq. ECDFdelta), one per orthant delta and weight vector,
 *                  evaluated by a Bentley divide and conquer that re-sorts at
 *                  every node (Sec. 2.2.3; no cached structure), then
 *                  recombined with the printed Matérn formulas
 *                  (eqs. matern_12_decomposition, matern_32_decomposition,
 *                  matern_52_decomposition) for the L1 kernel, and with
 *                  Proposition 2 (eq. product_decomposition) and the
 *                  one-dimensional factor pairs of eqs. k12_decomposition_phi,
 *                  k32_decomposition_phi, k52_decomposition_phi for the
 *                  product kernel.
 *
 * Lengthscales: the paper uses one scalar lengthscale (eq. scaled_kernel).
 * A per-dimension lengthscale ell_k is read as the same kernel applied to the
 * coordinates u_k = x_k / ell_k, after which the formulas run with ell = 1.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared (no -ffast-math: IEEE semantics).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_L1 0
#define ORC_PRODUCT 1

/* ---------------------------------------------------------------------- */
/* Closed-form kernels (App. C.1, eqs. matern_1_2 .. matern_9_2)           */
/* ---------------------------------------------------------------------- */

double orc_kernel(int two_nu, double u)
{
    u = fabs(u);
    switch (two_nu) {
    case 1:
        return exp(-u);
    case 3: {
        double s = sqrt(3.0) * u;
        return (1.0 + s) * exp(-s);
    }
    case 5: {
        double s = sqrt(5.0) * u;
        return (1.0 + s + (5.0 / 3.0) * u * u) * exp(-s);
    }
    case 7: { /* eq. matern_7_2 */
        double s = sqrt(7.0) * u;
        return (1.0 + s + (14.0 / 5.0) * u * u + (7.0 * sqrt(7.0) / 15.0) * u * u * u) * exp(-s);
    }
    case 9: { /* eq. matern_9_2 */
        double u2 = u * u;
        return (1.0 + 3.0 * u + (27.0 / 7.0) * u2 + (18.0 / 7.0) * u2 * u + (27.0 / 35.0) * u2 * u2) * exp(-3.0 * u);
    }
    default:
        return NAN;
    }
}

/* K(x_a - x_b) for the L1 or the product multivariate kernel, unit
 * outputscale, coordinates already divided by the lengthscales. */
static double kern_pair(const double *ua, const double *ub, int d, int two_nu, int kind)
{
    if (kind == ORC_L1) {
        double r = 0.0;
        for (int k = 0; k < d; ++k) r += fabs(ua[k] - ub[k]);
        return orc_kernel(two_nu, r);
    }
    double p = 1.0;
    for (int k = 0; k < d; ++k) p *= orc_kernel(two_nu, fabs(ua[k] - ub[k]));
    return p;
}

/* The definition (O1 and the dense forms) takes nu = 1/2 .. 9/2; the
 * paper's decompositions (O2) are printed for nu <= 5/2 only, and those
 * entry points check that separately (check_dc). */
static int check_args(long N, int d, int two_nu, const double *ell, int kind)
{
    if (N < 0 || d < 1 || d > 3) return -1;
    if (two_nu != 1 && two_nu != 3 && two_nu != 5 && two_nu != 7 && two_nu != 9) return -1;
    if (kind != ORC_L1 && kind != ORC_PRODUCT) return -1;
    for (int k = 0; k < d; ++k)
        if (!(ell[k] > 0.0) || !isfinite(ell[k])) return -1;
    return 0;
}

static int check_dc(long N, int d, int two_nu, const double *ell, int kind)
{
    if (two_nu != 1 && two_nu != 3 && two_nu != 5) return -1;
    return check_args(N, d, two_nu, ell, kind);
}

static double *scaled_coords(const double *X, long N, int d, const double *ell)
{
    double *U = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * (size_t)d);
    for (long i = 0; i < N; ++i)
        for (int k = 0; k < d; ++k) U[i * d + k] = X[i * d + k] / ell[k];
    return U;
}

/* ---------------------------------------------------------------------- */
/* O1: brute force (eqs. covariance_matrix, Ky)                             */
/* ---------------------------------------------------------------------- */

/* Y = s2 * K V.  X is N x d row-major, V is N x nrhs row-major.  If rows is
 * NULL every output row is computed and Y is N x nrhs; otherwise only the
 * listed rows are computed and Y is nrows x nrhs (row r of Y is output row
 * rows[r]).  Sums run over i = 0..N-1 in order with Neumaier compensation. */
int orc_mvm_brute(const double *X, long N, int d, int two_nu, const double *ell, double s2,
                  int kind, const double *V, int nrhs, const long *rows, long nrows, double *Y,
                  int nthreads)
{
    if (check_args(N, d, two_nu, ell, kind) || nrhs < 1) return -1;
    long nout = rows ? nrows : N;
    double *U = scaled_coords(X, N, d, ell);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int bad = 0;
#pragma omp parallel
    {
        double *sum = (double *)malloc(sizeof(double) * (size_t)nrhs);
        double *cmp = (double *)malloc(sizeof(double) * (size_t)nrhs);
#pragma omp for schedule(dynamic, 16)
        for (long r = 0; r < nout; ++r) {
            long j = rows ? rows[r] : r;
            if (j < 0 || j >= N) {
                bad = 1;
                continue;
            }
            for (int c = 0; c < nrhs; ++c) sum[c] = cmp[c] = 0.0;
            for (long i = 0; i < N; ++i) {
                double kij = kern_pair(U + j * d, U + i * d, d, two_nu, kind);
                for (int c = 0; c < nrhs; ++c) {
                    double term = kij * V[i * nrhs + c];
                    double t = sum[c] + term;
                    if (fabs(sum[c]) >= fabs(term))
                        cmp[c] += (sum[c] - t) + term;
                    else
                        cmp[c] += (term - t) + sum[c];
                    sum[c] = t;
                }
            }
            for (int c = 0; c < nrhs; ++c) Y[r * nrhs + c] = s2 * (sum[c] + cmp[c]);
        }
        free(sum);
        free(cmp);
    }
    free(U);
    return bad ? -1 : 0;
}

/* Dense K (N x N row-major) for small N: K_ij = s2 * K(x_i - x_j). */
int orc_kmat(const double *X, long N, int d, int two_nu, const double *ell, double s2, int kind,
             double *K)
{
    if (check_args(N, d, two_nu, ell, kind)) return -1;
    double *U = scaled_coords(X, N, d, ell);
    for (long i = 0; i < N; ++i)
        for (long j = 0; j < N; ++j) K[i * N + j] = s2 * kern_pair(U + i * d, U + j * d, d, two_nu, kind);
    free(U);
    return 0;
}

int orc_kcols(const double *X, long N, int d, int two_nu, const double *ell, double s2, int kind,
              const long *idx, long nidx, double *C)
{
    if (check_args(N, d, two_nu, ell, kind)) return -1;
    for (long c = 0; c < nidx; ++c)
        if (idx[c] < 0 || idx[c] >= N) return -1;
    double *U = scaled_coords(X, N, d, ell);
    for (long i = 0; i < N; ++i)
        for (long c = 0; c < nidx; ++c)
            C[i * nidx + c] = s2 * kern_pair(U + i * d, U + idx[c] * d, d, two_nu, kind);
    free(U);
    return 0;
}

int orc_kcross(const double *X, long N, const double *Zp, long M, int d, int two_nu, const double *ell, double s2,
               int kind, double *C)
{
    if (check_args(N, d, two_nu, ell, kind) || M < 1) return -1;
    double *U = scaled_coords(X, N, d, ell);
    double *V = scaled_coords(Zp, M, d, ell);
    for (long j = 0; j < M; ++j)
        for (long i = 0; i < N; ++i) C[j * N + i] = s2 * kern_pair(V + j * d, U + i * d, d, two_nu, kind);
    free(U);
    free(V);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Lengthscale derivatives (App. C.1 gradient formulas)                     */
/* ---------------------------------------------------------------------- */

/* which = 0: -u k'(u), the derivative of k(|x|/l) with respect to log l
 *            (u = |x| / l): nu=1/2: u e^{-u}; nu=3/2: 3 u^2 e^{-sqrt3 u};
 *            nu=5/2: (5/3)(u^2 + sqrt5 u^3) e^{-sqrt5 u}.
 * which = 1: -k'(u): e^{-u}; 3 u e^{-sqrt3 u}; (5/3)(u + sqrt5 u^2) e^{-sqrt5 u};
 *            nu=7/2, 9/2 from eqs. dmatern72_dl, dmatern92_dl. */
double orc_kernel_dlog(int two_nu, int which, double u)
{
    u = fabs(u);
    double m; /* -k'(u) */
    switch (two_nu) {
    case 1:
        m = exp(-u);
        break;
    case 3:
        m = 3.0 * u * exp(-sqrt(3.0) * u);
        break;
    case 5:
        m = (5.0 / 3.0) * (u + sqrt(5.0) * u * u) * exp(-sqrt(5.0) * u);
        break;
    case 7:
        m = ((7.0 / 5.0) * u + (7.0 * sqrt(7.0) / 5.0) * u * u + (49.0 / 15.0) * u * u * u) * exp(-sqrt(7.0) * u);
        break;
    case 9:
        m = ((9.0 / 7.0) * u + (27.0 / 7.0) * u * u + (162.0 / 35.0) * u * u * u + (81.0 / 35.0) * u * u * u * u) *
            exp(-3.0 * u);
        break;
    default:
        return NAN;
    }
    return which == 0 ? u * m : m;
}

/* dK(x_a - x_b)/d log l_dim (dim in [0, d)), or the sum over all dims
 * (dim = -1: every lengthscale scaled together), unit outputscale, scaled
 * coordinates.  L1: K = k(U), U = sum_k u_k, so the derivative is
 * u_dim (-k'(U)) and the sum over dims is U (-k'(U)).  Product:
 * prod_{k != dim} k(u_k) times (-u_dim k'(u_dim)). */
static double dkern_pair(const double *ua, const double *ub, int d, int two_nu, int kind, int dim)
{
    double u[3];
    double U = 0.0;
    for (int k = 0; k < d; ++k) {
        u[k] = fabs(ua[k] - ub[k]);
        U += u[k];
    }
    if (kind == ORC_L1) {
        double m = orc_kernel_dlog(two_nu, 1, U);
        return (dim < 0 ? U : u[dim]) * m;
    }
    double tot = 0.0;
    for (int mdim = 0; mdim < d; ++mdim) {
        if (dim >= 0 && mdim != dim) continue;
        double p = orc_kernel_dlog(two_nu, 0, u[mdim]);
        for (int k = 0; k < d; ++k)
            if (k != mdim) p *= orc_kernel(two_nu, u[k]);
        tot += p;
    }
    return tot;
}

/* Y = s2 (dK/d log l_dim) V (dim = -1: summed over the dims), same layout,
 * row selection and summation order as orc_mvm_brute. */
int orc_mvm_dlogell_brute(const double *X, long N, int d, int two_nu, const double *ell, double s2, int kind,
                          int dim, const double *V, int nrhs, const long *rows, long nrows, double *Y,
                          int nthreads)
{
    if (check_args(N, d, two_nu, ell, kind) || nrhs < 1 || dim < -1 || dim >= d) return -1;
    long nout = rows ? nrows : N;
    double *U = scaled_coords(X, N, d, ell);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int bad = 0;
#pragma omp parallel
    {
        double *sum = (double *)malloc(sizeof(double) * (size_t)nrhs);
        double *cmp = (double *)malloc(sizeof(double) * (size_t)nrhs);
#pragma omp for schedule(dynamic, 16)
        for (long r = 0; r < nout; ++r) {
            long j = rows ? rows[r] : r;
            if (j < 0 || j >= N) {
                bad = 1;
                continue;
            }
            for (int c = 0; c < nrhs; ++c) sum[c] = cmp[c] = 0.0;
            for (long i = 0; i < N; ++i) {
                double kij = dkern_pair(U + j * d, U + i * d, d, two_nu, kind, dim);
                for (int c = 0; c < nrhs; ++c) {
                    double term = kij * V[i * nrhs + c];
                    double t = sum[c] + term;
                    if (fabs(sum[c]) >= fabs(term))
                        cmp[c] += (sum[c] - t) + term;
                    else
                        cmp[c] += (term - t) + sum[c];
                    sum[c] = t;
                }
            }
            for (int c = 0; c < nrhs; ++c) Y[r * nrhs + c] = s2 * (sum[c] + cmp[c]);
        }
        free(sum);
        free(cmp);
    }
    free(U);
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* O2: the paper's decomposition, literally                                */
/* ---------------------------------------------------------------------- */

/* One point copy in an ECDF problem.  Every data point appears twice: once
 * as a source (it carries weights) and once as a query (it receives F).
 * key[k] encodes the generalised inequality of eq. ECDFdelta on dimension k
 * as a strict integer comparison, see make_keys(). */
typedef struct {
    long key[3];
    int src;
    long id;
} item_t;

static int g_sort_dim; /* qsort has no context argument */

static int cmp_item(const void *pa, const void *pb)
{
    const item_t *a = (const item_t *)pa, *b = (const item_t *)pb;
    long ka = a->key[g_sort_dim], kb = b->key[g_sort_dim];
    if (ka != kb) return ka < kb ? -1 : 1;
    if (a->src != b->src) return a->src > b->src ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

static void sort_items(item_t *it, long n, int k)
{
    g_sort_dim = k;
    qsort(it, (size_t)n, sizeof(item_t), cmp_item);
}

/* F[id*nw + m] += sum over sources s with key_t(s) < key_t(q) for every
 * dimension t = k..d-1 of W[s*nw + m], for every query q in it[0..n).
 * Bentley's divide and conquer: split on dimension k at the median (after a
 * fresh sort), recurse into both halves on dimension k, and hand the pairs
 * (source in the low half, query in the high half) -- for which dimension k
 * holds by construction -- to the problem on dimensions k+1..d-1.  The last
 * dimension is a sort followed by a running sum (fast sum updating, Sec. 2.1). */
static void ecdf_dc(item_t *it, long n, int k, int d, const double *W, int nw, double *F)
{
    if (n < 2) return;
    sort_items(it, n, k);
    if (k == d - 1) {
        double *acc = (double *)calloc((size_t)nw, sizeof(double));
        for (long a = 0; a < n; ++a) {
            if (it[a].src)
                for (int m = 0; m < nw; ++m) acc[m] += W[it[a].id * nw + m];
            else
                for (int m = 0; m < nw; ++m) F[it[a].id * nw + m] += acc[m];
        }
        free(acc);
        return;
    }
    long mid = n / 2;
    /* cross problem first, while the halves are still the sorted halves */
    item_t *cross = (item_t *)malloc(sizeof(item_t) * (size_t)n);
    long nc = 0;
    for (long a = 0; a < mid; ++a)
        if (it[a].src) cross[nc++] = it[a];
    for (long a = mid; a < n; ++a)
        if (!it[a].src) cross[nc++] = it[a];
    ecdf_dc(cross, nc, k + 1, d, W, nw, F);
    free(cross);
    ecdf_dc(it, mid, k, d, W, nw, F);
    ecdf_dc(it + mid, n - mid, k, d, W, nw, F);
}

typedef struct {
    double v;
    long i;
} vi_t;

static int cmp_vi(const void *pa, const void *pb)
{
    const vi_t *a = (const vi_t *)pa, *b = (const vi_t *)pb;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return a->i < b->i ? -1 : (a->i > b->i);
}

/* Integer keys for orthant delta.  On dimension k the coordinate compared is
 * delta_k * u_k.  Its dense rank r (equal values share a rank) turns
 * "x <= z" (delta_k = +1) into  2 r_src < 2 r_query + 1  and "x < z"
 * (delta_k = -1) into  2 r_src + 1 < 2 r_query, so that every comparison
 * between a source and a query is strict and no two of them tie. */
static void make_keys(const double *U, long N, int d, const int *delta, item_t *it)
{
    vi_t *tmp = (vi_t *)malloc(sizeof(vi_t) * (size_t)N);
    long *rank = (long *)malloc(sizeof(long) * (size_t)N);
    for (int k = 0; k < d; ++k) {
        for (long i = 0; i < N; ++i) {
            tmp[i].v = delta[k] * U[i * d + k];
            tmp[i].i = i;
        }
        qsort(tmp, (size_t)N, sizeof(vi_t), cmp_vi);
        long r = -1;
        for (long a = 0; a < N; ++a) {
            if (a == 0 || tmp[a].v != tmp[a - 1].v) ++r;
            rank[tmp[a].i] = r;
        }
        for (long i = 0; i < N; ++i) {
            long rs = delta[k] > 0 ? 2 * rank[i] : 2 * rank[i] + 1;
            long rq = delta[k] > 0 ? 2 * rank[i] + 1 : 2 * rank[i];
            it[2 * i].key[k] = rs;     /* source copy */
            it[2 * i + 1].key[k] = rq; /* query copy */
        }
    }
    for (long i = 0; i < N; ++i) {
        it[2 * i].src = 1;
        it[2 * i].id = i;
        it[2 * i + 1].src = 0;
        it[2 * i + 1].id = i;
    }
    free(tmp);
    free(rank);
}

/* Keys for sources at the data U (N points) and queries at new points Z
 * (M points): the dense ranks are taken over the union, with the same
 * strict source/query offsets as make_keys.  Items 0..N-1 are the sources
 * (id = data index), N..N+M-1 the queries (id = new-point index). */
static void make_keys_cross(const double *U, long N, const double *Zs, long M, int d, const int *delta, item_t *it)
{
    long T = N + M;
    vi_t *tmp = (vi_t *)malloc(sizeof(vi_t) * (size_t)T);
    long *rank = (long *)malloc(sizeof(long) * (size_t)T);
    for (int k = 0; k < d; ++k) {
        for (long i = 0; i < T; ++i) {
            tmp[i].v = delta[k] * (i < N ? U[i * d + k] : Zs[(i - N) * d + k]);
            tmp[i].i = i;
        }
        qsort(tmp, (size_t)T, sizeof(vi_t), cmp_vi);
        long r = -1;
        for (long a = 0; a < T; ++a) {
            if (a == 0 || tmp[a].v != tmp[a - 1].v) ++r;
            rank[tmp[a].i] = r;
        }
        for (long i = 0; i < T; ++i) {
            long rs = delta[k] > 0 ? 2 * rank[i] : 2 * rank[i] + 1;
            long rq = delta[k] > 0 ? 2 * rank[i] + 1 : 2 * rank[i];
            it[i].key[k] = i < N ? rs : rq;
        }
    }
    for (long i = 0; i < T; ++i) {
        it[i].src = i < N;
        it[i].id = i < N ? i : i - N;
    }
    free(tmp);
    free(rank);
}

/* One-dimensional factor pairs phi_{1,p}, phi_{2,p} with k(u - v) equal to
 * sum_p phi_{1,p}(u) phi_{2,p}(v) (Assumption 1), unit lengthscale:
 * eq. k12_decomposition_phi (P=1), eq. k32_decomposition_phi (P=2),
 * eq. k52_decomposition_phi (P=3; phi_{2,3}(v) = v^2 e^{sqrt5 v}, the form
 * printed beside the table, the expansion above it having a stray factor v).
 * p is 0-based here. */
static double phi1(int two_nu, int p, double u)
{
    if (two_nu == 1) return exp(-u);
    if (two_nu == 3) {
        double s3 = sqrt(3.0);
        return p == 0 ? (1.0 + s3 * u) * exp(-s3 * u) : -s3 * exp(-s3 * u);
    }
    double s5 = sqrt(5.0);
    if (p == 0) return (1.0 + s5 * u + (5.0 / 3.0) * u * u) * exp(-s5 * u);
    if (p == 1) return -(s5 + (10.0 / 3.0) * u) * exp(-s5 * u);
    return (5.0 / 3.0) * exp(-s5 * u);
}

static double phi2(int two_nu, int p, double v)
{
    if (two_nu == 1) return exp(v);
    double a = two_nu == 3 ? sqrt(3.0) : sqrt(5.0);
    if (p == 0) return exp(a * v);
    if (p == 1) return v * exp(a * v);
    return v * v * exp(a * v);
}

int orc_phi(int two_nu, int which, int p, double x, double *out)
{
    if (two_nu != 1 && two_nu != 3 && two_nu != 5) return -1;
    int P = (two_nu + 1) / 2;
    if (p < 0 || p >= P) return -1;
    *out = which == 1 ? phi1(two_nu, p, x) : phi2(two_nu, p, x);
    return 0;
}

/* Y = s2 * K V by the decomposition.  For the L1 kernel (Proposition 1 and
 * the Matérn examples of Sec. 2.3) the weight vectors are
 * w^{(p)}_i = v_i (delta.x_i)^p exp(a delta.x_i), p < P (eq. matern_weights
 * with ell = 1, a = sqrt(2 nu)), and the result is recombined by
 * eq. matern_12_decomposition / matern_32_decomposition /
 * matern_52_decomposition.  For the product kernel (Proposition 2,
 * eq. product_decomposition) the weight vectors are
 * w_{theta,i} = v_i prod_k phi_{2,theta_k}(delta_k x_{k,i}) and the result is
 * sum_theta prod_k phi_{1,theta_k}(delta_k z_k) F_theta. */
int orc_mvm_dc(const double *X, long N, int d, int two_nu, const double *ell, double s2, int kind,
               const double *V, int nrhs, double *Y)
{
    if (check_dc(N, d, two_nu, ell, kind) || nrhs < 1) return -1;
    int P = (two_nu + 1) / 2;
    double a = sqrt((double)two_nu);
    int nw = 1;
    if (kind == ORC_L1)
        nw = P;
    else
        for (int k = 0; k < d; ++k) nw *= P;
    double *U = scaled_coords(X, N, d, ell);
    item_t *it = (item_t *)malloc(sizeof(item_t) * (size_t)(2 * N + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nw);
    double *F = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nw);
    memset(Y, 0, sizeof(double) * (size_t)N * (size_t)nrhs);

    int ndelta = 1 << d;
    for (int c = 0; c < nrhs; ++c) {
        for (int mask = 0; mask < ndelta; ++mask) {
            int delta[3];
            for (int k = 0; k < d; ++k) delta[k] = (mask >> k) & 1 ? -1 : 1;
            /* weights of the sources */
            for (long i = 0; i < N; ++i) {
                double vi = V[i * nrhs + c];
                if (kind == ORC_L1) {
                    double dx = 0.0;
                    for (int k = 0; k < d; ++k) dx += delta[k] * U[i * d + k];
                    for (int p = 0; p < P; ++p) W[i * nw + p] = vi * pow(dx, p) * exp(a * dx);
                } else {
                    for (int t = 0; t < nw; ++t) {
                        double w = vi;
                        int rem = t;
                        for (int k = 0; k < d; ++k) {
                            int th = rem % P;
                            rem /= P;
                            w *= phi2(two_nu, th, delta[k] * U[i * d + k]);
                        }
                        W[i * nw + t] = w;
                    }
                }
            }
            memset(F, 0, sizeof(double) * (size_t)N * (size_t)nw);
            make_keys(U, N, d, delta, it);
            ecdf_dc(it, 2 * N, 0, d, W, nw, F);
            /* recombination */
            for (long j = 0; j < N; ++j) {
                double acc;
                if (kind == ORC_L1) {
                    double z = 0.0;
                    for (int k = 0; k < d; ++k) z += delta[k] * U[j * d + k];
                    const double *Fj = F + j * nw;
                    if (two_nu == 1) {
                        /* eq. matern_12_decomposition */
                        acc = exp(-z) * Fj[0];
                    } else if (two_nu == 3) {
                        /* eq. matern_32_decomposition */
                        acc = exp(-a * z) * ((1.0 + a * z) * Fj[0] - a * Fj[1]);
                    } else {
                        /* eq. matern_52_decomposition */
                        double c2 = 5.0 / 3.0;
                        acc = exp(-a * z) *
                              ((1.0 + a * z + c2 * z * z) * Fj[0] - (a + 2.0 * c2 * z) * Fj[1] + c2 * Fj[2]);
                    }
                } else {
                    acc = 0.0;
                    for (int t = 0; t < nw; ++t) {
                        double f = F[j * nw + t];
                        int rem = t;
                        for (int k = 0; k < d; ++k) {
                            int th = rem % P;
                            rem /= P;
                            f *= phi1(two_nu, th, delta[k] * U[j * d + k]);
                        }
                        acc += f;
                    }
                }
                Y[j * nrhs + c] += s2 * acc;
            }
        }
    }
    free(U);
    free(it);
    free(W);
    free(F);
    return 0;
}

/* The printed product Matérn-3/2 example (eqs. matern_product_weights_0,
 * matern_product_weights_1, matern_product_weights_vector,
 * matern_product_32_decomposition), with the typeset products read as
 * pi0(z) = prod_k (1 + a delta_k z_k)^{theta_k} and
 * pi1(x) = prod_k (-a delta_k x_k)^{1 - theta_k}, theta in {0,1}^d: the two
 * printed products are zero unless theta is all ones or all zeros, and this
 * reading is the binomial expansion of prod_k (1 + a delta_k (z_k - x_k)).
 * Kept beside orc_mvm_dc so the reading can be checked against
 * Proposition 2. */
/* The kernel sums at new points, Y_j = s2 sum_i K(z_j - x_i) V_i (the vector
 * k_z of eq. gp_mean times V; the kernel sum of eq. kde at any z), by the
 * same decomposition as orc_mvm_dc: sources at the data, queries at the new
 * points, one weighted ECDF per orthant and weight vector, recombined with
 * the printed Matérn formulas (L1) or Proposition 2 (product). */
int orc_mvm_dc_cross(const double *X, long N, const double *Zp, long M, int d, int two_nu, const double *ell,
                     double s2, int kind, const double *V, int nrhs, double *Y)
{
    if (check_dc(N, d, two_nu, ell, kind) || nrhs < 1 || M < 1) return -1;
    int P = (two_nu + 1) / 2;
    double a = sqrt((double)two_nu);
    int nw = 1;
    if (kind == ORC_L1)
        nw = P;
    else
        for (int k = 0; k < d; ++k) nw *= P;
    double *U = scaled_coords(X, N, d, ell);
    double *Zs = scaled_coords(Zp, M, d, ell);
    item_t *it = (item_t *)malloc(sizeof(item_t) * (size_t)(N + M + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nw);
    double *F = (double *)malloc(sizeof(double) * (size_t)(M + 1) * (size_t)nw);
    memset(Y, 0, sizeof(double) * (size_t)M * (size_t)nrhs);
    int ndelta = 1 << d;
    for (int c = 0; c < nrhs; ++c) {
        for (int mask = 0; mask < ndelta; ++mask) {
            int delta[3];
            for (int k = 0; k < d; ++k) delta[k] = (mask >> k) & 1 ? -1 : 1;
            for (long i = 0; i < N; ++i) {
                double vi = V[i * nrhs + c];
                if (kind == ORC_L1) {
                    double dx = 0.0;
                    for (int k = 0; k < d; ++k) dx += delta[k] * U[i * d + k];
                    for (int p = 0; p < P; ++p) W[i * nw + p] = vi * pow(dx, p) * exp(a * dx);
                } else {
                    for (int t = 0; t < nw; ++t) {
                        double w = vi;
                        int rem = t;
                        for (int k = 0; k < d; ++k) {
                            int th = rem % P;
                            rem /= P;
                            w *= phi2(two_nu, th, delta[k] * U[i * d + k]);
                        }
                        W[i * nw + t] = w;
                    }
                }
            }
            memset(F, 0, sizeof(double) * (size_t)M * (size_t)nw);
            make_keys_cross(U, N, Zs, M, d, delta, it);
            ecdf_dc(it, N + M, 0, d, W, nw, F);
            for (long j = 0; j < M; ++j) {
                double acc;
                const double *Fj = F + j * nw;
                if (kind == ORC_L1) {
                    double z = 0.0;
                    for (int k = 0; k < d; ++k) z += delta[k] * Zs[j * d + k];
                    if (two_nu == 1)
                        acc = exp(-z) * Fj[0];
                    else if (two_nu == 3)
                        acc = exp(-a * z) * ((1.0 + a * z) * Fj[0] - a * Fj[1]);
                    else {
                        double c2 = 5.0 / 3.0;
                        acc = exp(-a * z) *
                              ((1.0 + a * z + c2 * z * z) * Fj[0] - (a + 2.0 * c2 * z) * Fj[1] + c2 * Fj[2]);
                    }
                } else {
                    acc = 0.0;
                    for (int t = 0; t < nw; ++t) {
                        double f = Fj[t];
                        int rem = t;
                        for (int k = 0; k < d; ++k) {
                            int th = rem % P;
                            rem /= P;
                            f *= phi1(two_nu, th, delta[k] * Zs[j * d + k]);
                        }
                        acc += f;
                    }
                }
                Y[j * nrhs + c] += s2 * acc;
            }
        }
    }
    free(U);
    free(Zs);
    free(it);
    free(W);
    free(F);
    return 0;
}

/* The L1 kernel's lengthscale gradient by the paper's printed decompositions
 * (App. C.1: the gradient formulas after eqs. matern_12_decomposition,
 * matern_32_decomposition, matern_52_decomposition), evaluated with the same
 * weighted ECDFs F(delta z, delta; delta x, w^(p)) as orc_mvm_dc, one weight
 * order more (p <= P).  Returned as the derivative with respect to log ell
 * (ell times the printed d/d ell; every lengthscale scaled together when they
 * differ per dimension).  In scaled coordinates (z = delta . u_z):
 *   nu = 1/2:  e^{-z} (z F0 - F1)
 *   nu = 3/2:  3 e^{-a z} (z^2 F0 - 2 z F1 + F2)
 *   nu = 5/2:  5/3 e^{-a z} ((a z^3 + z^2) F0 - (2 z + 3 a z^2) F1 + (3 a z + 1) F2 - a F3) */
int orc_mvm_dc_dlogell_l1(const double *X, long N, int d, int two_nu, const double *ell, double s2,
                          const double *V, int nrhs, double *Y)
{
    if (check_dc(N, d, two_nu, ell, ORC_L1) || nrhs < 1) return -1;
    int P = (two_nu + 1) / 2;
    int nw = P + 1;
    double a = sqrt((double)two_nu);
    double *U = scaled_coords(X, N, d, ell);
    item_t *it = (item_t *)malloc(sizeof(item_t) * (size_t)(2 * N + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nw);
    double *F = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nw);
    memset(Y, 0, sizeof(double) * (size_t)N * (size_t)nrhs);
    int ndelta = 1 << d;
    for (int c = 0; c < nrhs; ++c) {
        for (int mask = 0; mask < ndelta; ++mask) {
            int delta[3];
            for (int k = 0; k < d; ++k) delta[k] = (mask >> k) & 1 ? -1 : 1;
            for (long i = 0; i < N; ++i) {
                double dx = 0.0;
                for (int k = 0; k < d; ++k) dx += delta[k] * U[i * d + k];
                for (int q = 0; q < nw; ++q) W[i * nw + q] = V[i * nrhs + c] * pow(dx, q) * exp(a * dx);
            }
            memset(F, 0, sizeof(double) * (size_t)N * (size_t)nw);
            make_keys(U, N, d, delta, it);
            ecdf_dc(it, 2 * N, 0, d, W, nw, F);
            for (long j = 0; j < N; ++j) {
                double z = 0.0;
                for (int k = 0; k < d; ++k) z += delta[k] * U[j * d + k];
                const double *Fj = F + j * nw;
                double acc;
                if (two_nu == 1)
                    acc = exp(-z) * (z * Fj[0] - Fj[1]);
                else if (two_nu == 3)
                    acc = 3.0 * exp(-a * z) * (z * z * Fj[0] - 2.0 * z * Fj[1] + Fj[2]);
                else
                    acc = (5.0 / 3.0) * exp(-a * z) *
                          ((a * z * z * z + z * z) * Fj[0] - (2.0 * z + 3.0 * a * z * z) * Fj[1] +
                           (3.0 * a * z + 1.0) * Fj[2] - a * Fj[3]);
                Y[j * nrhs + c] += s2 * acc;
            }
        }
    }
    free(U);
    free(it);
    free(W);
    free(F);
    return 0;
}

/* Coefficients f_q of a one-dimensional factor f(u) = sum_q f_q u^q e^{-a u}
 * (u = |x| / ell, a = sqrt(2 nu)): which = 0 the kernel k (App. C.1), which = 1
 * its log-lengthscale derivative -u k'(u). */
static int factor_coefs(int two_nu, int which, double *f)
{
    double a = sqrt((double)two_nu);
    for (int q = 0; q < 4; ++q) f[q] = 0.0;
    if (which == 0) {
        f[0] = 1.0;
        if (two_nu >= 3) f[1] = a;
        if (two_nu == 5) f[2] = 5.0 / 3.0;
        return (two_nu + 1) / 2;
    }
    if (two_nu == 1) f[1] = 1.0;
    if (two_nu == 3) f[2] = 3.0;
    if (two_nu == 5) {
        f[2] = 5.0 / 3.0;
        f[3] = 5.0 * a / 3.0;
    }
    return (two_nu + 3) / 2;
}

static double binom_d(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* The product kernel's lengthscale gradient through Proposition 2: in an
 * orthant delta every one-dimensional factor f(dz - dx) (dz = delta_k z_k,
 * dx = delta_k x_k, dz >= dx) splits by the binomial theorem as
 *   f(dz - dx) = sum_j chi1_j(dz) chi2_j(dx),
 *   chi1_j(dz) = e^{-a dz} sum_{q >= j} f_q C(q, j) dz^{q-j} (-1)^j,
 *   chi2_j(dx) = dx^j e^{a dx},
 * so the sum over sources of prod_k f_k is a sum over index patterns of
 * weighted ECDFs with weights prod_k chi2 (eq. ECDFdelta), recombined with
 * prod_k chi1 — eq. product_decomposition with the factor of dimension dim
 * replaced by -u k'(u) (dim = -1: summed over the dimensions). */
int orc_mvm_dc_dlogell_product(const double *X, long N, int d, int two_nu, const double *ell, double s2, int dim,
                               const double *V, int nrhs, double *Y)
{
    if (check_dc(N, d, two_nu, ell, ORC_PRODUCT) || nrhs < 1 || dim < -1 || dim >= d) return -1;
    double a = sqrt((double)two_nu);
    double *U = scaled_coords(X, N, d, ell);
    item_t *it = (item_t *)malloc(sizeof(item_t) * (size_t)(2 * N + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(N + 1) * 64);
    double *F = (double *)malloc(sizeof(double) * (size_t)(N + 1) * 64);
    memset(Y, 0, sizeof(double) * (size_t)N * (size_t)nrhs);
    int ndelta = 1 << d;
    for (int m = 0; m < d; ++m) {
        if (dim >= 0 && m != dim) continue;
        double f[3][4];
        int nj[3], nw = 1;
        for (int k = 0; k < d; ++k) {
            nj[k] = factor_coefs(two_nu, k == m ? 1 : 0, f[k]);
            nw *= nj[k];
        }
        for (int c = 0; c < nrhs; ++c) {
            for (int mask = 0; mask < ndelta; ++mask) {
                int delta[3];
                for (int k = 0; k < d; ++k) delta[k] = (mask >> k) & 1 ? -1 : 1;
                for (long i = 0; i < N; ++i)
                    for (int t = 0; t < nw; ++t) {
                        double w = V[i * nrhs + c];
                        int rem = t;
                        for (int k = 0; k < d; ++k) {
                            int j = rem % nj[k];
                            rem /= nj[k];
                            double dx = delta[k] * U[i * d + k];
                            w *= pow(dx, j) * exp(a * dx);
                        }
                        W[i * nw + t] = w;
                    }
                memset(F, 0, sizeof(double) * (size_t)N * (size_t)nw);
                make_keys(U, N, d, delta, it);
                ecdf_dc(it, 2 * N, 0, d, W, nw, F);
                for (long q = 0; q < N; ++q) {
                    double acc = 0.0;
                    for (int t = 0; t < nw; ++t) {
                        double g = F[q * nw + t];
                        int rem = t;
                        for (int k = 0; k < d; ++k) {
                            int j = rem % nj[k];
                            rem /= nj[k];
                            double dz = delta[k] * U[q * d + k];
                            double chi = 0.0;
                            for (int qq = j; qq < nj[k]; ++qq) chi += f[k][qq] * binom_d(qq, j) * pow(dz, qq - j);
                            g *= (j % 2 ? -1.0 : 1.0) * chi * exp(-a * dz);
                        }
                        acc += g;
                    }
                    Y[q * nrhs + c] += s2 * acc;
                }
            }
        }
    }
    free(U);
    free(it);
    free(W);
    free(F);
    return 0;
}

int orc_mvm_dc_product32_printed(const double *X, long N, int d, const double *ell, double s2,
                                 const double *V, double *Y)
{
    if (check_args(N, d, 3, ell, ORC_PRODUCT)) return -1;
    double a = sqrt(3.0);
    int nth = 1 << d;
    double *U = scaled_coords(X, N, d, ell);
    item_t *it = (item_t *)malloc(sizeof(item_t) * (size_t)(2 * N + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nth);
    double *F = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)nth);
    memset(Y, 0, sizeof(double) * (size_t)N);
    for (int mask = 0; mask < (1 << d); ++mask) {
        int delta[3];
        for (int k = 0; k < d; ++k) delta[k] = (mask >> k) & 1 ? -1 : 1;
        for (long i = 0; i < N; ++i) {
            double dx = 0.0;
            for (int k = 0; k < d; ++k) dx += delta[k] * U[i * d + k];
            for (int t = 0; t < nth; ++t) {
                double pi1 = 1.0;
                for (int k = 0; k < d; ++k)
                    if (!((t >> k) & 1)) pi1 *= -a * delta[k] * U[i * d + k];
                W[i * nth + t] = V[i] * pi1 * exp(a * dx);
            }
        }
        memset(F, 0, sizeof(double) * (size_t)N * (size_t)nth);
        make_keys(U, N, d, delta, it);
        ecdf_dc(it, 2 * N, 0, d, W, nth, F);
        for (long j = 0; j < N; ++j) {
            double z = 0.0;
            for (int k = 0; k < d; ++k) z += delta[k] * U[j * d + k];
            double acc = 0.0;
            for (int t = 0; t < nth; ++t) {
                double pi0 = 1.0;
                for (int k = 0; k < d; ++k)
                    if ((t >> k) & 1) pi0 *= 1.0 + a * delta[k] * U[j * d + k];
                acc += pi0 * exp(-a * z) * F[j * nth + t];
            }
            Y[j] += s2 * acc;
        }
    }
    free(U);
    free(it);
    free(W);
    free(F);
    return 0;
}

/* Number of OpenMP threads a parallel region gets (for reporting). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
