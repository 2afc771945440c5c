// K5-K7: the GP solve (K + sigma^2 I) alpha = y (eq. gp_mean_system) on top of
// the product, with optional GLS fixed effects.
//
// CG (App. A.1, Algorithm 2 with a zero initial guess; the preconditioner is
// the identity unless one is given, see below) runs on a block of columns at once; every column has its own
// alpha_j = rho_j / p_j^T A p_j and beta_j = rho'_j / rho_j and stops on its
// own once ||r_j|| is below its threshold (then its updates are masked).
// Vectors, inner products and scalars are FP64 and stay on the device; the
// host only reads a small status word every few iterations.  One iteration
// (product, two reductions, three vector updates) is captured once into a
// CUDA graph and replayed.
//
// Refinement.  X accumulates in FP64.  In mixed mode CG applies A with FP32
// scans (FP32 moments; FP64 vectors, inner products and scalars), so its
// recursive residual drifts from b - A X; whenever a column's recursive
// residual has dropped by a factor delta since the last time (and whenever
// it claims convergence), the true residual b - A X is recomputed with FP64
// scans and replaces the recursive one, and CG continues from it with the
// same search direction (residual replacement, "reliable updates").  This is
// iterative refinement with the correction solved in low precision, without
// restarting the Krylov space at every correction.  In FP64 mode the only
// replacement is the final confirmation.
//
// Preconditioning (App. A.3; Algorithm 2 with s_P = P^{-1}): with a
// pivoted-Cholesky preconditioner every iteration also forms z = P^{-1} r
// (Woodbury, three kernels in the captured graph), rho = r^T z and
// p = z + beta p; the stop test and the replacement triggers stay on the
// recursive ||r||^2.  Mixed precision then takes the plain refinement form:
// the FP32 iterations run until the recursive residual has dropped by
// delta = 1e-3 (or claims convergence), the FP64 true residual replaces it,
// and every column restarts from p = z.  Keeping p across a replacement, as
// without a preconditioner, is unstable here: P^{-1} magnifies the gap
// between the recursive and the true residual outside the span of L by up
// to 1/sigma^2, so r^T z of the replaced residual no longer matches the kept
// direction and the next step overshoots (measured: the true residual grew
// by orders of magnitude); a good preconditioner needs few iterations per
// refinement step, so the restarts cost little.
//
// FP32 breakdowns.  The FP32 product of a direction that lies mostly in the
// small-eigenvalue subspace of a badly conditioned A can have p^T A p <= 0
// although A is positive definite.  A column that meets it stops (masked);
// the host recomputes p^T A p with FP64 scans: still <= 0 is a true
// breakdown (the solve ends with FGK_ERR_BREAKDOWN); otherwise the residual
// is replaced and the column restarts from p = r.  After kMaxRestarts such
// restarts in one solve the remaining iterations run with FP64 scans.  A column stops once its FP64 true
// residual meets the tolerance; the reported residuals are those.
//
// Fixed effects (Sec. 3.2, the GLS step of Algorithm 1): the block is
// [y, H]; with alpha_y = A^{-1} y and alpha_H = A^{-1} H,
// beta = (H^T alpha_H)^{-1} H^T alpha_y and alpha = alpha_y - alpha_H beta.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kRedBlocks = 304;  // 2 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kMaxCols = 64;

// CG state on the device.  The vector kernels of an iteration read rho and
// active; the p-update's first block writes the new values to rho_next and
// active_next, which the next iteration's first kernel copies over, so no
// block ever reads a value another block of the same kernel may be writing.
struct ColState {
    double rho[kMaxCols];  // r^T z (z = r without a preconditioner)
    double rr[kMaxCols];   // recursive ||r||^2 after the last p-update
    double rho_next[kMaxCols];
    double beta[kMaxCols];
    double thr2[kMaxCols];
    int active[kMaxCols];
    int active_next[kMaxCols];
    int iters[kMaxCols];
    int bd[kMaxCols];  // column met p^T A p <= 0 (set by k_update_xr, cleared by the host)
    int n_active;
    int breakdown;
    // Lanczos coefficients (Algorithm 2): alpha of the last x/r update; when
    // lz is set, k_update_p logs (alpha, beta) of every iteration of every
    // column not stopped by the host, lz[(it * ncols + j) * 2 + {0, 1}],
    // it < lz_cap, and lz_n[j] counts them
    double alpha[kMaxCols];
    double *lz;
    int lz_cap;
    int lz_n[kMaxCols];
    int lz_stop[kMaxCols];
};

constexpr int kMaxRestarts = 4;
constexpr int kReplacementGap = 24;  // FP32 iterations between residual replacements (see cg_solve)

// partial[b * ncols + j] = sum over this block's rows of a_ij * (b_ij + sb c_ij).
// Thread tid owns column tid % ncols and a row subset, so the row-major
// blocks are read with consecutive threads on consecutive elements.
template <class TA, class TB>
__device__ __forceinline__ void block_col_dots(const TA *__restrict__ a, const TB *__restrict__ b, double sb,
                                               const double *__restrict__ c, int64_t N, int ncols,
                                               double *__restrict__ partial) {
    __shared__ double red[kRedThreads];
    const int per = kRedThreads / ncols;
    const int j = threadIdx.x % ncols, lr = threadIdx.x / ncols;
    double acc = 0.0;
    if (lr < per) {
        for (int64_t i = (int64_t)blockIdx.x * per + lr; i < N; i += (int64_t)gridDim.x * per) {
            const int64_t t = i * ncols + j;
            double bb = (double)b[t];
            if (c) bb += sb * c[t];
            acc += (double)a[t] * bb;
        }
    }
    const double s = block_col_sum(acc, ncols, red);
    if (threadIdx.x < ncols) partial[blockIdx.x * ncols + threadIdx.x] = s;
}

__global__ void k_col_dots(const double *__restrict__ a, const double *__restrict__ b, int64_t N, int ncols,
                           double *__restrict__ partial) {
    block_col_dots<double, double>(a, b, 0.0, nullptr, N, ncols, partial);
}

// partial sums of p_j^T (w_j + sigma2 p_j)
__global__ void k_col_pap(const double *__restrict__ p, const double *__restrict__ w, double sigma2, int64_t N,
                          int ncols, double *__restrict__ partial) {
    block_col_dots<double, double>(p, w, sigma2, p, N, ncols, partial);
}

// p_j = r_j (or z_j) on the columns flagged in bd (a CG restart)
__global__ void k_restart_cols(double *__restrict__ p, const double *__restrict__ r, int64_t N, int ncols,
                               const ColState *__restrict__ st) {
    const int64_t n = N * ncols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        if (st->bd[t % ncols]) p[t] = r[t];
}

__global__ void k_finalize_sums(const double *__restrict__ partial, int nblk, int ncols, double *__restrict__ out) {
    const int j = threadIdx.x;
    if (j >= ncols) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b * ncols + j];
    out[j] = s;
}

// Deterministic sum of the nblk partials of column j by one warp: lanes take
// strided partials, then a shuffle tree.
__device__ __forceinline__ double warp_col_sum(const double *__restrict__ partial, int nblk, int ncols, int j,
                                               int lane) {
    double acc = 0.0;
    for (int b = lane; b < nblk; b += 32) acc += partial[b * ncols + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// pw_j = p_j^T (w_j + sigma2 p_j); the first block also moves the state the
// previous p-update left in rho_next / active_next into rho / active.
template <class W>
__global__ void k_dot_pAp(const double *__restrict__ p, const W *__restrict__ w, double sigma2, int64_t N, int ncols,
                          double *__restrict__ partial, ColState *__restrict__ st) {
    if (st->n_active == 0) return;
    if (blockIdx.x == 0 && threadIdx.x < ncols) {
        st->rho[threadIdx.x] = st->rho_next[threadIdx.x];
        st->active[threadIdx.x] = st->active_next[threadIdx.x];
    }
    block_col_dots<double, W>(p, w, sigma2, p, N, ncols, partial);
}

// alpha_j = rho_j / p_j^T A p_j (every block from the partials), then
// x += alpha p, r -= alpha (w + sigma2 p), and partial sums of r^2.
// p^T A p <= 0 on an active column flags a breakdown (the column is left
// untouched and stops; the host decides what follows).
template <class W>
__global__ void k_update_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const W *__restrict__ w, double sigma2, int64_t N, int ncols,
                            const double *__restrict__ pw_partial, int nblk, double *__restrict__ partial,
                            ColState *__restrict__ st) {
    if (st->n_active == 0) return;
    __shared__ double s_alpha[kMaxCols];
    __shared__ double red[kRedThreads];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < ncols; j += nw) {
        const double pw = warp_col_sum(pw_partial, nblk, ncols, j, lane);
        if (lane == 0) {
            double a = 0.0;
            if (st->active[j]) {
                if (pw > 0.0)
                    a = st->rho[j] / pw;
                else if (blockIdx.x == 0) {
                    atomicOr(&st->breakdown, 1);
                    st->bd[j] = 1;
                }
            }
            s_alpha[j] = a;
            if (blockIdx.x == 0) st->alpha[j] = a;
        }
    }
    __syncthreads();
    const int per = kRedThreads / ncols;
    const int jj = threadIdx.x % ncols, lr = threadIdx.x / ncols;
    double acc = 0.0;
    if (lr < per) {
        const double a = s_alpha[jj];
        for (int64_t i = (int64_t)blockIdx.x * per + lr; i < N; i += (int64_t)gridDim.x * per) {
            const int64_t t = i * ncols + jj;
            double rv = r[t];
            if (a != 0.0) {
                const double pv = p[t];
                x[t] += a * pv;
                rv -= a * ((double)w[t] + sigma2 * pv);
                r[t] = rv;
            }
            acc += rv * rv;
        }
    }
    const double t = block_col_sum(acc, ncols, red);
    if (threadIdx.x < ncols) partial[blockIdx.x * ncols + threadIdx.x] = t;
}

// beta_j = rho'_j / rho_j and the stop test (every block from the partials);
// p = r + beta p on the columns still active; then, on every column, the FP32
// copy of p for the mixed product and W = s2 p, the diagonal term the next
// product starts from.
// The first block records the new state for the next iteration.
// With a preconditioner r is z = P^{-1} r and beta and rho use the partial
// sums of r^T z (rz_partial); the stop test always uses ||r||^2.
template <class W>
__global__ void k_update_p(double *__restrict__ p, float *__restrict__ p32, W *__restrict__ w,
                           const double *__restrict__ r, double s2, int64_t N, int ncols,
                           const double *__restrict__ rr_partial, const double *__restrict__ rz_partial,
                           int rz_nblk, ColState *__restrict__ st) {
    const int nblk = gridDim.x;  // rows of rr_partial: one per CTA of k_update_xr (same grid)
    if (st->n_active == 0) return;
    __shared__ double s_beta[kMaxCols];
    __shared__ int s_act[kMaxCols];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < ncols; j += nw) {
        const double rr = warp_col_sum(rr_partial, nblk, ncols, j, lane);
        const double rz = rz_partial ? warp_col_sum(rz_partial, rz_nblk, ncols, j, lane) : rr;
        if (lane == 0) {
            const int act = st->active[j];
            const double rho = st->rho[j];
            const int still = act && !st->bd[j] && rr > st->thr2[j];
            s_beta[j] = act ? (rho > 0.0 ? rz / rho : 0.0) : 0.0;
            s_act[j] = still;
            if (blockIdx.x == 0) {
                st->rho_next[j] = act ? rz : rho;
                if (act) st->rr[j] = rr;
                st->active_next[j] = still;
                st->beta[j] = s_beta[j];
                if (act && st->lz && !st->lz_stop[j] && st->lz_n[j] < st->lz_cap && !st->bd[j]) {
                    const int it = st->lz_n[j];
                    st->lz[((size_t)it * ncols + j) * 2] = st->alpha[j];
                    st->lz[((size_t)it * ncols + j) * 2 + 1] = s_beta[j];
                    st->lz_n[j] = it + 1;
                }
                if (act) st->iters[j] += 1;
            }
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int n = 0;
        for (int j = 0; j < ncols; ++j) n += s_act[j];
        st->n_active = n;
    }
    const int64_t n = N * ncols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % ncols);
        double pv = p[t];
        if (s_act[j]) {
            pv = r[t] + s_beta[j] * pv;
            p[t] = pv;
        }
        if (p32) {
            const float pf = (float)pv;
            p32[t] = pf;
            w[t] = (W)(s2 * (double)pf);
        } else {
            w[t] = (W)(s2 * pv);
        }
    }
}

// the FP32 copy of p and W = s2 p before the first product of a solve
template <class W>
__global__ void k_init_p(const double *__restrict__ p, float *__restrict__ p32, W *__restrict__ w, double s2,
                         int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double pv = p[t];
        if (p32) {
            const float pf = (float)pv;
            p32[t] = pf;
            w[t] = (W)(s2 * (double)pf);
        } else {
            w[t] = (W)(s2 * pv);
        }
    }
}

// R = B - (Y + sigma2 X) with Y = K X
__global__ void k_residual(const double *__restrict__ B, const double *__restrict__ Y, const double *__restrict__ X,
                           double sigma2, int64_t n, double *__restrict__ R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        R[t] = B[t] - (Y[t] + sigma2 * X[t]);
}

// B (q order, N x ncols) = [y | H]; H == NULL with L > 0 means [1, x].
__global__ void k_assemble_rhs(const double *__restrict__ y, int nrhs, const double *__restrict__ H, int L,
                               const double *__restrict__ xraw_q, int d, const int32_t *__restrict__ perm1, int64_t N,
                               double *__restrict__ B, int *__restrict__ bad) {
    const int ncols = nrhs + L;
    const int64_t n = N * ncols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / ncols;
        const int j = (int)(t - q * ncols);
        const int64_t i = perm1[q];
        double v;
        if (j < nrhs) v = y[i * nrhs + j];
        else if (H) v = H[i * L + (j - nrhs)];
        else v = (j == nrhs) ? 1.0 : xraw_q[q * d + (j - nrhs - 1)];
        if (!isfinite(v)) atomicOr(bad, 1);
        B[t] = v;
    }
}

// GLS: C = H^T [alpha_y | alpha_H] (L x ncols) -> beta (L x nrhs) by Cholesky
// of G = H^T alpha_H (symmetric positive definite in exact arithmetic);
// single thread, L <= 8.
__global__ void k_gls_beta(const double *__restrict__ C, int L, int nrhs, double *__restrict__ beta,
                           int *__restrict__ bad) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int ncols = nrhs + L;
    double G[kMaxH][kMaxH];
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b) G[a][b] = 0.5 * (C[a * ncols + nrhs + b] + C[b * ncols + nrhs + a]);
    // Cholesky G = U^T U (upper), in place
    for (int k = 0; k < L; ++k) {
        double s = G[k][k];
        for (int m = 0; m < k; ++m) s -= G[m][k] * G[m][k];
        if (!(s > 0.0)) {
            *bad = 1;
            return;
        }
        G[k][k] = sqrt(s);
        for (int c = k + 1; c < L; ++c) {
            double t = G[k][c];
            for (int m = 0; m < k; ++m) t -= G[m][k] * G[m][c];
            G[k][c] = t / G[k][k];
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        double z[kMaxH];
        for (int k = 0; k < L; ++k) {  // U^T z = g
            double t = C[k * ncols + r];
            for (int m = 0; m < k; ++m) t -= G[m][k] * z[m];
            z[k] = t / G[k][k];
        }
        for (int k = L - 1; k >= 0; --k) {  // U b = z
            double t = z[k];
            for (int m = k + 1; m < L; ++m) t -= G[k][m] * beta[m * nrhs + r];
            beta[k * nrhs + r] = t / G[k][k];
        }
    }
}

// C[l * ncols + j] partials: sum_q H_ql X_qj, H taken from B's columns
__global__ void k_hT_x(const double *__restrict__ B, const double *__restrict__ X, int64_t N, int nrhs, int L,
                       double *__restrict__ partial) {
    const int ncols = nrhs + L;
    __shared__ double red[kRedThreads];
    for (int l = 0; l < L; ++l)
        for (int j = 0; j < ncols; ++j) {
            double acc = 0.0;
            for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N;
                 q += (int64_t)gridDim.x * blockDim.x)
                acc += B[q * ncols + nrhs + l] * X[q * ncols + j];
            red[threadIdx.x] = acc;
            __syncthreads();
            for (int s = kRedThreads / 2; s > 0; s >>= 1) {
                if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
                __syncthreads();
            }
            if (threadIdx.x == 0) partial[blockIdx.x * (L * ncols) + l * ncols + j] = red[0];
            __syncthreads();
        }
}

// alpha (caller order) = X_y - X_H beta, read through rank1
__global__ void k_output_alpha(const double *__restrict__ X, int ncols, int nrhs, int L,
                               const double *__restrict__ beta, const int32_t *__restrict__ rank1, int64_t N,
                               double *__restrict__ alpha) {
    const int64_t n = N * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nrhs;
        const int r = (int)(t - i * nrhs);
        const int64_t q = rank1[i];
        double v = X[q * ncols + r];
        for (int l = 0; l < L; ++l) v -= X[q * ncols + nrhs + l] * beta[l * nrhs + r];
        alpha[t] = v;
    }
}

double env_double(const char *name, double dflt) {
    const char *s = getenv(name);
    if (!s || !*s) return dflt;
    char *end = nullptr;
    double v = strtod(s, &end);
    return (end && end != s) ? v : dflt;
}

}  // namespace

size_t solve_ws_bytes(const Plan *p, int ncols) {
    const size_t vec = (size_t)p->N * ncols * 8;
    return 7 * vec + (size_t)kRedBlocks * kMaxCols * kMaxH * 8 + sizeof(ColState) + 4096;
}

int cg_solve(Plan *p, Precond *pc, const double *y, int nrhs, double sigma2, const double *H, int L, double tol,
             int maxit, int mode, double *alpha, double *beta, fgk_cg_info *info, cudaStream_t user_s,
             LanczosLog *lzlog) {
    const int64_t N = p->N;
    const int ncols = nrhs + std::max(L, 0);
    if (ncols > kMaxCols) {
        set_error("fgk_cg_solve: nrhs + L = %d exceeds %d", ncols, kMaxCols);
        return FGK_ERR_INVALID;
    }
    // a private stream: the legacy default stream cannot be captured into a graph
    cudaStream_t s;
    FGK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t ev;
    FGK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FGK_CUDA(cudaEventRecord(ev, user_s));
    FGK_CUDA(cudaStreamWaitEvent(s, ev, 0));
    cudaStream_t saved = p->stream;
    p->stream = s;

    const size_t vec = (size_t)N * ncols;
    bool mixed = mode == FGK_MIXED;
    const int rz_blocks = pc ? pc_partial_blocks(pc) : kRedBlocks;
    size_t bytes = (pc ? 6 : 5) * vec * 8 + (mixed ? 2 * vec * 4 : 0) +
                   (size_t)kRedBlocks * kMaxCols * (kMaxH + 1) * 8 + (size_t)rz_blocks * ncols * 8 +
                   sizeof(ColState) + 8192;
    if (pc && pc_reserve(pc, ncols, s) != FGK_OK) {
        p->stream = saved;
        cudaStreamDestroy(s);
        cudaEventDestroy(ev);
        return FGK_ERR_OOM;
    }
    char *w = (char *)dev_alloc(bytes, s);
    if (!w) {
        p->stream = saved;
        set_error("fgk_cg_solve: workspace allocation of %zu bytes failed", bytes);
        cudaStreamDestroy(s);
        cudaEventDestroy(ev);
        return FGK_ERR_OOM;
    }
    auto carve = [&](size_t nbytes) {
        char *r = w;
        w += (nbytes + 255) / 256 * 256;
        return (void *)r;
    };
    double *B = (double *)carve(vec * 8);
    double *X = (double *)carve(vec * 8);
    double *Rv = (double *)carve(vec * 8);
    double *Pv = (double *)carve(vec * 8);
    double *W64 = (double *)carve(vec * 8);
    float *W32 = mixed ? (float *)carve(vec * 4) : nullptr;
    float *P32 = mixed ? (float *)carve(vec * 4) : nullptr;
    double *partial = (double *)carve((size_t)kRedBlocks * kMaxCols * kMaxH * 8);
    double *partial2 = (double *)carve((size_t)kRedBlocks * kMaxCols * 8);
    double *partial3 = (double *)carve((size_t)rz_blocks * ncols * 8);  // r^T z, one row per CTA of the apply
    double *Zv = pc ? (double *)carve(vec * 8) : nullptr;
    ColState *st = (ColState *)carve(sizeof(ColState));

    int rc = FGK_OK;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t graph_nodes = 0;
    std::vector<double> bnorm(ncols), rnorm(ncols), rho_ref(ncols);
    std::vector<int> confirmed(ncols, 0);
    std::vector<int> snap_lz_n(ncols, 0);  // Lanczos coefficients logged per column (last device snapshot)
    int iters_total = 0, refinements = 0, n_f32 = 0, n_f64 = 0;
    bool converged = false, breakdown = false;
    // mixed mode: replace the recursive residual by the FP64 true residual
    // once it has dropped by this factor since the last replacement
    double delta = mixed ? env_double("FGK_MIXED_DELTA", pc ? 1e-3 : 0.5) : 0.0;
    int restarts = 0;
    std::vector<double> pap(ncols);
    const int check_every = 8;
    int hbad = 0;
    double *dsum = partial + (size_t)kRedBlocks * kMaxCols * kMaxH - 2 * kMaxCols * kMaxH;  // tail scratch

    auto colnorms = [&](const double *A, std::vector<double> &out) -> int {
        k_col_dots<<<kRedBlocks, kRedThreads, 0, s>>>(A, A, N, ncols, partial);
        FGK_LAUNCH_CHECK();
        k_finalize_sums<<<1, kMaxCols, 0, s>>>(partial, kRedBlocks, ncols, dsum);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(out.data(), dsum, ncols * 8, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        for (auto &v : out) v = std::sqrt(v);
        return FGK_OK;
    };
    // per-column A^T B into out (no square root)
    auto coldots = [&](const double *A, const double *Bm, std::vector<double> &out) -> int {
        k_col_dots<<<kRedBlocks, kRedThreads, 0, s>>>(A, Bm, N, ncols, partial);
        FGK_LAUNCH_CHECK();
        k_finalize_sums<<<1, kMaxCols, 0, s>>>(partial, kRedBlocks, ncols, dsum);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(out.data(), dsum, ncols * 8, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        return FGK_OK;
    };
    // z = P^{-1} r and rz = r^T z per column (host), preconditioned solves only
    std::vector<double> hrz(ncols);
    auto precondition = [&]() -> int {
        FGK_TRY(pc_apply(pc, Rv, ncols, Zv, nullptr, s));
        FGK_TRY(pc_check(pc, s));
        return coldots(Rv, Zv, hrz);
    };
    // R = B - A X with FP64 scans (replaces the recursive residual)
    auto true_residual = [&]() -> int {
        FGK_TRY(mvm_q_f64(p, X, ncols, W64, s, nullptr));
        k_residual<<<kRedBlocks, kRedThreads, 0, s>>>(B, W64, X, sigma2, (int64_t)vec, Rv);
        FGK_LAUNCH_CHECK();
        ++refinements;
        ++n_f64;
        return colnorms(Rv, rnorm);
    };
    // one CG iteration; every kernel returns at once when no column is active.
    // The product starts from W = s2 p, written by the previous p-update.
    auto one_iteration = [&]() -> int {
        if (mixed) {
            FGK_TRY(mvm_q_f32(p, P32, ncols, W32, s, &st->n_active, false));
            k_dot_pAp<float><<<kRedBlocks, kRedThreads, 0, s>>>(Pv, W32, sigma2, N, ncols, partial, st);
            FGK_LAUNCH_CHECK();
            k_update_xr<float><<<kRedBlocks, kRedThreads, 0, s>>>(X, Rv, Pv, W32, sigma2, N, ncols, partial,
                                                                 kRedBlocks, partial2, st);
            FGK_LAUNCH_CHECK();
            if (pc) FGK_TRY(pc_apply(pc, Rv, ncols, Zv, partial3, s));
            k_update_p<float><<<kRedBlocks, kRedThreads, 0, s>>>(Pv, P32, W32, pc ? Zv : Rv, p->s2, N, ncols,
                                                                partial2, pc ? partial3 : nullptr, rz_blocks, st);
            FGK_LAUNCH_CHECK();
        } else {
            FGK_TRY(mvm_q_f64(p, Pv, ncols, W64, s, &st->n_active, false));
            k_dot_pAp<double><<<kRedBlocks, kRedThreads, 0, s>>>(Pv, W64, sigma2, N, ncols, partial, st);
            FGK_LAUNCH_CHECK();
            k_update_xr<double><<<kRedBlocks, kRedThreads, 0, s>>>(X, Rv, Pv, W64, sigma2, N, ncols, partial,
                                                                  kRedBlocks, partial2, st);
            FGK_LAUNCH_CHECK();
            if (pc) FGK_TRY(pc_apply(pc, Rv, ncols, Zv, partial3, s));
            k_update_p<double><<<kRedBlocks, kRedThreads, 0, s>>>(Pv, nullptr, W64, pc ? Zv : Rv, p->s2, N, ncols,
                                                                 partial2, pc ? partial3 : nullptr, rz_blocks, st);
            FGK_LAUNCH_CHECK();
        }
        return FGK_OK;
    };
    // p^T A p per column with FP64 scans (overwrites W64)
    auto pap64 = [&]() -> int {
        FGK_TRY(mvm_q_f64(p, Pv, ncols, W64, s, nullptr));
        ++n_f64;
        k_col_pap<<<kRedBlocks, kRedThreads, 0, s>>>(Pv, W64, sigma2, N, ncols, partial);
        FGK_LAUNCH_CHECK();
        k_finalize_sums<<<1, kMaxCols, 0, s>>>(partial, kRedBlocks, ncols, dsum);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(pap.data(), dsum, ncols * 8, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        return FGK_OK;
    };
    auto capture = [&]() -> int {
        const uint64_t c0 = kernel_launch_count();
        FGK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int crc = one_iteration();
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        graph_nodes = kernel_launch_count() - c0;
        add_kernel_launches(-(int64_t)graph_nodes);  // counted when replayed
        if (crc) return crc;
        FGK_CUDA(ce);
        FGK_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
        return FGK_OK;
    };
    auto init_p = [&]() -> int {
        if (mixed)
            k_init_p<float><<<kRedBlocks, kRedThreads, 0, s>>>(Pv, P32, W32, p->s2, (int64_t)vec);
        else
            k_init_p<double><<<kRedBlocks, kRedThreads, 0, s>>>(Pv, nullptr, W64, p->s2, (int64_t)vec);
        FGK_LAUNCH_CHECK();
        return FGK_OK;
    };

    do {
        FGK_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
        k_assemble_rhs<<<kRedBlocks, kRedThreads, 0, s>>>(y, nrhs, H, std::max(L, 0), p->xraw_q, p->d, p->perm[0], N,
                                                          B, p->dev_err);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(&hbad, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        if (hbad) {
            FGK_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
            set_error("fgk_cg_solve: y or H holds a NaN or an infinity");
            rc = FGK_ERR_NONFINITE;
            break;
        }
        if ((rc = colnorms(B, bnorm))) break;
        FGK_CUDA(cudaMemsetAsync(X, 0, vec * 8, s));
        FGK_CUDA(cudaMemcpyAsync(Rv, B, vec * 8, cudaMemcpyDeviceToDevice, s));
        rnorm = bnorm;
        if (pc) {  // p = z = P^{-1} b, rho = b^T z
            if ((rc = precondition())) break;
            FGK_CUDA(cudaMemcpyAsync(Pv, Zv, vec * 8, cudaMemcpyDeviceToDevice, s));
        } else {
            FGK_CUDA(cudaMemcpyAsync(Pv, B, vec * 8, cudaMemcpyDeviceToDevice, s));
        }
        // the products' workspace at its largest (the FP64 products of the residual
        // replacements run between graph launches and must not move the buffer the
        // captured FP32 products use); no product is run for it
        if ((rc = ensure_ws(p, std::max(mvm_ws_bytes(p, ncols, true), mvm_ws_bytes(p, ncols, false)), s))) break;
        // A residual replacement (one FP64 product) is allowed once the FP32
        // iterations since the last one have cost about as much, so that
        // replacements take at most about half of the solve: kReplacementGap
        // iterations, the FP64/FP32 scan cost ratio measured on GB300 (19x on
        // the d = 2 workload, 31x on the d = 3 one).  A fixed count keeps the
        // solve's path, and so its result, the same on every run, whatever
        // else shares the GPU.  The spacing only applies while the recursion
        // tracks the true residual: when a replacement finds a true residual
        // more than twice the recursive one, the FP32 iterations since the
        // last one were drifting and the next replacement is not held back.
        const int min_gap = mixed ? kReplacementGap : 0;
        int gap = 0;  // until the first replacement has shown how well the recursion tracks
        int last_replacement = 0;
        if ((rc = init_p())) break;
        ColState hs;
        std::memset(&hs, 0, sizeof(hs));
        for (int j = 0; j < ncols; ++j) {
            hs.rr[j] = rnorm[j] * rnorm[j];
            hs.rho[j] = hs.rho_next[j] = pc ? hrz[j] : hs.rr[j];
            rho_ref[j] = hs.rr[j];
            const double target = 0.5 * tol * bnorm[j];
            hs.thr2[j] = target * target;
            confirmed[j] = rnorm[j] <= tol * bnorm[j];
            hs.active[j] = hs.active_next[j] = !confirmed[j];
            hs.n_active += hs.active[j];
        }
        if (lzlog) {  // Lanczos coefficients: the start vector's norm^2 in the P^{-1} metric (rho_0)
            hs.lz = lzlog->dev_log;
            hs.lz_cap = lzlog->cap;
            for (int j = 0; j < ncols; ++j) lzlog->gamma[j] = hs.rho[j];
        }
        FGK_CUDA(cudaMemcpyAsync(st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
        if ((rc = capture())) break;
        ColState snap = hs;
        while (true) {
            bool all = true;
            for (int j = 0; j < ncols; ++j) all = all && confirmed[j];
            if (all) {
                converged = true;
                break;
            }
            if (iters_total >= maxit) break;
            const int k = std::min(check_every, maxit - iters_total);
            const int before = *std::max_element(snap.iters, snap.iters + ncols);
            for (int it = 0; it < k; ++it) FGK_CUDA(cudaGraphLaunch(gexec, s));
            add_kernel_launches((int64_t)graph_nodes * k);
            FGK_CUDA(cudaMemcpyAsync(&snap, st, sizeof(ColState), cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaStreamSynchronize(s));
            for (int j = 0; j < ncols; ++j) snap_lz_n[j] = snap.lz_n[j];
            const int after = *std::max_element(snap.iters, snap.iters + ncols);
            iters_total += after - before;
            if (mixed) n_f32 += after - before; else n_f64 += after - before;
            bool restart = false;
            if (snap.breakdown) {
                // FP64 mode: a true breakdown.  Mixed: decide with FP64 scans.
                if (!mixed) {
                    breakdown = true;
                    break;
                }
                if ((rc = pap64())) break;
                for (int j = 0; j < ncols; ++j)
                    if (snap.bd[j] && !(pap[j] > 0.0)) breakdown = true;
                if (breakdown) break;
                restart = true;
            }
            // replace the recursive residual when a column claims convergence
            // or (mixed) has reduced its residual by delta since the last time
            bool claims = false, dropped = false;
            for (int j = 0; j < ncols; ++j) {
                if (confirmed[j]) continue;
                if (!snap.active_next[j]) claims = true;
                if (snap.rr[j] <= delta * delta * rho_ref[j]) dropped = true;
            }
            if (!(restart || claims || (dropped && iters_total - last_replacement >= gap))) continue;
            last_replacement = iters_total;
            if ((rc = true_residual())) break;
            if (pc && (rc = precondition())) break;
            // Columns restart from p = z (z = r without a preconditioner) when
            // their search direction no longer fits the replaced residual: an
            // FP32 breakdown, a column that had stopped (its p missed the last
            // update), or a true residual more than twice the recursive one
            // (the recursion drifted; keeping p would pair a direction scaled
            // to the recursive residual with rho of the true one).
            bool drift = false, any_rs = false;
            for (int j = 0; j < ncols; ++j) {
                const bool dj = !confirmed[j] && rnorm[j] > 2.0 * std::sqrt(snap.rr[j]);
                drift = drift || dj;
                const bool rs = !confirmed[j] && (pc || snap.bd[j] || !snap.active_next[j] || dj) &&
                                !(rnorm[j] <= tol * bnorm[j]);
                snap.bd[j] = rs ? 1 : 0;
                any_rs = any_rs || rs;
            }
            gap = drift ? 0 : min_gap;
            if (any_rs) {
                FGK_CUDA(cudaMemcpyAsync(st, &snap, sizeof(ColState), cudaMemcpyHostToDevice, s));
                k_restart_cols<<<kRedBlocks, kRedThreads, 0, s>>>(Pv, pc ? Zv : Rv, N, ncols, st);
                FGK_LAUNCH_CHECK();
            }
            std::memset(snap.bd, 0, sizeof(snap.bd));
            snap.breakdown = 0;
            if (restart) {
                if (++restarts > kMaxRestarts && mixed) {
                    // the FP32 products cannot resolve this system: FP64 from here on
                    mixed = false;
                    delta = 0.0;
                    cudaGraphExecDestroy(gexec);
                    cudaGraphDestroy(graph);
                    gexec = nullptr;
                    graph = nullptr;
                    if ((rc = capture())) break;
                }
            }
            if ((rc = init_p())) break;  // the residual product overwrote W64 (FP64 mode)
            snap.n_active = 0;
            for (int j = 0; j < ncols; ++j) {
                snap.lz_stop[j] = 1;  // a replaced residual ends the column's Lanczos process
                if (!confirmed[j] && rnorm[j] <= tol * bnorm[j]) confirmed[j] = 1;
                snap.active[j] = snap.active_next[j] = !confirmed[j];
                if (!confirmed[j]) {
                    snap.rr[j] = rnorm[j] * rnorm[j];
                    snap.rho[j] = snap.rho_next[j] = pc ? hrz[j] : snap.rr[j];
                    rho_ref[j] = snap.rr[j];
                }
                snap.n_active += snap.active[j];
            }
            FGK_CUDA(cudaMemcpyAsync(st, &snap, sizeof(ColState), cudaMemcpyHostToDevice, s));
        }
        if (rc) break;
        if (pc && (rc = pc_check(pc, s))) break;  // a bulk-copy wait of the preconditioner expired
        if (!converged && refinements == 0 && (rc = true_residual())) break;  // report true residuals
        // GLS fixed effects
        double *beta_dev = nullptr;
        if (L > 0) {
            beta_dev = partial;  // L x nrhs at the head of the scratch
            double *part2 = partial + kMaxH * kMaxCols;
            const int nb = 64;
            k_hT_x<<<nb, kRedThreads, 0, s>>>(B, X, N, nrhs, L, part2);
            FGK_LAUNCH_CHECK();
            double *Cm = dsum;
            k_finalize_sums<<<1, kMaxCols * kMaxH, 0, s>>>(part2, nb, L * ncols, Cm);
            FGK_LAUNCH_CHECK();
            FGK_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
            k_gls_beta<<<1, 32, 0, s>>>(Cm, L, nrhs, beta_dev, p->dev_err);
            FGK_LAUNCH_CHECK();
            FGK_CUDA(cudaMemcpyAsync(&hbad, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaStreamSynchronize(s));
            if (hbad) {
                FGK_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
                set_error("fgk_cg_solve: H^T A^{-1} H is not positive definite (collinear fixed effects?)");
                rc = FGK_ERR_INVALID;
                break;
            }
            if (beta) FGK_CUDA(cudaMemcpyAsync(beta, beta_dev, (size_t)L * nrhs * 8, cudaMemcpyDeviceToDevice, s));
        }
        k_output_alpha<<<kRedBlocks, kRedThreads, 0, s>>>(X, ncols, nrhs, std::max(L, 0), beta_dev, p->rank1, N,
                                                           alpha);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaStreamSynchronize(s));
    } while (0);

    if (lzlog)
        for (int j = 0; j < ncols; ++j) lzlog->n[j] = snap_lz_n[j];
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    dev_free((void *)B, s);
    cudaStreamSynchronize(s);
    p->stream = saved;
    cudaEventDestroy(ev);
    cudaStreamDestroy(s);
    if (info) {
        info->iterations = iters_total;
        info->refinements = refinements;
        info->mvm_f32 = n_f32;
        info->mvm_f64 = n_f64;
        info->restarts = restarts;
        info->fp64_switch = (mode == FGK_MIXED && !mixed) ? 1 : 0;
        double mx = 0.0;
        for (int j = 0; j < ncols; ++j) {
            double r = bnorm[j] > 0 ? rnorm[j] / bnorm[j] : 0.0;
            mx = std::max(mx, r);
            if (info->true_resid) info->true_resid[j] = r;
        }
        info->max_true_resid = mx;
    }
    if (rc) return rc;
    if (breakdown) {
        set_error("fgk_cg_solve: p^T A p <= 0 met; the system is not positive definite");
        return FGK_ERR_BREAKDOWN;
    }
    if (!converged) {
        set_error("fgk_cg_solve: tolerance not reached within maxit = %d iterations", maxit);
        return FGK_NOT_CONVERGED;
    }
    return FGK_OK;
}

}  // namespace fgk
