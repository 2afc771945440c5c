// MINRES (Paige and Saunders) for (K + sigma2 I) alpha = y when the system is
// symmetric but not positive definite: the L1 kernel at nu >= 3/2 and d >= 2
// (App. B, Prop. 4 fails there; CG then meets p^T A p <= 0).
//
// Per column j, the Lanczos process started at b_j builds the tridiagonal T_k
// (alpha_k on the diagonal, beta_{k+1} below it); Givens rotations reduce T_k
// to upper-triangular form as it grows, and x_k, the minimiser of
// ||b - A x|| over the Krylov space K_k(A, b), is updated through the
// direction vectors of the triangular factor:
//   p = A v_k - alpha_k v_k - beta_k v_{k-1},  alpha_k = v_k^T A v_k,
//   beta_{k+1} = ||p||,  v_{k+1} = p / beta_{k+1};
//   the previous rotation (c, s) applied to (delta_k, alpha_k) and (0, beta_{k+1})
//   gives delta_k', gamma_k and the entries eps_{k+1}, delta_{k+1} of the
//   next column; a new rotation zeroes beta_{k+1} (gamma_k' = |(gamma_k,
//   beta_{k+1})|), tau_k = c phi_{k-1}, phi_k = s phi_{k-1} = ||r_k||;
//   d_k = (v_k - delta_k' d_{k-1} - eps_k d_{k-2}) / gamma_k',  x += tau_k d_k.
// The vectors and products stay on the device (FP64 scans, the plan's
// internal point order); the scalars of the rotations are host arithmetic,
// one synchronisation per iteration (alpha_k and beta_{k+1} of every column
// come back together).  A column stops when phi_k <= tol ||b||; its true
// residual b - A x is then recomputed with FP64 scans and, if it is above the
// tolerance (rounding in the recurrence), the process restarts on the
// residual from the current x.
#include <cmath>
#include <vector>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kMrThreads = 256;
constexpr int kMrBlocks = 304;
constexpr int kMrMaxCols = 64;

// partial[b * nc + j] = sum over this block's rows of a_ij (c_ij + sb a_ij)
__global__ void k_mr_dots(const double *a, const double *c, double sb, int64_t N, int nc,
                          double *__restrict__ partial) {
    __shared__ double red[kMrThreads];
    const int per = kMrThreads / nc, jj = threadIdx.x % nc, lr = threadIdx.x / nc;
    double acc = 0.0;
    if (lr < per)
        for (int64_t i = (int64_t)blockIdx.x * per + lr; i < N; i += (int64_t)gridDim.x * per) {
            const int64_t t = i * nc + jj;
            acc += a[t] * (c[t] + sb * a[t]);
        }
    const double t = block_col_sum(acc, nc, red);
    if (threadIdx.x < nc) partial[blockIdx.x * nc + threadIdx.x] = t;
}

// out[j] = sum over blocks of partial[b * nc + j], in a fixed order (one warp per column)
__global__ void k_mr_finalize(const double *__restrict__ partial, int nblk, int nc, double *__restrict__ out) {
    const int lane = threadIdx.x & 31, j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= nc) return;
    double acc = 0.0;
    for (int b = lane; b < nblk; b += 32) acc += partial[b * nc + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[j] = acc;
}

// Lanczos step on the active columns: W <- W + sigma2 V - alpha V - beta Vp
// (W held K V) and partial sums of ||W||^2 per column
__global__ void k_mr_lanczos(double *__restrict__ W, const double *__restrict__ V, const double *__restrict__ Vp,
                             double sigma2, const double *__restrict__ alpha, const double *__restrict__ coef,
                             int64_t N, int nc, double *__restrict__ partial) {
    __shared__ double red[kMrThreads];
    const int per = kMrThreads / nc, jj = threadIdx.x % nc, lr = threadIdx.x / nc;
    double acc = 0.0;
    if (lr < per) {
        const double a = alpha[jj], b = coef[jj * 8 + 0], act = coef[jj * 8 + 7];
        for (int64_t i = (int64_t)blockIdx.x * per + lr; i < N; i += (int64_t)gridDim.x * per) {
            const int64_t t = i * nc + jj;
            double w = W[t] + sigma2 * V[t] - a * V[t] - b * Vp[t];
            if (act == 0.0) w = 0.0;
            W[t] = w;
            acc += w * w;
        }
    }
    const double t = block_col_sum(acc, nc, red);
    if (threadIdx.x < nc) partial[blockIdx.x * nc + threadIdx.x] = t;
}

// d = (v - delta2 d_prev - eps d_pp) / gamma2 into Dpp (the oldest direction),
// x += tau d, v_next = p / beta_next into Vp (the oldest Lanczos vector);
// inactive columns are left as they are.  coef per column:
// [beta, delta2, eps, gamma2, tau, beta_next, -, active]
__global__ void k_mr_update(double *__restrict__ X, const double *__restrict__ V, double *__restrict__ Vp,
                            const double *__restrict__ P, const double *__restrict__ Dp, double *__restrict__ Dpp,
                            const double *__restrict__ coef, int64_t n, int nc) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % nc);
        const double *c = coef + j * 8;
        if (c[7] == 0.0) continue;
        const double d = (V[t] - c[1] * Dp[t] - c[2] * Dpp[t]) / c[3];
        Dpp[t] = d;
        X[t] += c[4] * d;
        Vp[t] = c[5] > 0.0 ? P[t] / c[5] : 0.0;
    }
}

// restart of the listed columns from R: V = R / ||R||, Vp = Dp = Dpp = 0
__global__ void k_mr_restart(const double *__restrict__ R, double *__restrict__ V, double *__restrict__ Vp,
                             double *__restrict__ Dp, double *__restrict__ Dpp, const double *__restrict__ coef,
                             int64_t n, int nc) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % nc);
        const double *c = coef + j * 8;
        if (c[7] == 0.0) continue;  // column not restarted
        V[t] = R[t] / c[0];
        Vp[t] = 0.0;
        Dp[t] = 0.0;
        Dpp[t] = 0.0;
    }
}

// R = B - (W + sigma2 X), W = K X
__global__ void k_mr_residual(const double *__restrict__ B, const double *__restrict__ W,
                              const double *__restrict__ X, double sigma2, int64_t n, double *__restrict__ R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        R[t] = B[t] - (W[t] + sigma2 * X[t]);
}

struct ColRot {  // the host side of one column's recurrence
    double beta1 = 0, beta = 0, delta1 = 0, eps = 0, c = -1, s = 0, phi = 0;
    bool active = false;
};

int minres(Plan *p, const double *y, int nrhs, double sigma2, double tol, int maxit, double *alpha,
           fgk_cg_info *info, cudaStream_t s) {
    const int64_t N = p->N;
    const int nc = nrhs;
    const int64_t vec = N * nc;
    const size_t vb = (size_t)vec * sizeof(double);
    const size_t small = (size_t)kMrBlocks * nc + 16 * nc;
    const size_t vslot = (vb + 255) / 256 * 256;
    char *mem = (char *)dev_alloc(8 * vslot + small * sizeof(double) + 256, s);
    if (!mem) {
        set_error("fgk_minres_solve: device allocation of %zu bytes failed", 8 * vb);
        return FGK_ERR_OOM;
    }
    auto slot = [&](int i) { return (double *)(mem + (size_t)i * vslot); };
    double *B = slot(0), *X = slot(1), *V = slot(2), *Vp = slot(3), *W = slot(4), *Dp = slot(5), *Dpp = slot(6),
           *R = slot(7);
    double *partial = slot(8), *alpha_d = partial + (size_t)kMrBlocks * nc, *beta_d = alpha_d + nc,
           *coef_d = beta_d + nc;
    std::vector<double> hab(2 * nc), coef(8 * nc), bnorm(nc), rnorm(nc);
    std::vector<ColRot> col(nc);
    int rc = FGK_OK, iters = 0, restarts = 0, n_f64 = 0;
    const unsigned vgrid = grid_for(vec, 256) < 2048 ? grid_for(vec, 256) : 2048;

    auto colnorms = [&](const double *A, std::vector<double> &out) -> int {
        k_mr_dots<<<kMrBlocks, kMrThreads, 0, s>>>(A, A, 0.0, N, nc, partial);
        FGK_LAUNCH_CHECK();
        k_mr_finalize<<<(nc + 7) / 8, 256, 0, s>>>(partial, kMrBlocks, nc, alpha_d);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(out.data(), alpha_d, nc * sizeof(double), cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        for (auto &v : out) v = std::sqrt(v);
        return FGK_OK;
    };
    // R = B - A X with FP64 scans, and its column norms
    auto residual = [&]() -> int {
        FGK_TRY(mvm_q_f64(p, X, nc, W, s, nullptr));
        ++n_f64;
        k_mr_residual<<<vgrid, 256, 0, s>>>(B, W, X, sigma2, vec, R);
        FGK_LAUNCH_CHECK();
        return colnorms(R, rnorm);
    };
    // (re)start the columns listed active in col from R
    auto start = [&]() -> int {
        for (int j = 0; j < nc; ++j) {
            ColRot &c = col[j];
            std::fill(coef.begin() + 8 * j, coef.begin() + 8 * j + 8, 0.0);
            if (!c.active) continue;
            c.beta = rnorm[j];
            c.delta1 = c.eps = c.s = 0.0;
            c.c = -1.0;
            c.phi = rnorm[j];
            coef[8 * j + 0] = rnorm[j];
            coef[8 * j + 7] = 1.0;
        }
        FGK_CUDA(cudaMemcpyAsync(coef_d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        k_mr_restart<<<vgrid, 256, 0, s>>>(R, V, Vp, Dp, Dpp, coef_d, vec, nc);
        FGK_LAUNCH_CHECK();
        // the next Lanczos step needs beta_k = 0 for v_0 = 0
        for (int j = 0; j < nc; ++j) coef[8 * j + 0] = 0.0;
        return FGK_OK;
    };

    // one MINRES step on every active column (one host synchronisation)
    auto step = [&]() -> int {
        for (int j = 0; j < nc; ++j) coef[8 * j + 7] = col[j].active ? 1.0 : 0.0;
        FGK_CUDA(cudaMemcpyAsync(coef_d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        FGK_TRY(mvm_q_f64(p, V, nc, W, s, nullptr));
        ++n_f64;
        k_mr_dots<<<kMrBlocks, kMrThreads, 0, s>>>(V, W, sigma2, N, nc, partial);
        FGK_LAUNCH_CHECK();
        k_mr_finalize<<<(nc + 7) / 8, 256, 0, s>>>(partial, kMrBlocks, nc, alpha_d);
        FGK_LAUNCH_CHECK();
        k_mr_lanczos<<<kMrBlocks, kMrThreads, 0, s>>>(W, V, Vp, sigma2, alpha_d, coef_d, N, nc, partial);
        FGK_LAUNCH_CHECK();
        k_mr_finalize<<<(nc + 7) / 8, 256, 0, s>>>(partial, kMrBlocks, nc, beta_d);
        FGK_LAUNCH_CHECK();
        // alpha_k and ||p||^2 of every column, contiguous on the device
        FGK_CUDA(cudaMemcpyAsync(hab.data(), alpha_d, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        for (int j = 0; j < nc; ++j) {
            ColRot &c = col[j];
            double *cf = &coef[8 * j];
            if (!c.active) {
                cf[7] = 0.0;
                continue;
            }
            const double a = hab[j], bn = std::sqrt(hab[nc + j]);
            const double delta2 = c.c * c.delta1 + c.s * a;
            const double gamma1 = c.s * c.delta1 - c.c * a;
            const double eps_next = c.s * bn;
            const double delta1_next = -c.c * bn;
            const double gamma2 = std::hypot(gamma1, bn);
            if (!(gamma2 > 0.0) || !std::isfinite(gamma2)) {  // T_k singular: the column cannot move
                c.active = false;
                cf[7] = 0.0;
                continue;
            }
            const double cn = gamma1 / gamma2, sn = bn / gamma2;
            const double tau = cn * c.phi;
            c.phi = sn * c.phi;
            cf[1] = delta2;
            cf[2] = c.eps;
            cf[3] = gamma2;
            cf[4] = tau;
            cf[5] = bn;
            cf[7] = 1.0;
            c.beta = bn;
            c.delta1 = delta1_next;
            c.eps = eps_next;
            c.c = cn;
            c.s = sn;
        }
        FGK_CUDA(cudaMemcpyAsync(coef_d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        k_mr_update<<<vgrid, 256, 0, s>>>(X, V, Vp, W, Dp, Dpp, coef_d, vec, nc);
        FGK_LAUNCH_CHECK();
        std::swap(V, Vp);    // v_{k+1} was written over v_{k-1}
        std::swap(Dp, Dpp);  // d_k was written over d_{k-2}
        for (int j = 0; j < nc; ++j) {
            coef[8 * j + 0] = col[j].beta;  // beta_{k+1}, for the next step
            if (col[j].active && (col[j].phi <= tol * col[j].beta1 || col[j].beta == 0.0))
                col[j].active = false;  // claims convergence (or an invariant Krylov space)
        }
        return FGK_OK;
    };
    auto run = [&]() -> int {
        FGK_TRY(to_q_order(p, y, B, nc, 8, s));
        FGK_CUDA(cudaMemsetAsync(X, 0, vb, s));
        FGK_CUDA(cudaMemcpyAsync(R, B, vb, cudaMemcpyDeviceToDevice, s));
        FGK_TRY(colnorms(B, bnorm));
        rnorm = bnorm;
        for (int j = 0; j < nc; ++j) {
            if (!std::isfinite(bnorm[j])) {
                set_error("fgk_minres_solve: y holds a NaN or an infinity");
                return FGK_ERR_NONFINITE;
            }
            col[j].beta1 = bnorm[j];
            col[j].active = bnorm[j] > 0.0;
        }
        FGK_TRY(start());
        while (true) {
            bool any = false;
            for (int j = 0; j < nc; ++j) any = any || col[j].active;
            if (any && iters < maxit) {
                ++iters;
                FGK_TRY(step());
                continue;
            }
            // every column stopped (or maxit): confirm with the FP64 true residual
            FGK_TRY(residual());
            bool again = false;
            for (int j = 0; j < nc; ++j) {
                col[j].active = !(rnorm[j] <= tol * bnorm[j]) && iters < maxit && rnorm[j] > 0.0;
                again = again || col[j].active;
            }
            if (!again) break;
            ++restarts;
            FGK_TRY(start());
        }
        FGK_TRY(from_q_order(p, X, alpha, nc, 8, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        return FGK_OK;
    };
    rc = run();
    if (info) {
        double mx = 0.0;
        for (int j = 0; j < nc; ++j) {
            const double r = bnorm[j] > 0.0 ? rnorm[j] / bnorm[j] : 0.0;
            mx = std::max(mx, r);
            if (info->true_resid) info->true_resid[j] = r;
        }
        info->iterations = iters;
        info->refinements = restarts;
        info->mvm_f32 = 0;
        info->mvm_f64 = n_f64;
        info->max_true_resid = mx;
        info->restarts = restarts;
        info->fp64_switch = 0;
    }
    dev_free(mem, s);
    if (rc) return rc;
    for (int j = 0; j < nc; ++j)
        if (!(rnorm[j] <= tol * bnorm[j])) {
            set_error("fgk_minres_solve: column %d reached ||r|| / ||b|| = %.3g after %d iterations (tol %.3g)", j,
                      bnorm[j] > 0 ? rnorm[j] / bnorm[j] : 0.0, iters, tol);
            return FGK_NOT_CONVERGED;
        }
    return FGK_OK;
}

}  // namespace

}  // namespace fgk

using namespace fgk;

extern "C" int fgk_minres_solve(fgk_handle h, const double *y, int nrhs, double sigma2, double tol, int maxit,
                                double *alpha, fgk_cg_info *info, fgk_stream_t stream) {
    clear_error();
    if (!h || !y || !alpha) {
        set_error("fgk_minres_solve: h, y and alpha must not be NULL");
        return FGK_ERR_INVALID;
    }
    if (nrhs < 1 || nrhs > kMrMaxCols || !(sigma2 >= 0.0) || !std::isfinite(sigma2) || !(tol > 0.0) || maxit < 1) {
        set_error("fgk_minres_solve: need 1 <= nrhs <= %d, finite sigma2 >= 0, tol > 0, maxit >= 1", kMrMaxCols);
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    p->stream = (cudaStream_t)stream;
    return minres(p, y, nrhs, sigma2, tol, maxit, alpha, info, (cudaStream_t)stream);
}
