// The gradient of the log marginal likelihood (eq. gp_log_likelihood_derivative)
// with respect to the log-parameters theta = (log ell_k, log varsigma^2,
// log sigma^2), with the trace terms by Hutchinson probes (App. A.2):
//   d/dtheta = 1/2 a^T dK a - 1/2 tr(A^{-1} dK),  A = K + sigma^2 I, a = A^{-1} y,
//   tr(A^{-1} dK) ~ mean_i (A^{-1} b_i)^T dK (P^{-1} b_i)   (b_i ~ N(0, P)).
// One CG solve of [y, b_1 .. b_n] gives a and the A^{-1} b_i; the lengthscale
// derivatives take gradient products of a and of z_i = P^{-1} b_i.  The
// outputscale needs none: dK = K, a^T K a = a^T y - sigma^2 a^T a and
// x_i^T K z_i = b_i^T z_i - sigma^2 x_i^T z_i (A symmetric, x_i = A^{-1} b_i);
// the noise: dA = sigma^2 I, tr by mean_i sigma^2 x_i^T z_i.
#include <cstring>
#include <vector>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

// out[j] = sum_i A[i * lda + j] B[i * ldb + j], one CTA per column, fixed order
__global__ void k_pair_dots(const double *__restrict__ A, int lda, const double *__restrict__ B, int ldb, int64_t N,
                            int ncols, double *__restrict__ out) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    if (j >= ncols) return;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc = fma(A[i * lda + j], B[i * ldb + j], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

// C = [y, B] (N x (1 + n) row-major)
__global__ void k_stack_rhs(const double *__restrict__ y, const double *__restrict__ B, int64_t N, int n,
                            double *__restrict__ C) {
    const int64_t tot = N * (n + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / (n + 1);
        const int c = (int)(t % (n + 1));
        C[t] = c == 0 ? y[i] : B[i * n + c - 1];
    }
}

// out[i] = A[i * lda + col]
__global__ void k_column(const double *__restrict__ A, int lda, int col, int64_t N, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = A[i * lda + col];
}

int pair_dots(const double *A, int lda, const double *B, int ldb, int64_t N, int ncols, double *dev_out,
              double *host_out, cudaStream_t s) {
    k_pair_dots<<<ncols, 256, 0, s>>>(A, lda, B, ldb, N, ncols, dev_out);
    FGK_LAUNCH_CHECK();
    FGK_CUDA(cudaMemcpyAsync(host_out, dev_out, (size_t)ncols * sizeof(double), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaStreamSynchronize(s));
    return FGK_OK;
}

}  // namespace

}  // namespace fgk

using namespace fgk;

extern "C" {

int fgk_loglik_grad(fgk_handle h, fgk_precond pch, double sigma2, const double *y, const double *B, int nprobe,
                    double tol, int maxit, int mode, double *grad, fgk_grad_report *rep, fgk_stream_t stream) {
    clear_error();
    if (!h || !y || (nprobe > 0 && !B) || !grad || !rep || nprobe < 0 || nprobe > 63 || !(sigma2 > 0.0) || !std::isfinite(sigma2) ||
        !(tol > 0.0) || maxit < 1 || (mode != FGK_F64 && mode != FGK_MIXED)) {
        set_error("fgk_loglik_grad: need h, y, B (nprobe > 0), grad, rep, 0 <= nprobe <= 63, sigma2 > 0, tol > 0, maxit >= 1 "
                  "and mode FGK_F64 or FGK_MIXED");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    Precond *pc = pc_of(pch);
    if (pc && (pc_plan(pc) != p || pc_sigma2(pc) != sigma2)) {
        set_error("fgk_loglik_grad: the preconditioner belongs to another plan or sigma2");
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = p->N;
    const int nc = nprobe + 1;
    const bool product = p->d > 1 && p->kind == FGK_PRODUCT;
    const int nl = product ? p->d : 1;  // lengthscale entries
    // scratch: C = [y, B], X = A^{-1} C, Z = P^{-1} B, Da (N), DZ (N x n), dots
    const size_t cb = (size_t)N * nc * 8, zb = (size_t)N * nprobe * 8;
    auto rnd = [](size_t b) { return (b + 255) / 256 * 256; };
    char *buf = (char *)dev_alloc(2 * rnd(cb) + 2 * rnd(zb) + rnd((size_t)N * 8) + 4096, s);
    if (!buf) {
        set_error("fgk_loglik_grad: workspace allocation failed");
        return FGK_ERR_OOM;
    }
    double *C = (double *)buf;
    double *X = (double *)(buf + rnd(cb));
    double *Z = (double *)(buf + 2 * rnd(cb));
    double *DZ = (double *)(buf + 2 * rnd(cb) + rnd(zb));
    double *Da = (double *)(buf + 2 * rnd(cb) + 2 * rnd(zb));
    double *dd = (double *)(buf + 2 * rnd(cb) + 2 * rnd(zb) + rnd((size_t)N * 8));
    int rc = FGK_OK;
    fgk_cg_info info;
    std::memset(&info, 0, sizeof(info));
    std::vector<double> g(nl + 2, 0.0);
    do {
        k_stack_rhs<<<grid_for(N * nc, 256), 256, 0, s>>>(y, B, N, nprobe, C);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("fgk_loglik_grad: launch failed");
            rc = FGK_ERR_CUDA;
            break;
        }
        rc = cg_solve(p, pc, C, nc, sigma2, nullptr, 0, tol, maxit, mode, X, nullptr, &info, s);
        const int solve_rc = rc;
        if (rc != FGK_OK && rc != FGK_NOT_CONVERGED) break;
        rc = FGK_OK;
        if (nprobe == 0) {
        } else if (pc) {
            if ((rc = fgk_precond_apply(pch, B, nprobe, Z, stream))) break;
        } else if (cudaMemcpyAsync(Z, B, zb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            set_error("fgk_loglik_grad: copy failed");
            rc = FGK_ERR_CUDA;
            break;
        }
        // a^T y, a^T a (column 0 of X with y, with itself)
        double ay = 0.0, aa = 0.0;
        if ((rc = pair_dots(X, nc, y, 1, N, 1, dd, &ay, s))) break;
        if ((rc = pair_dots(X, nc, X, nc, N, 1, dd, &aa, s))) break;
        // b_i^T z_i and x_i^T z_i
        std::vector<double> bz(nprobe), xz(nprobe);
        if (nprobe > 0) {
            if ((rc = pair_dots(B, nprobe, Z, nprobe, N, nprobe, dd, bz.data(), s))) break;
            if ((rc = pair_dots(X + 1, nc, Z, nprobe, N, nprobe, dd, xz.data(), s))) break;
        }
        double mbz = 0.0, mxz = 0.0;
        for (int i = 0; i < nprobe; ++i) {
            mbz += bz[i] / nprobe;
            mxz += xz[i] / nprobe;
        }
        // lengthscales: 1/2 a^T dK a - 1/2 mean x_i^T dK z_i, with a (column 0
        // of X) gathered contiguous into C (free after the solve)
        k_column<<<grid_for(N, 256), 256, 0, s>>>(X, nc, 0, N, C);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("fgk_loglik_grad: launch failed");
            rc = FGK_ERR_CUDA;
            break;
        }
        for (int m = 0; m < nl && rc == FGK_OK; ++m) {
            const int dim = product ? m : -1;
            if ((rc = fgk_matvec_dlogell(h, C, 1, Da, dim, FGK_F64, stream))) break;
            double ada = 0.0;
            std::vector<double> xdz(nprobe);
            if ((rc = pair_dots(C, 1, Da, 1, N, 1, dd, &ada, s))) break;
            if (nprobe > 0) {
                if ((rc = fgk_matvec_dlogell(h, Z, nprobe, DZ, dim, FGK_F64, stream))) break;
                if ((rc = pair_dots(X + 1, nc, DZ, nprobe, N, nprobe, dd, xdz.data(), s))) break;
            }
            double tr = 0.0;
            for (int i = 0; i < nprobe; ++i) tr += xdz[i] / nprobe;
            g[m] = 0.5 * ada - 0.5 * tr;
        }
        if (rc) break;
        g[nl] = 0.5 * (ay - sigma2 * aa) - 0.5 * (mbz - sigma2 * mxz);  // outputscale
        g[nl + 1] = 0.5 * sigma2 * aa - 0.5 * sigma2 * mxz;             // noise
        for (int k = 0; k < nl + 2; ++k) grad[k] = g[k];
        rep->yAy = ay;
        rep->alpha_sq = aa;
        rep->max_true_resid = info.max_true_resid;
        rep->iterations = info.iterations;
        rep->solve_status = solve_rc;
        rep->n_grad = nl + 2;
    } while (0);
    dev_free(buf, s);
    return rc;
}

}  // extern "C"
