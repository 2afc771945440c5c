// log det(K + sigma^2 I) by stochastic Lanczos quadrature (App. A.2,
// eq. approximationLogDet): CG with several probe right-hand sides records
// its coefficients (Algorithm 2), each column's coefficients give the
// tridiagonal Lanczos matrix T of the (preconditioned) operator started at
// that probe, and e_1^T log(T) e_1 is evaluated from the eigen-decomposition
// of T (Gauss quadrature: the eigenvalues are the nodes, the squared first
// components of the eigenvectors the weights).  With the preconditioner P the
// quadrature estimates log det(P^{-1}(K + sigma^2 I)) and log det P is added
// by Sylvester's theorem (App. A.3).
//
// The tridiagonal eigen-decomposition is host code: T is at most a few
// hundred rows, and only the first row of the eigenvector matrix is needed.
// It is the implicit symmetric QR iteration with Wilkinson shifts
// (Golub and Van Loan, Matrix Computations, Sec. 8.3), written for the
// diagonal/off-diagonal arrays, with the rotations accumulated into the first
// row of the eigenvector matrix only.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

// Eigenvalues of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal b (b[k] = T[k+1][k]) in lam, and the squared first components
// of the normalised eigenvectors in w.  Returns 0, or -1 if the iteration did
// not converge.
int tridiag_gauss(std::vector<double> a, std::vector<double> b, std::vector<double> &lam, std::vector<double> &w) {
    const int n = (int)a.size();
    std::vector<double> q(n, 0.0);  // first row of the accumulated rotations
    q[0] = 1.0;
    b.resize(n > 0 ? n : 1, 0.0);
    auto small = [&](int k) { return std::fabs(b[k]) <= DBL_EPSILON * (std::fabs(a[k]) + std::fabs(a[k + 1])); };
    int hi = n - 1, steps = 0;
    while (hi > 0) {
        if (small(hi - 1)) {  // a[hi] is an eigenvalue
            b[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;  // the unreduced block [lo, hi]
        while (lo > 0 && !small(lo - 1)) --lo;
        if (lo > 0) b[lo - 1] = 0.0;
        if (++steps > 60 * n) return -1;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 nearer a[hi]
        const double dd = 0.5 * (a[hi - 1] - a[hi]), bb = b[hi - 1];
        const double den = dd + (dd >= 0.0 ? 1.0 : -1.0) * std::hypot(dd, bb);
        const double mu = a[hi] - (den != 0.0 ? bb * bb / den : 0.0);
        // one implicit QR step: a rotation in plane (k, k+1) for each k,
        // the first chosen from the shifted column, the others chasing the
        // bulge T[k+1][k-1] down the band
        double x = a[lo] - mu, z = b[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = std::hypot(x, z);
            const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
            if (k > lo) b[k - 1] = r;
            const double ak = a[k], ak1 = a[k + 1], bk = b[k];
            a[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
            a[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
            b[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
            if (k + 1 < hi) {
                x = b[k];
                z = s * b[k + 1];  // the new bulge T[k+2][k]
                b[k + 1] *= c;
            }
            const double qk = q[k], qk1 = q[k + 1];
            q[k] = c * qk + s * qk1;
            q[k + 1] = -s * qk + c * qk1;
        }
    }
    lam = a;
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) w[i] = q[i] * q[i];
    return 0;
}

}  // namespace

// e_1^T log(T) e_1 for the Lanczos matrix of m CG steps (Algorithm 2):
// T[k][k] = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T[k+1][k] = sqrt(beta_k)/alpha_k.
int lanczos_logquad(const double *alpha, const double *beta, int m, double *out) {
    if (m < 1 || !alpha || (m > 1 && !beta) || !out) {
        set_error("lanczos quadrature: need m >= 1 coefficients");
        return FGK_ERR_INVALID;
    }
    std::vector<double> a(m), b(m > 1 ? m - 1 : 0), lam, w;
    for (int k = 0; k < m; ++k) {
        if (!(alpha[k] > 0.0) || !std::isfinite(alpha[k]) || (k + 1 < m && !(beta[k] >= 0.0))) {
            set_error("lanczos quadrature: coefficient %d is not a CG coefficient of an SPD operator", k);
            return FGK_ERR_INVALID;
        }
        a[k] = 1.0 / alpha[k] + (k > 0 ? beta[k - 1] / alpha[k - 1] : 0.0);
        if (k + 1 < m) b[k] = std::sqrt(beta[k]) / alpha[k];
    }
    if (tridiag_gauss(a, b, lam, w) != 0) {
        set_error("lanczos quadrature: the tridiagonal eigen-iteration did not converge");
        return FGK_ERR_INTERNAL;
    }
    double acc = 0.0;
    for (int i = 0; i < m; ++i) {
        if (!(lam[i] > 0.0)) {
            set_error("lanczos quadrature: Ritz value %g <= 0", lam[i]);
            return FGK_ERR_BREAKDOWN;
        }
        acc += w[i] * std::log(lam[i]);
    }
    *out = acc;
    return FGK_OK;
}

}  // namespace fgk

using namespace fgk;

extern "C" {

int fgk_lanczos_logquad(const double *alpha, const double *beta, int m, double *out) {
    clear_error();
    return lanczos_logquad(alpha, beta, m, out);
}

int fgk_slq_logdet(fgk_handle h, fgk_precond pch, double sigma2, const double *B, int nprobe, int m, double tol,
                   double *X, double *quad, int *steps, fgk_slq_report *rep, fgk_stream_t stream) {
    clear_error();
    if (!h || !B || !rep || nprobe < 1 || nprobe > 64 || m < 1 || !(sigma2 >= 0.0) || !std::isfinite(sigma2) ||
        !(tol > 0.0)) {
        set_error("fgk_slq_logdet: need h, B, rep, 1 <= nprobe <= 64, m >= 1, sigma2 >= 0 and tol > 0");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    Precond *pc = pc_of(pch);
    if (pc && (pc_plan(pc) != p || pc_sigma2(pc) != sigma2)) {
        set_error("fgk_slq_logdet: the preconditioner belongs to another plan or sigma2");
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t logb = (size_t)m * nprobe * 2 * sizeof(double);
    const size_t xb = X ? 0 : (size_t)p->N * nprobe * sizeof(double);
    char *buf = (char *)dev_alloc(logb + xb + 256, s);
    if (!buf) {
        set_error("fgk_slq_logdet: workspace allocation failed");
        return FGK_ERR_OOM;
    }
    LanczosLog lz;
    lz.dev_log = (double *)buf;
    lz.cap = m;
    double *Xd = X ? X : (double *)(buf + (logb + 255) / 256 * 256);
    fgk_cg_info info;
    std::memset(&info, 0, sizeof(info));
    int rc = cg_solve(p, pc, B, nprobe, sigma2, nullptr, 0, tol, m, FGK_F64, Xd, nullptr, &info, s, &lz);
    const int solve_rc = rc;
    if (rc == FGK_NOT_CONVERGED) rc = FGK_OK;  // a partial Lanczos process is what the quadrature takes
    std::vector<double> hlog((size_t)m * nprobe * 2);
    if (rc == FGK_OK) {
        if (cudaMemcpyAsync(hlog.data(), lz.dev_log, logb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("fgk_slq_logdet: copying the Lanczos coefficients failed");
            rc = FGK_ERR_CUDA;
        }
    }
    dev_free(buf, s);
    if (rc) return rc;
    double sum = 0.0;
    int smax = 0;
    std::vector<double> al(m), be(m);
    for (int j = 0; j < nprobe; ++j) {
        const int n = lz.n[j];
        double qj = 0.0;
        if (n > 0) {
            for (int k = 0; k < n; ++k) {
                al[k] = hlog[((size_t)k * nprobe + j) * 2];
                be[k] = hlog[((size_t)k * nprobe + j) * 2 + 1];
            }
            double e = 0.0;
            FGK_TRY(lanczos_logquad(al.data(), be.data(), n, &e));
            qj = lz.gamma[j] * e;
        }
        if (quad) quad[j] = qj;
        if (steps) steps[j] = n;
        sum += qj;
        smax = std::max(smax, n);
    }
    rep->logdet_precond = pc ? pc_logdet(pc) : 0.0;
    rep->logdet = rep->logdet_precond + sum / nprobe;
    rep->steps_max = smax;
    rep->solve_status = solve_rc;
    rep->max_true_resid = info.max_true_resid;
    return FGK_OK;
}

}  // extern "C"
