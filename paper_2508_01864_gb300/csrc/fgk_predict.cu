// The posterior mean at new evaluation points (eq. gp_mean, eq. gp_mean_2):
// E[f(z)] = k_z^T alpha + h(z)^T beta for M points z.
//
// k_z^T alpha is a product with a rectangular block of the kernel matrix.
// It is computed exactly with the machinery of the square product: the plan
// of the union U = [X; Z] (the data in the plan's order, then the new
// points), the vector V = [alpha; 0] and one product Y = K_UU V; the rows of Y
// at the new points are sum_i K(z_j, x_i) alpha_i + s2 * 0, the sum over the
// data alone because every new point carries weight 0.  Building the union's
// sort and dominance structure costs about one build of N + M points; the
// product is the usual O((N + M) log^{d-1}(N + M)) one.
#include <algorithm>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

// U = [xraw_q; Z] row-major (N + M) x d; V = [alpha_q; 0] (N + M) x nrhs
__global__ void k_union_inputs(const double *__restrict__ xq, const double *__restrict__ Z, int64_t N, int64_t M,
                               int d, double *__restrict__ U) {
    const int64_t n = (N + M) * d;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / d;
        U[t] = row < N ? xq[t] : Z[t - N * d];
    }
}

template <class T>
__global__ void k_union_weights(const double *__restrict__ aq, int64_t N, int64_t M, int nrhs, T *__restrict__ V) {
    const int64_t n = (N + M) * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        V[t] = t < N * nrhs ? (T)aq[t] : T(0);
}

// out[j][c] = Y[N + j][c] + sum_l h_l(z_j) beta[l][c]; h = HZ rows, or the
// default [1, z] (unscaled coordinates) when HZ is NULL and L > 0
template <class T>
__global__ void k_predict_out(const T *__restrict__ Y, int64_t N, int64_t M, int nrhs, const double *__restrict__ HZ,
                              const double *__restrict__ Z, int d, int L, const double *__restrict__ beta,
                              double *__restrict__ out) {
    const int64_t n = M * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nrhs;
        const int c = (int)(t % nrhs);
        double v = (double)Y[N * nrhs + t];
        for (int l = 0; l < L; ++l) {
            const double h = HZ ? HZ[j * L + l] : (l == 0 ? 1.0 : Z[j * d + (l - 1)]);
            v += h * beta[l * nrhs + c];
        }
        out[t] = v;
    }
}

__global__ void k_finite_check(const double *__restrict__ a, int64_t n, int *__restrict__ bad) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[t])) atomicOr(bad, 1);
}

}  // namespace

}  // namespace fgk

using namespace fgk;

extern "C" int fgk_predict(fgk_handle h, const double *alpha, int nrhs, const double *Z, int64_t M,
                           const double *HZ, int L, const double *beta, int precision, double *out,
                           fgk_stream_t stream) {
    clear_error();
    if (!h || !alpha || !Z || !out || nrhs < 1 || M < 1 || (precision != FGK_F64 && precision != FGK_F32)) {
        set_error("fgk_predict: need h, alpha, Z, out, nrhs >= 1, M >= 1 and precision FGK_F64 or FGK_F32");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    if (HZ == nullptr && L != 0 && L != -1) {
        set_error("fgk_predict: without HZ, L must be 0 (no fixed effects) or -1 (default [1, z])");
        return FGK_ERR_INVALID;
    }
    if (HZ != nullptr && (L < 1 || L > kMaxH)) {
        set_error("fgk_predict: L = %d is outside [1, %d]", L, kMaxH);
        return FGK_ERR_INVALID;
    }
    if (L == -1) L = 1 + p->d;
    if (L > 0 && !beta) {
        set_error("fgk_predict: fixed effects need beta");
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = p->N, NU = N + M;
    const size_t elem = precision == FGK_F64 ? 8 : 4;
    double *U = (double *)dev_alloc((size_t)NU * p->d * 8, s);
    double *aq = (double *)dev_alloc((size_t)N * nrhs * 8, s);
    void *V = dev_alloc((size_t)NU * nrhs * elem, s);
    void *Y = dev_alloc((size_t)NU * nrhs * elem, s);
    int *bad = (int *)dev_alloc(16, s);
    fgk_handle hu = nullptr;
    int rc = FGK_OK;
    do {
        if (!U || !aq || !V || !Y || !bad) {
            set_error("fgk_predict: device allocation failed");
            rc = FGK_ERR_OOM;
            break;
        }
        FGK_CUDA(cudaMemsetAsync(bad, 0, 16, s));
        k_finite_check<<<grid_for((int64_t)N * nrhs, 256), 256, 0, s>>>(alpha, (int64_t)N * nrhs, bad);
        FGK_LAUNCH_CHECK();
        int hbad = 0;
        FGK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        if (hbad) {
            set_error("fgk_predict: alpha holds a NaN or an infinity");
            rc = FGK_ERR_NONFINITE;
            break;
        }
        k_union_inputs<<<grid_for(NU * p->d, 256), 256, 0, s>>>(p->xraw_q, Z, N, M, p->d, U);
        FGK_LAUNCH_CHECK();
        if ((rc = to_q_order(p, alpha, aq, nrhs, 8, s))) break;
        if (precision == FGK_F64)
            k_union_weights<double><<<grid_for(NU * nrhs, 256), 256, 0, s>>>(aq, N, M, nrhs, (double *)V);
        else
            k_union_weights<float><<<grid_for(NU * nrhs, 256), 256, 0, s>>>(aq, N, M, nrhs, (float *)V);
        FGK_LAUNCH_CHECK();
        // the union's plan (it validates Z: NaN / infinity -> FGK_ERR_NONFINITE)
        if ((rc = fgk_build(U, NU, p->d, p->two_nu, p->ell, p->s2, p->kind, stream, &hu))) break;
        if ((rc = fgk_matvec(hu, V, nrhs, Y, precision, stream))) break;
        if (precision == FGK_F64)
            k_predict_out<double><<<grid_for(M * nrhs, 256), 256, 0, s>>>((const double *)Y, N, M, nrhs, HZ, Z, p->d,
                                                                        L, beta, out);
        else
            k_predict_out<float><<<grid_for(M * nrhs, 256), 256, 0, s>>>((const float *)Y, N, M, nrhs, HZ, Z, p->d,
                                                                       L, beta, out);
        FGK_LAUNCH_CHECK();
    } while (0);
    if (hu) {
        const int rd = fgk_destroy(hu);
        if (!rc) rc = rd;
    }
    if (U) dev_free(U, s);
    if (aq) dev_free(aq, s);
    if (V) dev_free(V, s);
    if (Y) dev_free(Y, s);
    if (bad) dev_free(bad, s);
    return rc;
}
