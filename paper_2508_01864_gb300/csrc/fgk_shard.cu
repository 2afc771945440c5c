// One d = 1 problem split across devices by contiguous ranges of the sorted
// order (shards): each shard's plan gives the product over its own pairs;
// the pairs between shards need only P moments per shard and direction.
//
// With scaled coordinates a source j before a query i (x_j <= x_i) at
// distance x_i - x_j = D + delta_j, delta_j = x_a - x_j its distance to an
// anchor x_a <= x_i and D = x_i - x_a, contributes (Sec. 2.1, the fast sum
// updating of eq. fast_exact_decomposition_1d, with the running sums taken
// relative to the anchor so that every factor lies in [0, 1])
//   v_j k(D + delta_j) = e^{-D} sum_p c_p sum_{q<=p} C(p,q) D^{p-q}
//                        (v_j delta_j^q e^{-delta_j}),
// so the sources of a whole shard act through its moments
//   M_q = sum_j v_j delta_j^q e^{-delta_j},  q < P,
// taken relative to its last point (forward) or, mirrored, to its first
// point (backward).  fgk_shard_moments returns them; the host composes the
// moments of all earlier (later) shards at this shard's first (last) point
// by the binomial step M'_q = e^{-g} sum_{t<=q} C(q,t) g^{q-t} M_t over the
// gaps g between shards; fgk_shard_fixup adds the resulting terms to Y.
#include <cmath>
#include <vector>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kShThreads = 256;
constexpr int kShBlocks = 152;
constexpr int kShMaxP = 5;

__host__ __device__ constexpr double binom_d(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// partial[((b * nrhs + r) * 2 + dir) * P + q] = sum over this block's points
// of v delta^q e^{-delta}, delta = x_last - x (dir 0) or x - x_first (dir 1)
__global__ void k_shard_moments(const double *__restrict__ xq, const int32_t *__restrict__ perm,
                                const double *__restrict__ V, int64_t N, int nrhs, int P, double *__restrict__ partial) {
    __shared__ double red[kShThreads];
    const int r = blockIdx.y;
    const double xf = xq[0], xl = xq[N - 1];
    double acc[2][kShMaxP] = {};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const double v = V[(int64_t)perm[q] * nrhs + r];
        const double x = xq[q];
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const double dl = dir == 0 ? xl - x : x - xf;
            double w = v * exp(-dl);
#pragma unroll
            for (int k = 0; k < kShMaxP; ++k) {
                if (k < P) acc[dir][k] += w;
                w *= dl;
            }
        }
    }
    // block sums in a fixed tree order, one moment at a time
    for (int dir = 0; dir < 2; ++dir)
        for (int k = 0; k < P; ++k) {
            red[threadIdx.x] = acc[dir][k];
            __syncthreads();
            for (int h = blockDim.x / 2; h > 0; h >>= 1) {
                if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
                __syncthreads();
            }
            if (threadIdx.x == 0) partial[(((size_t)blockIdx.x * nrhs + r) * 2 + dir) * P + k] = red[0];
            __syncthreads();
        }
}

// out[(r * 2 + dir) * P + k] = sum over blocks, in block order
__global__ void k_shard_moments_sum(const double *__restrict__ partial, int nblk, int nout, double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nout) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += partial[(size_t)b * nout + t];
    out[t] = acc;
}

struct FixupArgs {
    double c[kShMaxP];               // Matérn coefficients c_p
    double s2;
};

// Y[point at q] += s2 (e^{-D} sum_p c_p sum_q C(p,q) D^{p-q} Cf_q
//                     + e^{-D'} sum_p c_p sum_q C(p,q) D'^{p-q} Cb_q),
// D = x - x_first, D' = x_last - x; carry = [r][dir][P] (dir 0: sources
// before the shard, anchored at x_first; dir 1: after it, at x_last)
__global__ void k_shard_fixup(const double *__restrict__ xq, const int32_t *__restrict__ perm,
                              const double *__restrict__ carry, int64_t N, int nrhs, int P, FixupArgs fa,
                              double *__restrict__ Y) {
    const double xf = xq[0], xl = xq[N - 1];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / nrhs;
        const int r = (int)(t - q * nrhs);
        const double x = xq[q];
        double acc = 0.0;
        for (int dir = 0; dir < 2; ++dir) {
            const double D = dir == 0 ? x - xf : xl - x;
            const double *M = carry + ((size_t)r * 2 + dir) * P;
            double Dp[kShMaxP];
            Dp[0] = 1.0;
            for (int k = 1; k < P; ++k) Dp[k] = Dp[k - 1] * D;
            double s = 0.0;
            for (int p = 0; p < P; ++p) {
                double inner = 0.0;
                for (int k = 0; k <= p; ++k) inner += binom_d(p, k) * Dp[p - k] * M[k];
                s += fa.c[p] * inner;
            }
            acc += exp(-D) * s;
        }
        Y[(int64_t)perm[q] * nrhs + r] += fa.s2 * acc;
    }
}

}  // namespace

}  // namespace fgk

using namespace fgk;

extern "C" int fgk_shard_moments(fgk_handle h, const double *V, int nrhs, double *out, fgk_stream_t stream) {
    clear_error();
    if (!h || !V || !out || nrhs < 1 || nrhs > 64) {
        set_error("fgk_shard_moments: need h, V, out and 1 <= nrhs <= 64");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    if (p->d != 1) {
        set_error("fgk_shard_moments: sharded products are built for d = 1 (d = %d)", p->d);
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int P = p->P;
    const int nout = nrhs * 2 * P;
    double *buf = (double *)dev_alloc(sizeof(double) * ((size_t)kShBlocks * nout + nout + 2), s);
    if (!buf) {
        set_error("fgk_shard_moments: workspace allocation failed");
        return FGK_ERR_OOM;
    }
    double *partial = buf, *sum = buf + (size_t)kShBlocks * nout;
    int rc = FGK_OK;
    auto run = [&]() -> int {
        k_shard_moments<<<dim3(kShBlocks, nrhs), kShThreads, 0, s>>>(p->xq[0], p->perm[0], V, p->N, nrhs, P, partial);
        FGK_LAUNCH_CHECK();
        k_shard_moments_sum<<<grid_for(nout, 128), 128, 0, s>>>(partial, kShBlocks, nout, sum);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(out, p->xq[0], sizeof(double), cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaMemcpyAsync(out + 1, p->xq[0] + p->N - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaMemcpyAsync(out + 2, sum, sizeof(double) * nout, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        return FGK_OK;
    };
    rc = run();
    dev_free(buf, s);
    return rc;
}

extern "C" int fgk_shard_fixup(fgk_handle h, const double *carry, int nrhs, double *Y, fgk_stream_t stream) {
    clear_error();
    if (!h || !carry || !Y || nrhs < 1 || nrhs > 64) {
        set_error("fgk_shard_fixup: need h, carry, Y and 1 <= nrhs <= 64");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    if (p->d != 1) {
        set_error("fgk_shard_fixup: sharded products are built for d = 1 (d = %d)", p->d);
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int P = p->P;
    const int ncar = nrhs * 2 * P;
    for (int i = 0; i < ncar; ++i)
        if (!std::isfinite(carry[i])) {
            set_error("fgk_shard_fixup: the carry holds a NaN or an infinity");
            return FGK_ERR_NONFINITE;
        }
    FixupArgs fa{};
    {
        // c_p of k(r) = sum_p c_p r^p e^{-r} (eq. matern_explicit in scaled units)
        auto fact = [](int n) {
            double f = 1.0;
            for (int k = 2; k <= n; ++k) f *= k;
            return f;
        };
        for (int q = 0; q < P; ++q)
            fa.c[q] = fact(P - 1) * fact(2 * P - 2 - q) * std::ldexp(1.0, q) / (fact(2 * P - 2) * fact(q) * fact(P - 1 - q));
    }
    fa.s2 = p->s2;
    double *dcar = (double *)dev_alloc(sizeof(double) * ncar, s);
    if (!dcar) {
        set_error("fgk_shard_fixup: workspace allocation failed");
        return FGK_ERR_OOM;
    }
    auto run = [&]() -> int {
        FGK_CUDA(cudaMemcpyAsync(dcar, carry, sizeof(double) * ncar, cudaMemcpyHostToDevice, s));
        const int64_t n = p->N * nrhs;
        k_shard_fixup<<<std::min<int64_t>(grid_for(n, 256), 4096), 256, 0, s>>>(p->xq[0], p->perm[0], dcar, p->N,
                                                                               nrhs, P, fa, Y);
        FGK_LAUNCH_CHECK();
        return FGK_OK;
    };
    const int rc = run();
    dev_free(dcar, s);
    return rc;
}
