// fgk_fma_rate: the device's fused multiply-add throughput, measured (the
// denominator of the ALU roofline that the FP64 scans and the FP32 scans with
// many moments are bound by).  Each thread runs 16 independent FMA chains
// x <- x * a + b with a = 1 - 2^-10 and b = 2^-12 (the chains contract
// toward b / (1 - a) and never overflow), so the pipe, not latency, limits
// the rate; the chains' sum is stored when a run-time flag is set, which
// keeps the compiler from dropping them.
#include <algorithm>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kFmaChains = 16;
constexpr int kFmaThreads = 256;
constexpr int kFmaIters = 4096;

template <class T>
__global__ void __launch_bounds__(kFmaThreads) k_fma(T a, T b, int store, T *__restrict__ out) {
    T x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = T(threadIdx.x + c);
#pragma unroll 4
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int fma_rate(int reps, double *flops, cudaStream_t s) {
    int dev = 0, sms = 0;
    FGK_CUDA(cudaGetDevice(&dev));
    FGK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    T *out = (T *)dev_alloc(sizeof(T) * (size_t)blocks * kFmaThreads, s);
    if (!out) {
        set_error("fgk_fma_rate: allocation failed");
        return FGK_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FGK_OK;
    auto run = [&]() -> int {
        FGK_CUDA(cudaEventCreate(&e0));
        FGK_CUDA(cudaEventCreate(&e1));
        const T a = T(1) - T(1.0 / 1024), b = T(1.0 / 4096);
        k_fma<T><<<blocks, kFmaThreads, 0, s>>>(a, b, 0, out);  // warm-up
        FGK_LAUNCH_CHECK();
        float best = 1e30f;
        for (int r = 0; r < reps; ++r) {
            FGK_CUDA(cudaEventRecord(e0, s));
            k_fma<T><<<blocks, kFmaThreads, 0, s>>>(a, b, 0, out);
            FGK_LAUNCH_CHECK();
            FGK_CUDA(cudaEventRecord(e1, s));
            FGK_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            FGK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        *flops = 2.0 * kFmaChains * kFmaIters * (double)blocks * kFmaThreads / (best * 1e-3);
        return FGK_OK;
    };
    rc = run();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(out, s);
    return rc;
}

}  // namespace

}  // namespace fgk

using namespace fgk;

extern "C" int fgk_fma_rate(int precision, int reps, double *flops, fgk_stream_t stream) {
    clear_error();
    if (!flops || reps < 1 || (precision != FGK_F32 && precision != FGK_F64)) {
        set_error("fgk_fma_rate: need flops, reps >= 1 and precision FGK_F32 or FGK_F64");
        return FGK_ERR_INVALID;
    }
    return precision == FGK_F64 ? fma_rate<double>(reps, flops, (cudaStream_t)stream)
                                : fma_rate<float>(reps, flops, (cudaStream_t)stream);
}
