// fgk_matvec_q_noalloc: the product in the plan's internal order for callers
// that must not allocate device memory during the call.
//
// The level scans need scratch for the per-tile aggregates and carries of
// segments longer than a tile.  The ordinary entry points take it from the
// plan's workspace, which grows with cudaMallocAsync when a larger nrhs
// arrives.  Callers whose device memory is fully planned before they start
// (a serving loop that has handed its whole budget to admitted requests, an
// engine that forbids allocation once its memory plan is fixed, a real-time
// path that cannot afford an allocator call) cannot accept that.  This entry
// point uses instead one fixed scratch array compiled into the library:
//
//   - kNoAllocScratchBytes (16 MiB) of __device__ memory, reserved on every
//     GPU that loads the library for as long as the process lives;
//   - its device address is looked up once per device, with that device
//     current, by cudaGetSymbolAddress on the first call made on that
//     device (make that first call before any stream capture);
//   - every call on a device shares the array and it keeps the last call's
//     contents; nothing in it has to start at zero (each slot is written
//     before it is read within a call), but two calls whose work overlaps on
//     the GPU (different streams, or other threads) race on it and must be
//     ordered by the caller;
//   - a product whose scratch need exceeds the array is rejected with
//     FGK_ERR_INVALID before anything is launched.
#include <mutex>

#include "fgk_scan.cuh"

namespace fgk {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device (set up once)
int noalloc_scratch(void **out) {
    int dev = 0;
    FGK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fgk_matvec_q_noalloc: device ordinal %d is outside [0, %d)", dev, kMaxDevices);
        return FGK_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("fgk_matvec_q_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                      cudaGetErrorString(e));
            return FGK_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FGK_OK;
}

// bytes of tile aggregates and carries the level scans of this plan need:
// per long tile, direction, rhs and pass, an aggregate and a carry of
// 1 + (channels per pass) x (offset groups per pass) x P values
size_t noalloc_need(const Plan *p, int nrhs, size_t elem) {
    const int noff = p->d - 1;
    int na = 1;
    if (p->kind == FGK_PRODUCT && p->P > 1)
        for (int k = 0; k < noff; ++k) na *= p->P;
    const size_t cp = noff == 0 ? 1 : 2;
    const size_t npass = noff == 2 ? 2 : 1;
    const size_t gp = (na > 1 && cp * na * p->P > 12) ? 1 : na;  // as the scan kernels split them
    const size_t ngp = na / gp;
    const size_t ag = 1 + cp * gp * p->P;
    return (size_t)2 * p->n_long * 2 * nrhs * npass * ngp * ag * elem;
}

}  // namespace

}  // namespace fgk

using namespace fgk;

extern "C" int fgk_matvec_q_noalloc(fgk_handle h, const void *Vq, int nrhs, void *Yq, int precision,
                                    fgk_stream_t stream) {
    clear_error();
    if (!h || !Vq || !Yq || nrhs < 1 || (precision != FGK_F64 && precision != FGK_F32)) {
        set_error("fgk_matvec_q_noalloc: bad argument");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t elem = precision == FGK_F64 ? sizeof(double) : sizeof(float);
    const size_t need = noalloc_need(p, nrhs, elem);
    if (need > kNoAllocScratchBytes) {
        set_error("fgk_matvec_q_noalloc: this product needs %zu bytes of scratch, more than the %zu-byte "
                  "array; use fewer right-hand sides or fgk_matvec_q",
                  need, kNoAllocScratchBytes);
        return FGK_ERR_INVALID;
    }
    void *scratch = nullptr;
    FGK_TRY(noalloc_scratch(&scratch));
    const int64_t n = p->N * nrhs;
    if (precision == FGK_F64) {
        k_diag_init<double><<<grid_for(n, 256), 256, 0, s>>>((const double *)Vq, n, p->s2, (double *)Yq, nullptr);
        FGK_LAUNCH_CHECK();
        if (p->nlev == 0) return FGK_OK;
        return run_levels_dispatch<double>(p, (const double *)Vq, nrhs, (double *)Yq, (double *)scratch, s, nullptr);
    }
    k_diag_init<float><<<grid_for(n, 256), 256, 0, s>>>((const float *)Vq, n, (float)p->s2, (float *)Yq, nullptr);
    FGK_LAUNCH_CHECK();
    if (p->nlev == 0) return FGK_OK;
    return run_levels_dispatch<float>(p, (const float *)Vq, nrhs, (float *)Yq, (float *)scratch, s, nullptr);
}
