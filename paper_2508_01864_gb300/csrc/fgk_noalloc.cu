// fgk_matvec_q_noalloc: the product in the plan's internal order for callers
// that must not allocate device memory during the call.
//
// A product needs scratch: one output row per level of the structure (the
// levels are summed in a fixed order afterwards) and the aggregates and
// carries of the segments longer than a tile.  The ordinary entry points take
// it from the plan's workspace, which grows with cudaMallocAsync (or the
// caller's allocator hook) when a product needs more.  Some callers cannot
// accept an allocation at that point: a serving loop that has handed its whole
// memory budget to admitted requests, an engine whose memory plan is fixed
// before it starts, a latency-critical path that cannot afford an allocator
// call or a possible out-of-memory error in the middle of its work.  This
// entry point uses instead one fixed scratch array compiled into the library:
//
//   - kNoAllocScratchBytes (64 MiB) of __device__ memory in this file's
//     module.  The CUDA runtime loads modules lazily, so the array is
//     reserved on a device when the module is first used there: the first
//     fgk_build on each device does that (noalloc_setup looks the array's
//     address up by cudaGetSymbolAddress, with that device current) and the
//     memory then stays reserved until the process exits.  fgk_build also has
//     the runtime load the plan's product kernels, so no call here loads code.
//   - every call on a device shares the array and it keeps the last call's
//     contents; nothing in it has to start at zero (each slot is written
//     before it is read within a call), but two calls whose work overlaps on
//     the GPU (different streams, or other threads) race on it and must be
//     ordered by the caller;
//   - a product whose scratch need exceeds the array is rejected with
//     FGK_ERR_INVALID before anything is launched, and so is a call made
//     while another device than the plan's is current.
#include <mutex>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// In host code this name stands for the array but is not its device
// address: only noalloc_setup's lookup gives that.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// the array's device address on the current device, looked up by
// noalloc_setup; NULL before that
void *noalloc_ptr(int dev) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    return (dev >= 0 && dev < kMaxDevices) ? g_noalloc_ptr[dev] : nullptr;
}

}  // namespace

int noalloc_setup() {
    int dev = 0;
    FGK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d is outside [0, %d)", dev, kMaxDevices);
        return FGK_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            set_error("cudaGetSymbolAddress of the fixed product scratch failed: %s", cudaGetErrorString(e));
            return FGK_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    return FGK_OK;
}

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
    const bool f64 = precision == FGK_F64;
    const size_t need = mvm_ws_bytes(p, nrhs, f64);
    if (need > kNoAllocScratchBytes) {
        set_error("fgk_matvec_q_noalloc: this product needs %zu bytes of scratch, more than the %zu-byte "
                  "array; use fewer right-hand sides or fgk_matvec_q",
                  need, kNoAllocScratchBytes);
        return FGK_ERR_INVALID;
    }
    int dev = -1;
    FGK_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) {
        set_error("fgk_matvec_q_noalloc: device %d is current but the plan was built on device %d", dev,
                  p->device);
        return FGK_ERR_INVALID;
    }
    void *scratch = noalloc_ptr(dev);
    if (!scratch) {  // fgk_build sets it up; reaching this means that failed
        set_error("fgk_matvec_q_noalloc: the fixed scratch of device %d was never set up", dev);
        return FGK_ERR_INTERNAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return f64 ? mvm_q_f64_ws(p, (const double *)Vq, nrhs, (double *)Yq, (double *)scratch, s)
               : mvm_q_f32_ws(p, (const float *)Vq, nrhs, (float *)Yq, (float *)scratch, s);
}
