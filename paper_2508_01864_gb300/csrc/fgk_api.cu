// The C ABI of libfgk (declared in include/fgk.h): argument checking, the
// allocator hook, plan lifetime, the build sequence (K0-K2), products in the
// caller's point order, and copies of the cached structure for inspection.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>

#include "fgk_internal.cuh"

namespace fgk {

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = {0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

// ---------------------------------------------------------------- launch counter / scan timing
static std::atomic<int64_t> g_launches{0};
void add_kernel_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t kernel_launch_count() { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

static std::mutex g_timing_mu;
static std::atomic<bool> g_timing_on[kTimedKernels];
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_timing_events[kTimedKernels];
static double g_timing_ms[kTimedKernels] = {};
static int64_t g_timing_n[kTimedKernels] = {};

bool kernel_timing_enabled(int id) { return g_timing_on[id].load(std::memory_order_relaxed); }
void kernel_timing_record(int id, cudaEvent_t start, cudaEvent_t stop) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timing_events[id].emplace_back(start, stop);
}
bool scan_timing_enabled() { return kernel_timing_enabled(kTimedScanOut); }
void scan_timing_record(cudaEvent_t start, cudaEvent_t stop) { kernel_timing_record(kTimedScanOut, start, stop); }
// folds recorded event pairs into the totals (synchronises on each pair)
static int timing_drain(int id) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (auto &e : g_timing_events[id]) {
        FGK_CUDA(cudaEventSynchronize(e.second));
        float ms = 0.f;
        FGK_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
        g_timing_ms[id] += ms;
        ++g_timing_n[id];
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    g_timing_events[id].clear();
    return FGK_OK;
}

// ---------------------------------------------------------------- allocator
static std::mutex g_alloc_mu;
static fgk_alloc_fn g_alloc = nullptr;
static fgk_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

void *dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    fgk_alloc_fn fa;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        fa = g_alloc;
        ctx = g_alloc_ctx;
    }
    if (fa) return fa(bytes, (fgk_stream_t)s, ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, cudaStream_t s) {
    if (!p) return;
    fgk_free_fn ff;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        ff = g_free;
        ctx = g_alloc_ctx;
    }
    if (ff) {
        ff(p, (fgk_stream_t)s, ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

int plan_alloc(Plan *p, void **ptr, size_t bytes) {
    void *q = dev_alloc(bytes, p->stream);
    if (!q) {
        set_error("device allocation of %zu bytes failed", bytes);
        return FGK_ERR_OOM;
    }
    p->owned.push_back(Buf{q, bytes});
    p->bytes_held += bytes;
    *ptr = q;
    return FGK_OK;
}

int ensure_ws(Plan *p, size_t bytes, cudaStream_t s) {
    if (p->ws.bytes >= bytes) return FGK_OK;
    if (p->ws.p) {
        dev_free(p->ws.p, s);
        p->bytes_held -= p->ws.bytes;
        p->ws = Buf{};
    }
    size_t want = std::max(bytes, (size_t)4096);
    void *q = dev_alloc(want, s);
    if (!q) {
        set_error("device allocation of a %zu-byte workspace failed", want);
        return FGK_ERR_OOM;
    }
    p->ws = Buf{q, want};
    p->bytes_held += want;
    return FGK_OK;
}

int check_dev_error(Plan *p, const char *where) {
    int h = 0;
    FGK_CUDA(cudaMemcpyAsync(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    FGK_CUDA(cudaStreamSynchronize(p->stream));
    if (h == DEV_OK) return FGK_OK;
    FGK_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), p->stream));
    if (h == DEV_TIMEOUT) {
        set_error("%s: a bounded device-side wait expired", where);
        return FGK_ERR_TIMEOUT;
    }
    set_error("%s: a device-side consistency check failed (code %d)", where, h);
    return FGK_ERR_INTERNAL;
}

static void plan_release(Plan *p) {
    cudaStream_t s = p->stream;
    for (auto &b : p->owned) dev_free(b.p, s);
    p->owned.clear();
    if (p->ws.p) dev_free(p->ws.p, s);
    p->ws = Buf{};
    p->bytes_held = 0;
}

// ---------------------------------------------------------------- work lists
int build_worklists(Plan *p) {
    const int64_t N = p->N;
    const int ntiles = (int)((N + kTile - 1) / kTile);
    std::vector<WorkItem> items, longs;
    std::vector<int32_t> segs;
    std::vector<uint32_t> map_long, map_short;
    int slot = 0;
    for (int lev = 0; lev < p->nlev; ++lev) {
        const int log2S = p->lev_log2S[lev];
        const int64_t S = int64_t(1) << log2S;
        (S <= kTile ? map_short : map_long).push_back((uint32_t)lev | ((uint32_t)log2S << 16));
        if (S <= kTile) {
            for (int t = 0; t < ntiles; ++t) items.push_back(WorkItem{lev, t, -1, 0, 0, log2S});
        } else {
            const int tps = (int)(S / kTile);
            for (int t0 = 0; t0 < ntiles; t0 += tps) {
                const int nt = std::min(tps, ntiles - t0);
                segs.push_back(slot);
                segs.push_back(nt);
                for (int t = t0; t < t0 + nt; ++t) {
                    WorkItem w{lev, t, slot++, t0, nt, log2S};
                    longs.push_back(w);
                }
            }
        }
    }
    // long-segment tiles first in the output launch: they carry more work per tile
    std::vector<WorkItem> all = longs;
    all.insert(all.end(), items.begin(), items.end());
    p->items_host = all;
    p->n_items = (int)all.size();
    p->n_long = (int)longs.size();
    p->n_long_segments = (int)(segs.size() / 2);
    p->long_seg_host = segs;
    p->ntiles = ntiles;
    // the kernels find their work item from the block index: level rows of
    // ntiles blocks each, in the order of the list (long levels first)
    std::vector<uint32_t> map = map_long;
    map.insert(map.end(), map_short.begin(), map_short.end());
    if (p->nlev > 0xffff) {
        set_error("fgk_build: %d levels exceed the level map", p->nlev);
        return FGK_ERR_INVALID;
    }
    if (!map.empty()) {
        FGK_TRY(plan_alloc(p, (void **)&p->lv_map, sizeof(uint32_t) * map.size()));
        FGK_CUDA(cudaMemcpyAsync(p->lv_map, map.data(), sizeof(uint32_t) * map.size(), cudaMemcpyHostToDevice,
                                 p->stream));
    }
    if (p->n_items) {
        FGK_TRY(plan_alloc(p, (void **)&p->items, sizeof(WorkItem) * all.size()));
        FGK_CUDA(cudaMemcpyAsync(p->items, all.data(), sizeof(WorkItem) * all.size(), cudaMemcpyHostToDevice,
                                 p->stream));
        p->long_items = p->items;  // the long tiles lead the list
    }
    if (!segs.empty()) {
        FGK_TRY(plan_alloc(p, (void **)&p->long_seg, sizeof(int32_t) * segs.size()));
        FGK_CUDA(cudaMemcpyAsync(p->long_seg, segs.data(), sizeof(int32_t) * segs.size(), cudaMemcpyHostToDevice,
                                 p->stream));
    }
    // the host vectors must outlive the asynchronous copies
    FGK_CUDA(cudaStreamSynchronize(p->stream));
    return FGK_OK;
}

// ---------------------------------------------------------------- permutation of vectors
namespace {
template <class T>
__global__ void k_gather_rows_t(const T *__restrict__ src, const int32_t *__restrict__ idx, int64_t N, int nrhs,
                                T *__restrict__ dst) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    const int64_t i = t / nrhs, r = t - i * nrhs;
    dst[t] = src[(int64_t)idx[i] * nrhs + r];
}
}  // namespace

int to_q_order(const Plan *p, const void *src, void *dst, int nrhs, int elem_bytes, cudaStream_t s) {
    const int64_t n = p->N * nrhs;
    if (elem_bytes == 8)
        k_gather_rows_t<double><<<grid_for(n, 256), 256, 0, s>>>((const double *)src, p->perm[0], p->N, nrhs,
                                                                (double *)dst);
    else
        k_gather_rows_t<float><<<grid_for(n, 256), 256, 0, s>>>((const float *)src, p->perm[0], p->N, nrhs,
                                                               (float *)dst);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

int from_q_order(const Plan *p, const void *src, void *dst, int nrhs, int elem_bytes, cudaStream_t s) {
    const int64_t n = p->N * nrhs;
    if (elem_bytes == 8)
        k_gather_rows_t<double><<<grid_for(n, 256), 256, 0, s>>>((const double *)src, p->rank1, p->N, nrhs,
                                                                (double *)dst);
    else
        k_gather_rows_t<float><<<grid_for(n, 256), 256, 0, s>>>((const float *)src, p->rank1, p->N, nrhs,
                                                               (float *)dst);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}


size_t plan_bytes_estimate(int64_t N, int d, int two_nu, int kind, int nrhs) {
    const int L = ceil_log2_i64(N);
    const int64_t nlev = d == 1 ? 1 : (d == 2 ? L : (int64_t)L * (L + 1) / 2);
    const int64_t E = nlev * ((N + 63) / 64 * 64);
    size_t b = 0;
    b += (size_t)E * (4 + 4 + 8 + (size_t)(d - 1) * 12);                // levels
    b += (size_t)N * (4 * d + 4 + 8 * d + 8 * d);                         // perms, rank, xq, xraw
    const int64_t ntiles = (N + kTile - 1) / kTile;
    b += (size_t)nlev * ntiles * sizeof(WorkItem) + (size_t)ntiles * 8;  // work lists
    b += (size_t)2 * nlev * ntiles * 2 * nrhs * 4 * 29 * 8;             // scan aggregates (upper bound)
    b += (size_t)nlev * N * nrhs * 8;                                      // level rows of an FP64 product
    b += (size_t)d * E * 8;                                                // stored FP64 decays
    b += (size_t)N * nrhs * 8 * 10 + (size_t)N * 8 * 12;                 // solver vectors
    (void)two_nu;
    (void)kind;
    return b + (1 << 20);
}

}  // namespace fgk

using namespace fgk;

// ====================================================================== ABI
extern "C" {

int fgk_set_allocator(fgk_alloc_fn alloc, fgk_free_fn free_fn, void *ctx) {
    clear_error();
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("fgk_set_allocator: give both functions or neither");
        return FGK_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return FGK_OK;
}

const char *fgk_last_error(void) { return g_err; }

size_t fgk_bytes_estimate(int64_t N, int d, int two_nu, int kind, int nrhs) {
    if (N < 1 || N > (int64_t(1) << 30) || d < 1 || d > 3 || two_nu < 1 || two_nu > 9 || two_nu % 2 == 0 ||
        (two_nu == 9 && d == 3) ||
        (kind != FGK_L1 && kind != FGK_PRODUCT) || nrhs < 1)
        return 0;
    return plan_bytes_estimate(N, d, two_nu, kind, nrhs);
}

int fgk_build(const double *X, int64_t N, int d, int two_nu, const double *ell, double outscale2, int kind,
              fgk_stream_t stream, fgk_handle *out) {
    clear_error();
    if (out) *out = nullptr;
    if (!out || !X || !ell) {
        set_error("fgk_build: X, ell and out must not be NULL");
        return FGK_ERR_INVALID;
    }
    if (N < 1 || N > (int64_t(1) << 30)) {
        set_error("fgk_build: N = %lld is outside [1, 2^30]", (long long)N);
        return FGK_ERR_INVALID;
    }
    if (d < 1 || d > 3) {
        set_error("fgk_build: d = %d is not 1, 2 or 3", d);
        return FGK_ERR_INVALID;
    }
    if (two_nu < 1 || two_nu > 9 || two_nu % 2 == 0) {
        set_error("fgk_build: two_nu = %d is not 1, 3, 5, 7 or 9", two_nu);
        return FGK_ERR_INVALID;
    }
    if (two_nu == 9 && d == 3) {
        set_error("fgk_build: nu = 9/2 is built for d <= 2 (its five-moment scans at d = 3 are not built)");
        return FGK_ERR_INVALID;
    }
    if (kind != FGK_L1 && kind != FGK_PRODUCT) {
        set_error("fgk_build: kind = %d is not FGK_L1 or FGK_PRODUCT", kind);
        return FGK_ERR_INVALID;
    }
    for (int k = 0; k < d; ++k)
        if (!(ell[k] > 0.0) || !std::isfinite(ell[k])) {
            set_error("fgk_build: ell[%d] = %g is not a finite positive number", k, ell[k]);
            return FGK_ERR_INVALID;
        }
    if (!(outscale2 > 0.0) || !std::isfinite(outscale2)) {
        set_error("fgk_build: outscale2 = %g is not a finite positive number", outscale2);
        return FGK_ERR_INVALID;
    }
    fgk_plan *p = new fgk_plan();
    p->N = N;
    p->d = d;
    p->two_nu = two_nu;
    p->kind = kind;
    p->P = (two_nu + 1) / 2;
    p->s2 = outscale2;
    p->stream = (cudaStream_t)stream;
    for (int k = 0; k < d; ++k) {
        p->ell[k] = ell[k];
        p->a[k] = std::sqrt((double)two_nu) / ell[k];
    }
    p->L = ceil_log2_i64(N);
    p->nlev = d == 1 ? 1 : (d == 2 ? p->L : p->L * (p->L + 1) / 2);
    p->ldN = (N + 63) / 64 * 64;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        set_error("fgk_build: cudaGetDevice failed");
        return FGK_ERR_CUDA;
    }
    int rc = plan_alloc(p, (void **)&p->dev_err, 16);
    if (rc == FGK_OK) rc = cudaMemsetAsync(p->dev_err, 0, 16, p->stream) == cudaSuccess ? FGK_OK : FGK_ERR_CUDA;
    if (rc == FGK_OK) rc = build_sort(p, X);
    if (rc == FGK_OK) rc = build_levels(p);
    if (rc == FGK_OK) rc = build_worklists(p);
    if (rc == FGK_OK) rc = scan_preload_f32(p);
    if (rc == FGK_OK) rc = scan_preload_f64(p);
    if (rc == FGK_OK) rc = noalloc_setup();
    if (rc == FGK_OK) rc = check_dev_error(p, "fgk_build");
    if (rc != FGK_OK) {
        plan_release(p);
        cudaStreamSynchronize(p->stream);
        delete p;
        return rc;
    }
    *out = p;
    return FGK_OK;
}

int fgk_matvec(fgk_handle h, const void *V, int nrhs, void *Y, int precision, fgk_stream_t stream) {
    clear_error();
    if (!h || !V || !Y) {
        set_error("fgk_matvec: h, V and Y must not be NULL");
        return FGK_ERR_INVALID;
    }
    if (nrhs < 1) {
        set_error("fgk_matvec: nrhs = %d < 1", nrhs);
        return FGK_ERR_INVALID;
    }
    if (precision != FGK_F64 && precision != FGK_F32) {
        set_error("fgk_matvec: precision must be FGK_F64 or FGK_F32");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int eb = precision == FGK_F64 ? 8 : 4;
    const size_t vb = (size_t)p->N * nrhs * eb;
    char *tmp = (char *)dev_alloc(2 * vb + 256, s);
    if (!tmp) {
        set_error("fgk_matvec: workspace allocation of %zu bytes failed", 2 * vb);
        return FGK_ERR_OOM;
    }
    void *Vq = tmp;
    void *Yq = tmp + ((vb + 255) / 256) * 256;
    int rc = to_q_order(p, V, Vq, nrhs, eb, s);
    if (rc == FGK_OK)
        rc = precision == FGK_F64 ? mvm_q_f64(p, (const double *)Vq, nrhs, (double *)Yq, s, nullptr)
                                  : mvm_q_f32(p, (const float *)Vq, nrhs, (float *)Yq, s, nullptr);
    if (rc == FGK_OK) rc = from_q_order(p, Yq, Y, nrhs, eb, s);
    dev_free(tmp, s);
    return rc;
}

int fgk_matvec_dlogell(fgk_handle h, const void *V, int nrhs, void *Y, int dim, int precision,
                       fgk_stream_t stream) {
    clear_error();
    if (!h || !V || !Y || nrhs < 1 || (precision != FGK_F64 && precision != FGK_F32)) {
        set_error("fgk_matvec_dlogell: need h, V, Y, nrhs >= 1 and precision FGK_F64 or FGK_F32");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    if (dim < -1 || dim >= p->d) {
        set_error("fgk_matvec_dlogell: dim = %d is outside [-1, %d)", dim, p->d);
        return FGK_ERR_INVALID;
    }
    const bool product = p->d > 1 && p->kind == FGK_PRODUCT;
    if (!product && p->d > 1 && dim >= 0) {
        set_error("fgk_matvec_dlogell: the L1 kernel's per-coordinate derivative is not supported "
                  "(pass dim = -1 for all lengthscales together)");
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    const int eb = precision == FGK_F64 ? 8 : 4;
    const size_t vb = (size_t)p->N * nrhs * eb;
    char *tmp = (char *)dev_alloc(2 * vb + 256, s);
    if (!tmp) {
        set_error("fgk_matvec_dlogell: workspace allocation of %zu bytes failed", 2 * vb);
        return FGK_ERR_OOM;
    }
    void *Vq = tmp;
    void *Yq = tmp + ((vb + 255) / 256) * 256;
    int rc = to_q_order(p, V, Vq, nrhs, eb, s);
    if (rc == FGK_OK && cudaMemsetAsync(Yq, 0, vb, s) != cudaSuccess) {
        set_error("fgk_matvec_dlogell: cudaMemsetAsync failed");
        rc = FGK_ERR_CUDA;
    }
    // product kernel: one scan per coordinate (summed for dim = -1);
    // radial (L1 or d = 1): one scan with the derivative's coefficients
    const int m0 = product ? (dim < 0 ? 0 : dim) : -1;
    const int m1 = product ? (dim < 0 ? p->d : dim + 1) : 0;
    for (int m = m0; rc == FGK_OK && m < m1; ++m)
        rc = precision == FGK_F64 ? dlogell_q_f64(p, m, (const double *)Vq, nrhs, (double *)Yq, s)
                                  : dlogell_q_f32(p, m, (const float *)Vq, nrhs, (float *)Yq, s);
    if (rc == FGK_OK) rc = from_q_order(p, Yq, Y, nrhs, eb, s);
    dev_free(tmp, s);
    return rc;
}

int fgk_matvec_q(fgk_handle h, const void *Vq, int nrhs, void *Yq, int precision, fgk_stream_t stream) {
    clear_error();
    if (!h || !Vq || !Yq || nrhs < 1 || (precision != FGK_F64 && precision != FGK_F32)) {
        set_error("fgk_matvec_q: bad argument");
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    cudaStream_t s = (cudaStream_t)stream;
    p->stream = s;
    return precision == FGK_F64 ? mvm_q_f64(p, (const double *)Vq, nrhs, (double *)Yq, s, nullptr)
                                : mvm_q_f32(p, (const float *)Vq, nrhs, (float *)Yq, s, nullptr);
}

uint64_t fgk_kernel_launches(void) { return kernel_launch_count(); }

int fgk_kernel_timing(int kernel, int enable, double *total_ms, int64_t *launches) {
    clear_error();
    if (kernel < 0 || kernel >= kTimedKernels) {
        set_error("fgk_kernel_timing: unknown kernel id %d", kernel);
        return FGK_ERR_INVALID;
    }
    int rc = timing_drain(kernel);
    if (rc != FGK_OK) return rc;
    if (total_ms) *total_ms = g_timing_ms[kernel];
    if (launches) *launches = g_timing_n[kernel];
    if (enable >= 0) {
        if (enable == 1 && !g_timing_on[kernel].load()) {
            g_timing_ms[kernel] = 0.0;
            g_timing_n[kernel] = 0;
        }
        g_timing_on[kernel].store(enable == 1);
    }
    return FGK_OK;
}

int fgk_scan_timing(int enable, double *total_ms, int64_t *launches) {
    return fgk_kernel_timing(FGK_TIMED_SCAN_OUT, enable, total_ms, launches);
}

static int cg_entry(const char *name, fgk_handle h, fgk_precond pc, const double *y, int nrhs, double sigma2,
                    const double *H, int L, double tol, int maxit, int mode, double *alpha, double *beta,
                    fgk_cg_info *info, fgk_stream_t stream) {
    clear_error();
    if (!h || !y || !alpha) {
        set_error("%s: h, y and alpha must not be NULL", name);
        return FGK_ERR_INVALID;
    }
    if (nrhs < 1 || !(sigma2 >= 0.0) || !std::isfinite(sigma2) || !(tol > 0.0) || maxit < 1) {
        set_error("%s: need nrhs >= 1, finite sigma2 >= 0, tol > 0, maxit >= 1", name);
        return FGK_ERR_INVALID;
    }
    if (mode != FGK_F64 && mode != FGK_MIXED) {
        set_error("%s: mode must be FGK_F64 or FGK_MIXED", name);
        return FGK_ERR_INVALID;
    }
    if (H == nullptr && L != 0 && L != -1) {
        set_error("%s: without H, L must be 0 (no fixed effects) or -1 (default [1, x])", name);
        return FGK_ERR_INVALID;
    }
    if (H != nullptr && (L < 1 || L > kMaxH)) {
        set_error("%s: L = %d is outside [1, %d]", name, L, kMaxH);
        return FGK_ERR_INVALID;
    }
    Plan *p = h;
    Precond *pcp = pc_of(pc);
    if (pcp && (pc_plan(pcp) != p || pc_sigma2(pcp) != sigma2)) {
        set_error("%s: the preconditioner was built for another plan or another sigma2", name);
        return FGK_ERR_INVALID;
    }
    if (L == -1) {
        L = 1 + p->d;
    }
    p->stream = (cudaStream_t)stream;
    return cg_solve(p, pcp, y, nrhs, sigma2, H, L, tol, maxit, mode, alpha, beta, info, (cudaStream_t)stream);
}

int fgk_cg_solve(fgk_handle h, const double *y, int nrhs, double sigma2, const double *H, int L, double tol,
                 int maxit, int mode, double *alpha, double *beta, fgk_cg_info *info, fgk_stream_t stream) {
    return cg_entry("fgk_cg_solve", h, nullptr, y, nrhs, sigma2, H, L, tol, maxit, mode, alpha, beta, info, stream);
}

int fgk_cg_solve_pc(fgk_handle h, fgk_precond pc, const double *y, int nrhs, double sigma2, const double *H, int L,
                    double tol, int maxit, int mode, double *alpha, double *beta, fgk_cg_info *info,
                    fgk_stream_t stream) {
    return cg_entry("fgk_cg_solve_pc", h, pc, y, nrhs, sigma2, H, L, tol, maxit, mode, alpha, beta, info, stream);
}

int fgk_destroy(fgk_handle h) {
    clear_error();
    if (!h) return FGK_OK;
    plan_release(h);
    delete h;
    return FGK_OK;
}

int fgk_get_info(fgk_handle h, fgk_plan_info *out) {
    clear_error();
    if (!h || !out) {
        set_error("fgk_get_info: NULL argument");
        return FGK_ERR_INVALID;
    }
    std::memset(out, 0, sizeof(*out));
    out->N = h->N;
    out->d = h->d;
    out->two_nu = h->two_nu;
    out->kind = h->kind;
    out->L = h->L;
    out->n_levels = h->nlev;
    out->outscale2 = h->s2;
    for (int k = 0; k < h->d; ++k) out->ell[k] = h->ell[k];
    out->device_bytes = h->bytes_held;
    return FGK_OK;
}

int fgk_get_permutation(fgk_handle h, int dim, int32_t *perm) {
    clear_error();
    if (!h || !perm || dim < 0 || dim >= h->d) {
        set_error("fgk_get_permutation: bad argument");
        return FGK_ERR_INVALID;
    }
    FGK_CUDA(cudaMemcpyAsync(perm, h->perm[dim], h->N * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    FGK_CUDA(cudaStreamSynchronize(h->stream));
    return FGK_OK;
}

int fgk_get_level(fgk_handle h, int level, uint32_t *q, uint8_t *roles, double *dl64, float *dl32, double *off64,
                  float *off32, int64_t *seg_size) {
    clear_error();
    if (!h || level < 0 || level >= h->nlev) {
        set_error("fgk_get_level: bad handle or level");
        return FGK_ERR_INVALID;
    }
    const int64_t N = h->N;
    const size_t lo = (size_t)level * h->ldN;
    cudaStream_t s = h->stream;
    if (seg_size) *seg_size = int64_t(1) << h->lev_log2S[level];
    std::vector<uint32_t> raw(N);
    FGK_CUDA(cudaMemcpyAsync(raw.data(), h->lv_q + lo, N * 4, cudaMemcpyDeviceToHost, s));
    if (dl64) FGK_CUDA(cudaMemcpyAsync(dl64, h->lv_dl64 + lo, N * 8, cudaMemcpyDeviceToHost, s));
    if (dl32) FGK_CUDA(cudaMemcpyAsync(dl32, h->lv_dl32 + lo, N * 4, cudaMemcpyDeviceToHost, s));
    const int nof = h->d - 1;
    std::vector<double> o64((size_t)N * std::max(nof, 1));
    std::vector<float> o32((size_t)N * std::max(nof, 1));
    for (int k = 0; k < nof; ++k) {
        const size_t src = ((size_t)k * h->nlev + level) * h->ldN;
        FGK_CUDA(cudaMemcpyAsync(o64.data() + (size_t)k * N, h->lv_off64 + src, N * 8, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaMemcpyAsync(o32.data() + (size_t)k * N, h->lv_off32 + src, N * 4, cudaMemcpyDeviceToHost, s));
    }
    FGK_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < N; ++i) {
        if (q) q[i] = raw[i] & 0x3fffffffu;
        if (roles) roles[i] = (uint8_t)(((raw[i] >> 31) & 1u) | (((raw[i] >> 30) & 1u) << 1));
        for (int k = 0; k < nof; ++k) {
            if (off64) off64[i * nof + k] = o64[(size_t)k * N + i];
            if (off32) off32[i * nof + k] = o32[(size_t)k * N + i];
        }
    }
    if (h->d < 3 && roles)
        for (int64_t i = 0; i < N; ++i) roles[i] &= (h->d == 2 ? 1 : 0);
    return FGK_OK;
}

}  // extern "C"
