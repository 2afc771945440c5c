// Internal declarations shared by the libfgk translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "fgk.h"

namespace fgk {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();

// Status carried through internal calls; converted to the C codes at the ABI.
#define FGK_TRY(expr)                      \
    do {                                   \
        int _rc = (expr);                  \
        if (_rc != FGK_OK) return _rc;     \
    } while (0)

#define FGK_CUDA(expr)                                                                        \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess) {                                                              \
            ::fgk::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                             __LINE__);                                                       \
            return FGK_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

// Every kernel launch is followed by FGK_LAUNCH_CHECK(), which also counts it.
void add_kernel_launches(int64_t n);
uint64_t kernel_launch_count();
#define FGK_LAUNCH_CHECK()                    \
    do {                                      \
        ::fgk::add_kernel_launches(1);        \
        FGK_CUDA(cudaGetLastError());         \
    } while (0)

// Optional CUDA-event timing of selected kernels (tools; off by default).
enum : int { kTimedScanOut = FGK_TIMED_SCAN_OUT, kTimedPcLtr = FGK_TIMED_PC_LTR,
             kTimedPcApply = FGK_TIMED_PC_APPLY, kTimedKernels = 3 };
bool kernel_timing_enabled(int id);
void kernel_timing_record(int id, cudaEvent_t start, cudaEvent_t stop);
bool scan_timing_enabled();
void scan_timing_record(cudaEvent_t start, cudaEvent_t stop);

// Brackets one launch with events when timing of `id` is on and the stream
// is not being captured: begin() before the launch, end() after it.
struct TimedLaunch {
    int id;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TimedLaunch(int id_, cudaStream_t s_) : id(id_), s(s_) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (kernel_timing_enabled(id) && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
            cs == cudaStreamCaptureStatusNone && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess)
            cudaEventRecord(e0, s);
    }
    void end() {
        if (e1) {
            cudaEventRecord(e1, s);
            kernel_timing_record(id, e0, e1);
            e0 = e1 = nullptr;
        }
    }
};

// ---------------------------------------------------------------- memory
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// A device buffer owned by a plan (freed in the plan's destructor path).
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------- device error word
// Set by kernels whose bounded waits expire or whose checks fail (never a trap).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_INTERNAL = 2 };

// ---------------------------------------------------------------- constants
constexpr int kMaxD = 3;
constexpr int kMaxH = 8;

// Level-scan tiling: a CTA owns kTile consecutive entries of one level.
constexpr int kScanThreads = 256;
constexpr int kScanEPT = 8;  // entries per thread (power of two)
constexpr int kTile = kScanThreads * kScanEPT;

// One unit of scan work: tile `tile` of level `level`.  For levels whose
// segments are longer than a tile, `seg_tile0`/`seg_ntiles` give the tile
// range of the segment and `agg` indexes the aggregate/carry slot.
struct WorkItem {
    int32_t level;
    int32_t tile;
    int32_t agg;        // -1 for short-segment levels
    int32_t seg_tile0;  // first tile of this tile's segment (long levels)
    int32_t seg_ntiles; // tiles in this tile's segment (long levels)
    int32_t log2S;      // segment size of the level
};

// ---------------------------------------------------------------- plan
struct Plan {
    int64_t N = 0;
    int d = 0, two_nu = 0, kind = 0, P = 0;
    double s2 = 1.0;
    double ell[kMaxD] = {0, 0, 0};
    double a[kMaxD] = {0, 0, 0};  // sqrt(2 nu) / ell_k
    int L = 0;
    int nlev = 0;
    int64_t ldN = 0;  // stride between levels: N rounded up to a multiple of 64 entries
    cudaStream_t stream = nullptr;
    int device = 0;   // the CUDA device the plan was built on (current during fgk_build)
    int sort_spin_limit = 1 << 24;  // bound on the sort's look-back spins per predecessor

    // sort results (device)
    int32_t *perm[kMaxD] = {nullptr, nullptr, nullptr};  // position in x'_k order -> point
    int32_t *rank1 = nullptr;                            // point -> position in x'_1 order
    double *xq[kMaxD] = {nullptr, nullptr, nullptr};     // x'_k of the point at q (x'_1 order)
    double *xraw_q = nullptr;                            // N x d unscaled x in x'_1 order

    // structure: nlev levels of N entries, level-major with stride ldN
    uint32_t *lv_q = nullptr;  // q | r1 << 31 | r2 << 30
    float *lv_dl32 = nullptr;
    double *lv_dl64 = nullptr;
    float *lv_off32 = nullptr;   // (d-1) arrays of nlev x ldN, dimension-major
    double *lv_off64 = nullptr;
    double *lv_edl64 = nullptr;   // e^{-gap} of every FP64 gap (1 past each level's end)
    double *lv_eoff64 = nullptr;  // e^{-offset} of every FP64 offset (1 past each level's end)
    std::vector<int> lev_log2S;  // host

    // scan work lists (device + host copies)
    std::vector<WorkItem> items_host;
    WorkItem *items = nullptr;     // all items
    WorkItem *long_items = nullptr;
    int n_items = 0, n_long = 0;
    int ntiles = 0;                // tiles per level
    uint32_t *lv_map = nullptr;    // per block row of the lists: level | log2S << 16 (long levels first)
    int n_long_segments = 0;
    std::vector<int32_t> long_seg_host;  // [first agg, n tiles] per long segment
    int32_t *long_seg = nullptr;

    int *dev_err = nullptr;  // device error word

    std::vector<Buf> owned;
    size_t bytes_held = 0;

    // workspace (grown on demand)
    Buf ws;
    int ws_users = 0;
};

int plan_alloc(Plan *p, void **ptr, size_t bytes);  // plan-owned allocation
int check_dev_error(Plan *p, const char *where);    // reads and clears the error word (syncs)

// ---------------------------------------------------------------- build steps
int build_sort(Plan *p, const double *X);     // K0 + K1 (fgk_sort.cu)
int build_levels(Plan *p);                    // K2 (fgk_struct.cu)
int build_worklists(Plan *p);                 // host work lists for the scans (fgk_scan_*.cu)

// ---------------------------------------------------------------- product
// Y_q = s2 (V_q + sum_levels ...) for vectors in x'_1 order (q order).
// Vin: FP64 or FP32 (vin_f64), Yout of the scan precision (f64 flag), both
// N x nrhs row-major in q order.  Workspace is taken from p->ws.
// gate (device, may be NULL): when it points at 0 every kernel of the product
// returns at once (used inside captured CG iterations after convergence).
// init_diag = false: Yq already holds s2 * Vq (the diagonal term), written by
// the caller's own kernel.
int mvm_q_f64(Plan *p, const double *Vq, int nrhs, double *Yq, cudaStream_t s, const int *gate,
              bool init_diag = true);
int mvm_q_f32(Plan *p, const float *Vq, int nrhs, float *Yq, cudaStream_t s, const int *gate,
              bool init_diag = true);
size_t mvm_ws_bytes(const Plan *p, int nrhs, bool f64);
// the same products (init_diag, no gate) on caller-supplied scratch of
// mvm_ws_bytes(p, nrhs, f64) bytes; allocate nothing
int mvm_q_f64_ws(Plan *p, const double *Vq, int nrhs, double *Yq, double *ws, cudaStream_t s);
int mvm_q_f32_ws(Plan *p, const float *Vq, int nrhs, float *Yq, float *ws, cudaStream_t s);
// the runtime loads kernels lazily, on first launch; these make it load the
// plan's product kernels at build time instead
int scan_preload_f32(Plan *p);
int scan_preload_f64(Plan *p);
// the fixed scratch of fgk_matvec_q_noalloc on the current device: looked up
// (and the array reserved) once per device, at the first fgk_build there
int noalloc_setup();
// Y_q += s2 (dK/d log ell_dim) V_q in q order (fgk_dscan.cuh); dim in [0, d)
// for the product kernel, -1 for the radial (L1 or d = 1) derivative
int dlogell_q_f64(Plan *p, int dim, const double *Vq, int nrhs, double *Yq, cudaStream_t s);
int dlogell_q_f32(Plan *p, int dim, const float *Vq, int nrhs, float *Yq, cudaStream_t s);

int ensure_ws(Plan *p, size_t bytes, cudaStream_t s);

// gather/scatter between the caller's point order and q order
int to_q_order(const Plan *p, const void *src, void *dst, int nrhs, int elem_bytes, cudaStream_t s);
int from_q_order(const Plan *p, const void *src, void *dst, int nrhs, int elem_bytes, cudaStream_t s);

// Pivoted-Cholesky preconditioner (fgk_precond.cu).  pc_apply: Z = P^{-1} R
// for N x ncols FP64 row-major vectors in q order (ncols <= kPcMaxCols); when
// rz_partial is not NULL it also writes per-CTA partial sums of R .* Z per
// column, pc_partial_blocks(pc) rows of them (partial[b * ncols + j]).
// No host synchronisation and no allocation (after pc_reserve for ncols):
// safe inside stream capture.
struct Precond;
constexpr int kPcMaxCols = 64;
constexpr int kRedThreadsPc = 256;
int pc_apply(const Precond *pc, const double *R, int ncols, double *Z, double *rz_partial, cudaStream_t s,
             const int *gate = nullptr);  // gate: device int, 0 = skip (every kernel returns at once)
int pc_partial_blocks(const Precond *pc);           // CTAs (rows of partials) pc_apply's rz_partial has
int pc_check(const Precond *pc, cudaStream_t s);    // reads and clears the apply's error word (syncs)
int pc_reserve(Precond *pc, int ncols, cudaStream_t s);  // apply scratch for ncols (allocates; not in capture)
Precond *pc_of(fgk_precond h);  // the handle's preconditioner (NULL for NULL)
double pc_sigma2(const Precond *pc);
const Plan *pc_plan(const Precond *pc);

double pc_logdet(const Precond *pc);  // log det P (Sylvester)
int pc_rank(const Precond *pc);

// Lanczos coefficients recorded by a CG solve (Algorithm 2): dev_log holds
// (alpha, beta) per iteration and column, [(it * ncols + j) * 2 + {0, 1}] for
// it < cap; after the solve n[j] counts the iterations of column j's single
// Lanczos process (it ends at the column's first residual replacement) and
// gamma[j] = b_j^T P^{-1} b_j, the squared norm of its start vector.
struct LanczosLog {
    double *dev_log = nullptr;
    int cap = 0;
    int n[64] = {};
    double gamma[64] = {};
};

// CG / refinement / GLS (fgk_solve.cu); pc may be NULL (s_P = I)
int cg_solve(Plan *p, Precond *pc, const double *y, int nrhs, double sigma2, const double *H, int L,
             double tol, int maxit, int mode, double *alpha, double *beta, fgk_cg_info *info, cudaStream_t s,
             LanczosLog *lz = nullptr);
size_t solve_ws_bytes(const Plan *p, int ncols);

inline int ceil_log2_i64(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

// Column sums of a row-major block held one value per thread: thread t holds
// a value of column t % ncols (threads at or beyond (blockDim / ncols) * ncols
// hold 0).  Returns the column's total in threads 0..ncols-1 (other threads:
// unspecified).  red needs blockDim.x doubles; every thread of the block calls.
// A power-of-two ncols <= 32 folds within each warp with shuffles first (the
// lanes of one column sit ncols apart), then sums the warps' partials; any
// other ncols takes a shared-memory tree over the row slots.
__device__ __forceinline__ double block_col_sum(double v, int ncols, double *red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (ncols <= 32 && (ncols & (ncols - 1)) == 0) {
        for (int o = 16; o >= ncols; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int lane = tid & 31, warp = tid >> 5;
        if (lane < ncols) red[warp * ncols + lane] = v;
        __syncthreads();
        double t = 0.0;
        if (tid < ncols)
            for (int w = 0; w < (nt >> 5); ++w) t += red[w * ncols + tid];
        __syncthreads();
        return t;
    }
    red[tid] = v;
    __syncthreads();
    const int lr = tid / ncols;
    for (int n = nt / ncols; n > 1;) {
        const int h = (n + 1) >> 1;
        if (lr < h && lr + h < n) red[tid] += red[tid + h * ncols];
        __syncthreads();
        n = h;
    }
    const double t = tid < ncols ? red[tid] : 0.0;
    __syncthreads();
    return t;
}

inline unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace fgk

// The public opaque handle is the plan itself.
struct fgk_plan : public fgk::Plan {};
