// Batches: many independent GP problems (each its own plan, d <= 2) and
// their right-hand sides advanced together.
//
// Products.  The vectors of all problems are packed one after the other
// (problem b occupies rows [off_b, off_b + N_b), each row its nrhs values, in
// that problem's x'_1 order).  One launch per phase of the product covers the
// whole batch: the tile-aggregate pass over every long-segment tile of every
// problem, the carry scan over every long segment, and the output pass over
// every tile; each CTA reads its problem's descriptor and runs the scan
// instantiated for that problem's nu, d and kernel kind.  The right-hand
// sides of a tile can be split across CTAs (rhs_per_cta), which the autotuner
// of the Python engine picks.
//
// Solves (mixed precision, as fgk_cg_solve): CG over all columns of all
// problems at once, each column with its own alpha, beta and stop test, the
// inner products reduced per problem over row chunks; one iteration (batched
// product + three vector kernels) is captured once as a CUDA graph and
// replayed.  A problem whose columns have all stopped is skipped by every
// kernel.  Residual replacements (FP64 products) are taken per problem with
// the single-plan FP64 product, spaced by the measured cost ratio.  With
// per-problem pivoted-Cholesky preconditioners (fgk_batch_cg_solve_pc) the
// iteration also applies each problem's P^{-1} (gated on the problem being
// active), rho = r^T z and p = z + beta p, and replacements restart every
// column from p = z (plain refinement with delta = 1e-3, as fgk_cg_solve_pc).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fgk_scan.cuh"

namespace fgk {

struct BatchProb {
    const uint32_t *lv_q;
    const float *lv_dl;
    const float *lv_off;
    int64_t N, ldN;
    int nlev;
    int variant;  // (P * 3 + d - 1) * 2 + kind, kind folded to L1 when nu = 1/2 or d = 1
    float s2;
    int64_t voff;     // first packed row
    int64_t agg_off;  // first float of this problem's aggregate / carry slots
};

struct BatchItem {
    WorkItem w;
    int32_t prob;
    int32_t r0, r1;  // right-hand sides handled by the CTA
};

struct BatchSeg {
    int32_t prob, a0, nt, pad;
};

struct Chunk {
    int32_t prob, row0, row1, first;  // packed rows [row0, row1) of problem prob; first chunk of it?
};

struct BatchArgs {
    const BatchProb *probs;
    const BatchItem *items;
    const BatchSeg *segs;
    int nseg;
    const float *V;
    float *Y;
    int nrhs;
    float *agg;
    float *carry;
    const int *prob_active;  // NULL, or per problem the number of active columns
    int *err;
};

namespace {

constexpr int kChunkRows = 2048;
constexpr int kRedThreads = 256;

constexpr int variant_key(int P, int noff, int kind) { return (P * 3 + noff) * 2 + kind; }

// One kernel per variant (P, split dimensions, kind), over that variant's
// contiguous range of the work list (items first .. first + gridDim.x - 1):
// each variant gets its own register allocation instead of the largest one's.
template <int MODE, int PP, int NO, int KK>
__global__ void __launch_bounds__(kScanThreads, FGK_SCAN_MINB) k_batch_scan(BatchArgs B, int first) {
    const BatchItem bi = B.items[first + blockIdx.x];
    if (B.prob_active && B.prob_active[bi.prob] == 0) return;
    const BatchProb pr = B.probs[bi.prob];
    if (pr.variant != variant_key(PP, NO, KK)) {  // the host groups the list by variant
        if (threadIdx.x == 0) atomicExch(B.err, DEV_INTERNAL);
        return;
    }
    ScanArgs<float> A;
    A.lv_q = pr.lv_q;
    A.lv_dl = pr.lv_dl;
    A.lv_off = pr.lv_off;
    A.lv_edl = nullptr;  // FP32: decays computed per entry
    A.lv_eoff = nullptr;
    A.N = pr.N;
    A.ldN = pr.ldN;
    A.nlev = pr.nlev;
    A.items = nullptr;
    A.lv_map = nullptr;  // the work item comes from the batch list
    A.ntiles = 0;
    A.n_long = 0;
    A.V = B.V + pr.voff * B.nrhs;
    A.nrhs = B.nrhs;
    A.Y = B.Y + pr.voff * B.nrhs;
    A.rows = nullptr;  // outputs added to Y atomically
    A.row_stride = 0;
    A.agg = (MODE == SCAN_AGG ? B.agg : B.carry) + pr.agg_off;
    A.s2 = pr.s2;
    A.err = B.err;
    A.gate = nullptr;
    scan_tile<float, PP, NO, KK, MODE, false, false>(A, bi.w, bi.r0, bi.r1);
}

// the variants a batch can hold (d <= 2, nu <= 5/2; nu = 1/2 and d = 1 use the L1 scans)
constexpr int kBatchVariants = 8;
constexpr int kBatchVariantKey[kBatchVariants] = {
    variant_key(1, 0, FGK_L1), variant_key(2, 0, FGK_L1), variant_key(3, 0, FGK_L1), variant_key(1, 1, FGK_L1),
    variant_key(2, 1, FGK_L1), variant_key(3, 1, FGK_L1), variant_key(2, 1, FGK_PRODUCT),
    variant_key(3, 1, FGK_PRODUCT)};

template <int MODE>
int launch_batch_scan(int v, const BatchArgs &A, int first, int count, cudaStream_t s) {
    switch (v) {
#define FGK_BCASE(I, PP, NO, KK)                                                  \
    case I:                                                                       \
        k_batch_scan<MODE, PP, NO, KK><<<count, kScanThreads, 0, s>>>(A, first); \
        break;
        FGK_BCASE(0, 1, 0, FGK_L1)
        FGK_BCASE(1, 2, 0, FGK_L1)
        FGK_BCASE(2, 3, 0, FGK_L1)
        FGK_BCASE(3, 1, 1, FGK_L1)
        FGK_BCASE(4, 2, 1, FGK_L1)
        FGK_BCASE(5, 3, 1, FGK_L1)
        FGK_BCASE(6, 2, 1, FGK_PRODUCT)
        FGK_BCASE(7, 3, 1, FGK_PRODUCT)
#undef FGK_BCASE
        default:
            set_error("batch: unknown scan variant %d", v);
            return FGK_ERR_INTERNAL;
    }
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

// one warp per (segment, direction, rhs, pass); passes beyond a variant's own
// count return at once
constexpr int kMaxBatchNPT = 3;

__global__ void k_batch_carry(BatchArgs B) {
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t total = (int64_t)B.nseg * 2 * B.nrhs * kMaxBatchNPT;
    if (wid >= total) return;
    const int pq = (int)(wid % kMaxBatchNPT);
    const int r = (int)((wid / kMaxBatchNPT) % B.nrhs);
    const int dir = (int)((wid / ((int64_t)kMaxBatchNPT * B.nrhs)) % 2);
    const BatchSeg sg = B.segs[wid / ((int64_t)kMaxBatchNPT * B.nrhs * 2)];
    if (B.prob_active && B.prob_active[sg.prob] == 0) return;
    const BatchProb pr = B.probs[sg.prob];
    const float *agg = B.agg + pr.agg_off;
    float *carry = B.carry + pr.agg_off;
    switch (pr.variant) {
#define FGK_BCASE(PP, NO, KK)                                                                  \
    case variant_key(PP, NO, KK):                                                              \
        if (pq < Traits<PP, NO, KK>::NPT)                                                      \
            carry_warp<float, PP, NO, KK>(agg, carry, sg.a0, sg.nt, dir, r, pq, B.nrhs);       \
        break;
        FGK_BCASE(1, 0, FGK_L1)
        FGK_BCASE(2, 0, FGK_L1)
        FGK_BCASE(3, 0, FGK_L1)
        FGK_BCASE(1, 1, FGK_L1)
        FGK_BCASE(2, 1, FGK_L1)
        FGK_BCASE(3, 1, FGK_L1)
        FGK_BCASE(2, 1, FGK_PRODUCT)
        FGK_BCASE(3, 1, FGK_PRODUCT)
#undef FGK_BCASE
        default:
            break;
    }
}

// Y = s2_b V on every packed row (the diagonal term), chunk by chunk
__global__ void k_batch_diag(const float *__restrict__ V, float *__restrict__ Y, const Chunk *__restrict__ chunks,
                             const BatchProb *__restrict__ probs, int nrhs) {
    const Chunk c = chunks[blockIdx.x];
    const float s2 = probs[c.prob].s2;
    for (int64_t t = (int64_t)c.row0 * nrhs + threadIdx.x; t < (int64_t)c.row1 * nrhs; t += blockDim.x)
        Y[t] = s2 * V[t];
}

// ------------------------------------------------------------------ batched CG
struct BState {
    double *rho, *rho_next, *thr2;
    double *rr;  // recursive ||r||^2 after the last p-update (rho is r^T z)
    int *active, *active_next, *iters;
    int *prob_active, *prob_active_next;
    int *bd;  // per column: met p^T A p <= 0 in FP32 (cleared by the host)
    int *breakdown;
};

// sum over a problem's chunks of the partials of column j (one warp)
__device__ __forceinline__ double warp_prob_sum(const double *__restrict__ partial, int c0, int nc, int nrhs, int j,
                                                int lane) {
    double acc = 0.0;
    for (int c = c0 + lane; c < c0 + nc; c += 32) acc += partial[(size_t)c * nrhs + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// block-wide column sums over the chunk's rows: out[j] = sum_rows f(row, j).
// Thread tid owns column tid % nrhs and every (blockDim / nrhs)-th row, so a
// warp reads consecutive elements of the row-major block in one pass.
template <class F>
__device__ __forceinline__ void chunk_col_sums(const Chunk &c, int nrhs, F f, double *out, double *red) {
    const int per = kRedThreads / nrhs;  // rows handled at once
    const int j = threadIdx.x % nrhs, lane_row = threadIdx.x / nrhs;
    double acc = 0.0;
    if (lane_row < per)
        for (int64_t row = c.row0 + lane_row; row < c.row1; row += per) acc += f(row, j);
    const double t = block_col_sum(acc, nrhs, red);
    if (threadIdx.x < nrhs) out[threadIdx.x] = t;
}

// p^T (w + sigma2 p) per chunk and column; the first chunk of each problem
// moves its columns' next state into the current state
__global__ void k_bdot(const double *__restrict__ p, const float *__restrict__ w, const double *__restrict__ sig2,
                       const Chunk *__restrict__ chunks, const int *__restrict__ prob_c0, int nrhs,
                       double *__restrict__ partial, BState st) {
    __shared__ double red[kRedThreads];
    const Chunk c = chunks[blockIdx.x];
    // the state move comes first: a problem that has just stopped must be seen
    // as stopped by the next kernels of this iteration
    if (c.first && threadIdx.x < nrhs) {
        const int col = c.prob * nrhs + threadIdx.x;
        st.rho[col] = st.rho_next[col];
        st.active[col] = st.active_next[col];
    }
    if (c.first && threadIdx.x == 0) st.prob_active[c.prob] = st.prob_active_next[c.prob];
    if (st.prob_active_next[c.prob] == 0) return;
    const double s = sig2[c.prob];
    chunk_col_sums(
        c, nrhs,
        [&](int64_t row, int j) {
            const int64_t t = row * nrhs + j;
            return p[t] * ((double)w[t] + s * p[t]);
        },
        partial + (size_t)blockIdx.x * nrhs, red);
}

__global__ void k_bupdate_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                             const float *__restrict__ w, const double *__restrict__ sig2,
                             const Chunk *__restrict__ chunks, const int *__restrict__ prob_c0,
                             const int *__restrict__ prob_nc, int nrhs, const double *__restrict__ pw_partial,
                             double *__restrict__ partial, BState st) {
    __shared__ double red[kRedThreads];
    __shared__ double s_alpha[64];
    const Chunk c = chunks[blockIdx.x];
    if (st.prob_active[c.prob] == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c0 = prob_c0[c.prob], nc = prob_nc[c.prob];
    for (int j = warp; j < nrhs; j += nw) {
        const double pw = warp_prob_sum(pw_partial, c0, nc, nrhs, j, lane);
        if (lane == 0) {
            const int col = c.prob * nrhs + j;
            double a = 0.0;
            if (st.active[col]) {
                if (pw > 0.0)
                    a = st.rho[col] / pw;
                else if (c.first) {
                    atomicOr(st.breakdown, 1);
                    st.bd[col] = 1;
                }
            }
            s_alpha[j] = a;
        }
    }
    __syncthreads();
    const double s = sig2[c.prob];
    for (int64_t t = (int64_t)c.row0 * nrhs + threadIdx.x; t < (int64_t)c.row1 * nrhs; t += blockDim.x) {
        const double a = s_alpha[t % nrhs];
        if (a != 0.0) {
            const double pv = p[t];
            x[t] += a * pv;
            r[t] -= a * ((double)w[t] + s * pv);
        }
    }
    __syncthreads();
    chunk_col_sums(
        c, nrhs, [&](int64_t row, int j) { const double v = r[row * nrhs + j]; return v * v; },
        partial + (size_t)blockIdx.x * nrhs, red);
}

// r: the new direction's source (z = P^{-1} r with preconditioners, else r);
// rz_partial: chunk partials of r^T z (NULL: rho is ||r||^2)
__global__ void k_bupdate_p(double *__restrict__ p, float *__restrict__ p32, float *__restrict__ w,
                            const double *__restrict__ r, const BatchProb *__restrict__ probs,
                            const Chunk *__restrict__ chunks, const int *__restrict__ prob_c0,
                            const int *__restrict__ prob_nc, int nrhs, const double *__restrict__ rr_partial,
                            const double *__restrict__ rz_partial, BState st) {
    __shared__ double s_beta[64];
    __shared__ int s_act[64];
    const Chunk c = chunks[blockIdx.x];
    if (st.prob_active[c.prob] == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c0 = prob_c0[c.prob], nc = prob_nc[c.prob];
    for (int j = warp; j < nrhs; j += nw) {
        const double rr = warp_prob_sum(rr_partial, c0, nc, nrhs, j, lane);
        const double rz = rz_partial ? warp_prob_sum(rz_partial, c0, nc, nrhs, j, lane) : rr;
        if (lane == 0) {
            const int col = c.prob * nrhs + j;
            const int act = st.active[col];
            const double rho = st.rho[col];
            const int still = act && !st.bd[col] && rr > st.thr2[col];
            s_beta[j] = act ? (rho > 0.0 ? rz / rho : 0.0) : 0.0;
            s_act[j] = still;
            if (c.first) {
                st.rho_next[col] = act ? rz : rho;
                if (act) st.rr[col] = rr;
                st.active_next[col] = still;
                if (act) st.iters[col] += 1;
            }
        }
    }
    __syncthreads();
    if (c.first && threadIdx.x == 0) {
        int n = 0;
        for (int j = 0; j < nrhs; ++j) n += s_act[j];
        st.prob_active_next[c.prob] = n;
    }
    const float s2 = probs[c.prob].s2;
    for (int64_t t = (int64_t)c.row0 * nrhs + threadIdx.x; t < (int64_t)c.row1 * nrhs; t += blockDim.x) {
        const int j = (int)(t % nrhs);
        double pv = p[t];
        if (s_act[j]) {
            pv = r[t] + s_beta[j] * pv;
            p[t] = pv;
        }
        const float pf = (float)pv;
        p32[t] = pf;
        w[t] = s2 * pf;
    }
}

__global__ void k_to_f32_diag(const double *__restrict__ p, float *__restrict__ p32, float *__restrict__ w,
                              const BatchProb *__restrict__ probs, const Chunk *__restrict__ chunks, int nrhs) {
    const Chunk c = chunks[blockIdx.x];
    const float s2 = probs[c.prob].s2;
    for (int64_t t = (int64_t)c.row0 * nrhs + threadIdx.x; t < (int64_t)c.row1 * nrhs; t += blockDim.x) {
        const float pf = (float)p[t];
        p32[t] = pf;
        w[t] = s2 * pf;
    }
}

__global__ void k_residual_slice(const double *__restrict__ B, const double *__restrict__ Y,
                                 const double *__restrict__ X, double sigma2, int64_t n, double *__restrict__ R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        R[t] = B[t] - (Y[t] + sigma2 * X[t]);
}

// p_j^T (w_j + sigma2 p_j) per chunk (partials), w from FP64 scans
__global__ void k_chunk_pap(const double *__restrict__ P, const double *__restrict__ W,
                            const double *__restrict__ sig2, const Chunk *__restrict__ chunks, int nrhs,
                            double *__restrict__ partial) {
    __shared__ double red[kRedThreads];
    const Chunk c = chunks[blockIdx.x];
    const double sg = sig2[c.prob];
    chunk_col_sums(
        c, nrhs,
        [&](int64_t row, int j) {
            const int64_t t = row * nrhs + j;
            return P[t] * (W[t] + sg * P[t]);
        },
        partial + (size_t)blockIdx.x * nrhs, red);
}

// p_j = r_j on the columns flagged in bd (a CG restart)
__global__ void k_brestart(double *__restrict__ P, const double *__restrict__ R, const Chunk *__restrict__ chunks,
                           int nrhs, const int *__restrict__ bd) {
    const Chunk c = chunks[blockIdx.x];
    for (int64_t t = (int64_t)c.row0 * nrhs + threadIdx.x; t < (int64_t)c.row1 * nrhs; t += blockDim.x)
        if (bd[c.prob * nrhs + (int)(t % nrhs)]) P[t] = R[t];
}

// r_j^T z_j per chunk (partials), for active problems (gate: prob_active_next
// as the p-update of this iteration reads it)
__global__ void k_chunk_rz(const double *__restrict__ R, const double *__restrict__ Zv,
                           const Chunk *__restrict__ chunks, int nrhs, const int *__restrict__ prob_active,
                           double *__restrict__ partial) {
    __shared__ double red[kRedThreads];
    const Chunk c = chunks[blockIdx.x];
    if (prob_active && prob_active[c.prob] == 0) return;
    chunk_col_sums(
        c, nrhs, [&](int64_t row, int j) { return R[row * nrhs + j] * Zv[row * nrhs + j]; },
        partial + (size_t)blockIdx.x * nrhs, red);
}

// squared column norms per chunk (partials; summed per problem by k_prob_sums)
__global__ void k_chunk_norms2(const double *__restrict__ A, const Chunk *__restrict__ chunks, int nrhs,
                               double *__restrict__ partial) {
    __shared__ double red[kRedThreads];
    const Chunk c = chunks[blockIdx.x];
    chunk_col_sums(
        c, nrhs, [&](int64_t row, int j) { const double v = A[row * nrhs + j]; return v * v; },
        partial + (size_t)blockIdx.x * nrhs, red);
}

// out[i * nrhs + j] = sum over problem i's chunks of partial[., j] (one warp each)
__global__ void k_prob_sums(const double *__restrict__ partial, const int *__restrict__ prob_c0,
                            const int *__restrict__ prob_nc, int n, int nrhs, double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)n * nrhs) return;
    const int i = (int)(w / nrhs), j = (int)(w % nrhs);
    const double t = warp_prob_sum(partial, prob_c0[i], prob_nc[i], nrhs, j, lane);
    if (lane == 0) out[w] = t;
}

double env_double_b(const char *name, double dflt) {
    const char *s = getenv(name);
    if (!s || !*s) return dflt;
    char *end = nullptr;
    double v = strtod(s, &end);
    return (end && end != s) ? v : dflt;
}

}  // namespace

struct Batch {
    std::vector<Plan *> plans;
    int n = 0, nrhs = 0, rpc = 0;
    int64_t rows = 0;
    std::vector<int64_t> voff;
    cudaStream_t stream = nullptr;
    BatchProb *probs = nullptr;
    BatchItem *long_items = nullptr, *all_items = nullptr;
    int n_long_items = 0, n_all_items = 0;
    // per variant (kBatchVariantKey order), its range of each list: [first, first + count)
    int long_first[kBatchVariants] = {}, long_count[kBatchVariants] = {};
    int all_first[kBatchVariants] = {}, all_count[kBatchVariants] = {};
    BatchSeg *segs = nullptr;
    int nseg = 0;
    Chunk *chunks = nullptr;
    int nchunk = 0;
    int *prob_c0 = nullptr, *prob_nc = nullptr;
    std::vector<int> h_prob_c0, h_prob_nc;
    float *agg = nullptr, *carry = nullptr;
    int *err = nullptr;
    std::vector<void *> owned;
};

static int batch_alloc(Batch *b, void **p, size_t bytes) {
    void *q = dev_alloc(bytes, b->stream);
    if (!q) {
        set_error("batch: device allocation of %zu bytes failed", bytes);
        return FGK_ERR_OOM;
    }
    b->owned.push_back(q);
    *p = q;
    return FGK_OK;
}

static void batch_release(Batch *b) {
    for (void *q : b->owned) dev_free(q, b->stream);
    b->owned.clear();
}

static int batch_product(Batch *b, const float *V, float *Y, const int *prob_active, cudaStream_t s) {
    BatchArgs A;
    A.probs = b->probs;
    A.segs = b->segs;
    A.nseg = b->nseg;
    A.V = V;
    A.Y = Y;
    A.nrhs = b->nrhs;
    A.agg = b->agg;
    A.carry = b->carry;
    A.prob_active = prob_active;
    A.err = b->err;
    if (b->n_long_items > 0) {
        A.items = b->long_items;
        for (int v = 0; v < kBatchVariants; ++v)
            if (b->long_count[v] > 0) FGK_TRY(launch_batch_scan<SCAN_AGG>(v, A, b->long_first[v], b->long_count[v], s));
        const int64_t nthr = (int64_t)b->nseg * 2 * b->nrhs * kMaxBatchNPT * 32;
        k_batch_carry<<<grid_for(nthr, 256), 256, 0, s>>>(A);
        FGK_LAUNCH_CHECK();
    }
    if (b->n_all_items > 0) {
        A.items = b->all_items;
        for (int v = 0; v < kBatchVariants; ++v)
            if (b->all_count[v] > 0) FGK_TRY(launch_batch_scan<SCAN_OUT>(v, A, b->all_first[v], b->all_count[v], s));
    }
    return FGK_OK;
}

}  // namespace fgk

using namespace fgk;

struct fgk_batch_s : public fgk::Batch {};

extern "C" {

int fgk_batch_create(const fgk_handle *handles, int n, int nrhs, int rhs_per_cta, fgk_stream_t stream,
                     fgk_batch *out) {
    clear_error();
    if (out) *out = nullptr;
    if (!handles || !out || n < 1 || nrhs < 1 || nrhs > 64) {
        set_error("fgk_batch_create: need handles, out, n >= 1 and 1 <= nrhs <= 64");
        return FGK_ERR_INVALID;
    }
    for (int i = 0; i < n; ++i)
        if (!handles[i] || handles[i]->d > 2 || handles[i]->P > 3) {
            set_error("fgk_batch_create: handle %d is NULL, has d > 2 or nu > 5/2 (batches take d <= 2, "
                      "nu <= 5/2)", i);
            return FGK_ERR_INVALID;
        }
    fgk_batch_s *b = new fgk_batch_s();
    b->n = n;
    b->nrhs = nrhs;
    b->rpc = (rhs_per_cta < 1 || rhs_per_cta > nrhs) ? nrhs : rhs_per_cta;
    b->stream = (cudaStream_t)stream;
    std::vector<BatchProb> probs(n);
    std::vector<BatchItem> longs, all;
    std::vector<BatchSeg> segs;
    std::vector<Chunk> chunks;
    int64_t row = 0, aggf = 0;
    for (int i = 0; i < n; ++i) {
        Plan *p = handles[i];
        b->plans.push_back(p);
        b->voff.push_back(row);
        const int noff = p->d - 1;
        const int kind = (p->P == 1 || noff == 0) ? FGK_L1 : p->kind;
        BatchProb &pr = probs[i];
        pr.lv_q = p->lv_q;
        pr.lv_dl = p->lv_dl32;
        pr.lv_off = p->lv_off32;
        pr.N = p->N;
        pr.ldN = p->ldN;
        pr.nlev = p->nlev;
        pr.variant = variant_key(p->P, noff, kind);
        pr.s2 = (float)p->s2;
        pr.voff = row;
        pr.agg_off = aggf;
        // per long slot: 2 directions x nrhs x (passes x aggregate) <= 2 x nrhs x 32 floats
        aggf += (int64_t)p->n_long * 2 * nrhs * 32;
        for (const WorkItem &w : p->items_host) {
            for (int r0 = 0; r0 < nrhs; r0 += b->rpc) {
                BatchItem bi{w, i, r0, std::min(nrhs, r0 + b->rpc)};
                if (w.agg >= 0) longs.push_back(bi);
                all.push_back(bi);
            }
        }
        for (size_t k = 0; k + 1 < p->long_seg_host.size(); k += 2)
            segs.push_back(BatchSeg{i, p->long_seg_host[k], p->long_seg_host[k + 1], 0});
        b->h_prob_c0.push_back((int)chunks.size());
        for (int64_t r0 = 0; r0 < p->N; r0 += kChunkRows)
            chunks.push_back(Chunk{i, (int32_t)(row + r0), (int32_t)(row + std::min<int64_t>(p->N, r0 + kChunkRows)),
                                   r0 == 0 ? 1 : 0});
        b->h_prob_nc.push_back((int)chunks.size() - b->h_prob_c0.back());
        row += p->N;
    }
    // group each list by variant (stable: each problem's items keep their order)
    auto group = [&](std::vector<BatchItem> &list, int *first, int *count) -> bool {
        std::vector<BatchItem> out;
        out.reserve(list.size());
        for (int v = 0; v < kBatchVariants; ++v) {
            first[v] = (int)out.size();
            for (const BatchItem &bi : list)
                if (probs[bi.prob].variant == kBatchVariantKey[v]) out.push_back(bi);
            count[v] = (int)out.size() - first[v];
        }
        const bool all_placed = out.size() == list.size();
        list.swap(out);
        return all_placed;
    };
    if (!group(longs, b->long_first, b->long_count) || !group(all, b->all_first, b->all_count)) {
        set_error("fgk_batch_create: a problem's scan variant has no batched kernel (internal)");
        delete b;
        return FGK_ERR_INTERNAL;
    }
    b->rows = row;
    b->n_long_items = (int)longs.size();
    b->n_all_items = (int)all.size();
    b->nseg = (int)segs.size();
    b->nchunk = (int)chunks.size();
    int rc = FGK_OK;
    cudaStream_t s = b->stream;
    auto up = [&](void **dst, const void *src, size_t bytes) -> int {
        FGK_TRY(batch_alloc(b, dst, bytes > 0 ? bytes : 16));
        if (bytes) FGK_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s));
        return FGK_OK;
    };
    do {
        if ((rc = up((void **)&b->probs, probs.data(), sizeof(BatchProb) * probs.size()))) break;
        if ((rc = up((void **)&b->long_items, longs.data(), sizeof(BatchItem) * longs.size()))) break;
        if ((rc = up((void **)&b->all_items, all.data(), sizeof(BatchItem) * all.size()))) break;
        if ((rc = up((void **)&b->segs, segs.data(), sizeof(BatchSeg) * segs.size()))) break;
        if ((rc = up((void **)&b->chunks, chunks.data(), sizeof(Chunk) * chunks.size()))) break;
        if ((rc = up((void **)&b->prob_c0, b->h_prob_c0.data(), sizeof(int) * n))) break;
        if ((rc = up((void **)&b->prob_nc, b->h_prob_nc.data(), sizeof(int) * n))) break;
        if ((rc = batch_alloc(b, (void **)&b->agg, sizeof(float) * (size_t)std::max<int64_t>(aggf, 16)))) break;
        if ((rc = batch_alloc(b, (void **)&b->carry, sizeof(float) * (size_t)std::max<int64_t>(aggf, 16)))) break;
        if ((rc = batch_alloc(b, (void **)&b->err, 16))) break;
        if (cudaMemsetAsync(b->err, 0, 16, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("fgk_batch_create: CUDA error while uploading the batch");
            rc = FGK_ERR_CUDA;
        }
    } while (0);
    if (rc) {
        batch_release(b);
        delete b;
        return rc;
    }
    *out = b;
    return FGK_OK;
}

int fgk_batch_destroy(fgk_batch b) {
    clear_error();
    if (!b) return FGK_OK;
    batch_release(b);
    cudaStreamSynchronize(b->stream);
    delete b;
    return FGK_OK;
}

int fgk_batch_layout(fgk_batch b, int64_t *row_offsets) {
    clear_error();
    if (!b || !row_offsets) {
        set_error("fgk_batch_layout: NULL argument");
        return FGK_ERR_INVALID;
    }
    for (int i = 0; i < b->n; ++i) row_offsets[i] = b->voff[i];
    row_offsets[b->n] = b->rows;
    return FGK_OK;
}

int fgk_batch_matvec_q(fgk_batch b, const float *Vq, float *Yq, fgk_stream_t stream) {
    clear_error();
    if (!b || !Vq || !Yq) {
        set_error("fgk_batch_matvec_q: NULL argument");
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_batch_diag<<<b->nchunk, 256, 0, s>>>(Vq, Yq, b->chunks, b->probs, b->nrhs);
    FGK_LAUNCH_CHECK();
    return batch_product(b, Vq, Yq, nullptr, s);
}

static int batch_cg(fgk_batch b, const fgk_precond *pch, const double *const *y, const double *sigma2, double tol,
                    int maxit, double *const *alpha, fgk_cg_info *info, fgk_stream_t stream) {
    clear_error();
    if (!b || !y || !sigma2 || !alpha || !(tol > 0.0) || maxit < 1) {
        set_error("fgk_batch_cg_solve: bad argument");
        return FGK_ERR_INVALID;
    }
    const int n = b->n, nrhs = b->nrhs, C = n * nrhs;
    for (int i = 0; i < n; ++i)
        if (!y[i] || !alpha[i] || !(sigma2[i] >= 0.0) || !std::isfinite(sigma2[i])) {
            set_error("fgk_batch_cg_solve: problem %d has a NULL vector or a bad sigma2", i);
            return FGK_ERR_INVALID;
        }
    std::vector<Precond *> pcs;
    if (pch) {
        for (int i = 0; i < n; ++i) {
            Precond *pc = pc_of(pch[i]);
            if (!pc || pc_plan(pc) != b->plans[i] || pc_sigma2(pc) != sigma2[i]) {
                set_error("fgk_batch_cg_solve_pc: preconditioner %d is NULL or was built for another plan or sigma2",
                          i);
                return FGK_ERR_INVALID;
            }
            FGK_TRY(pc_reserve(pc, nrhs, (cudaStream_t)stream));
            pcs.push_back(pc);
        }
    }
    const bool pcon = !pcs.empty();
    cudaStream_t us = (cudaStream_t)stream;
    cudaStream_t s;
    FGK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t ev;
    FGK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FGK_CUDA(cudaEventRecord(ev, us));
    FGK_CUDA(cudaStreamWaitEvent(s, ev, 0));
    const size_t vec = (size_t)b->rows * nrhs;
    std::vector<void *> mine;
    auto take = [&](size_t bytes) -> void * {
        void *q = dev_alloc(bytes > 0 ? bytes : 16, s);
        if (q) mine.push_back(q);
        return q;
    };
    double *Bv = (double *)take(vec * 8), *X = (double *)take(vec * 8), *Rv = (double *)take(vec * 8);
    double *Pv = (double *)take(vec * 8), *W64 = (double *)take(vec * 8);
    float *P32 = (float *)take(vec * 4), *W32 = (float *)take(vec * 4);
    double *pw_part = (double *)take((size_t)b->nchunk * nrhs * 8), *rr_part = (double *)take((size_t)b->nchunk * nrhs * 8);
    double *sig2 = (double *)take(n * 8), *nrm = (double *)take((size_t)C * 8);
    double *nrm_part = (double *)take((size_t)b->nchunk * nrhs * 8);
    double *Zv = pcon ? (double *)take(vec * 8) : nullptr;
    double *rz_part = pcon ? (double *)take((size_t)b->nchunk * nrhs * 8) : nullptr;
    BState st;
    st.rr = (double *)take(C * 8);
    st.rho = (double *)take(C * 8);
    st.rho_next = (double *)take(C * 8);
    st.thr2 = (double *)take(C * 8);
    st.active = (int *)take(C * 4);
    st.active_next = (int *)take(C * 4);
    st.iters = (int *)take(C * 4);
    st.prob_active = (int *)take(n * 4);
    st.prob_active_next = (int *)take(n * 4);
    st.bd = (int *)take(C * 4);
    st.breakdown = (int *)take(16);
    int rc = FGK_OK;
    for (void *q : mine)
        if (!q) rc = FGK_ERR_OOM;
    std::vector<double> bnorm(C), rnorm(C), rho_ref(C), hrho(C), hthr2(C), hnorm(C), hrr(C), hrz(C);
    std::vector<int> hact(C), hiters(C, 0), confirmed(C, 0), hpa(n), last_repl(n, 0);
    // gap[i]: min_gap[i] while problem i's last replacement found a true
    // residual within twice the recursive one, else 0 (the FP32 recursion was
    // drifting: replace at every drop by delta)
    std::vector<int> min_gap(n, 0), gap(n, 0), restarts(n, 0), hbd(C, 0);
    constexpr int kMaxRestarts = 8;
    int limit_prob = -1;
    int iters_total = 0, refinements = 0, n32 = 0, n64 = 0;
    bool converged = false, breakdown = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t graph_nodes = 0;
    const double delta = env_double_b("FGK_MIXED_DELTA", pcon ? 1e-3 : 0.5);
    const int check_every = 8;

    // squared column norms of every problem's slice of A into hnorm (one sync)
    auto all_norms = [&](const double *A) -> int {
        k_chunk_norms2<<<b->nchunk, kRedThreads, 0, s>>>(A, b->chunks, nrhs, nrm_part);
        FGK_LAUNCH_CHECK();
        k_prob_sums<<<grid_for((int64_t)C * 32, 256), 256, 0, s>>>(nrm_part, b->prob_c0, b->prob_nc, n, nrhs, nrm);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(hnorm.data(), nrm, (size_t)C * 8, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        return FGK_OK;
    };
    // FP64 true residuals of the listed problems into Rv's slices (the other
    // slices keep their last residual); norms of the listed ones into rnorm
    auto residuals = [&](const std::vector<int> &list) -> int {
        for (int i : list) {
            Plan *p = b->plans[i];
            const size_t o = (size_t)b->voff[i] * nrhs, m = (size_t)p->N * nrhs;
            FGK_TRY(mvm_q_f64(p, X + o, nrhs, W64 + o, s, nullptr));
            k_residual_slice<<<256, 256, 0, s>>>(Bv + o, W64 + o, X + o, sigma2[i], (int64_t)m, Rv + o);
            FGK_LAUNCH_CHECK();
            ++refinements;
            ++n64;
        }
        FGK_TRY(all_norms(Rv));
        for (int i : list)
            for (int j = 0; j < nrhs; ++j) rnorm[i * nrhs + j] = std::sqrt(hnorm[i * nrhs + j]);
        return FGK_OK;
    };
    // z = P^{-1} r for every problem and r^T z per column into hrz (one sync)
    auto precondition = [&]() -> int {
        for (int i = 0; i < n; ++i) {
            const size_t o = (size_t)b->voff[i] * nrhs;
            FGK_TRY(pc_apply(pcs[i], Rv + o, nrhs, Zv + o, nullptr, s));
        }
        k_chunk_rz<<<b->nchunk, kRedThreads, 0, s>>>(Rv, Zv, b->chunks, nrhs, nullptr, nrm_part);
        FGK_LAUNCH_CHECK();
        k_prob_sums<<<grid_for((int64_t)C * 32, 256), 256, 0, s>>>(nrm_part, b->prob_c0, b->prob_nc, n, nrhs, nrm);
        FGK_LAUNCH_CHECK();
        FGK_CUDA(cudaMemcpyAsync(hrz.data(), nrm, (size_t)C * 8, cudaMemcpyDeviceToHost, s));
        FGK_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) FGK_TRY(pc_check(pcs[i], s));
        return FGK_OK;
    };
    auto upload_state = [&]() -> int {
        std::vector<int> pa(n, 0);
        for (int c = 0; c < C; ++c) pa[c / nrhs] += hact[c];
        FGK_CUDA(cudaMemcpyAsync(st.rr, hrr.data(), C * 8, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.rho, hrho.data(), C * 8, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.rho_next, hrho.data(), C * 8, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.thr2, hthr2.data(), C * 8, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.active, hact.data(), C * 4, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.active_next, hact.data(), C * 4, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.iters, hiters.data(), C * 4, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.prob_active, pa.data(), n * 4, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(st.prob_active_next, pa.data(), n * 4, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaStreamSynchronize(s));  // the host vectors are reused
        return FGK_OK;
    };

    do {
        if (rc) break;
        // right-hand sides into the packed q order; sigma2 per problem
        for (int i = 0; i < n && !rc; ++i) {
            rc = to_q_order(b->plans[i], y[i], Bv + (size_t)b->voff[i] * nrhs, nrhs, 8, s);
        }
        if (rc) break;
        FGK_CUDA(cudaMemcpyAsync(sig2, sigma2, n * 8, cudaMemcpyHostToDevice, s));
        FGK_CUDA(cudaMemsetAsync(X, 0, vec * 8, s));
        FGK_CUDA(cudaMemcpyAsync(Rv, Bv, vec * 8, cudaMemcpyDeviceToDevice, s));
        FGK_CUDA(cudaMemcpyAsync(Pv, Bv, vec * 8, cudaMemcpyDeviceToDevice, s));
        FGK_CUDA(cudaMemsetAsync(st.breakdown, 0, 16, s));
        FGK_CUDA(cudaMemsetAsync(st.bd, 0, (size_t)C * 4, s));
        if ((rc = all_norms(Bv))) break;
        for (int c = 0; c < C; ++c) bnorm[c] = std::sqrt(hnorm[c]);
        rnorm = bnorm;
        if (pcon) {  // p = z = P^{-1} b, rho = b^T z
            if ((rc = precondition())) break;
            FGK_CUDA(cudaMemcpyAsync(Pv, Zv, vec * 8, cudaMemcpyDeviceToDevice, s));
        }
        for (int c = 0; c < C; ++c) {
            hrr[c] = rnorm[c] * rnorm[c];
            hrho[c] = pcon ? hrz[c] : hrr[c];
            rho_ref[c] = hrr[c];
            const double t = 0.5 * tol * bnorm[c];
            hthr2[c] = t * t;
            confirmed[c] = rnorm[c] <= tol * bnorm[c];
            hact[c] = !confirmed[c];
        }
        if ((rc = upload_state())) break;
        // the FP32 copy of p and the product's starting point; timed warm-up products
        k_to_f32_diag<<<b->nchunk, 256, 0, s>>>(Pv, P32, W32, b->probs, b->chunks, nrhs);
        FGK_LAUNCH_CHECK();
        cudaEvent_t t0, t1;
        FGK_CUDA(cudaEventCreate(&t0));
        FGK_CUDA(cudaEventCreate(&t1));
        // Spacing of each problem's replacements: its FP64 over its FP32 product
        // time (each timed on its own), the rule the single-problem solve
        // uses, so a problem converges in the batch as it does alone.  It
        // applies only while the recursion tracks the true residual (see gap).
        FGK_CUDA(cudaEventRecord(t0, s));
        if ((rc = batch_product(b, P32, W32, nullptr, s))) break;  // warm-up
        FGK_CUDA(cudaEventRecord(t1, s));
        FGK_CUDA(cudaEventSynchronize(t1));
        for (int i = 0; i < n && !rc; ++i) {
            Plan *p = b->plans[i];
            const size_t o = (size_t)b->voff[i] * nrhs;
            float ms32 = 0.f, ms64 = 0.f;
            FGK_CUDA(cudaEventRecord(t0, s));
            if ((rc = mvm_q_f32(p, P32 + o, nrhs, W32 + o, s, nullptr))) break;
            FGK_CUDA(cudaEventRecord(t1, s));
            FGK_CUDA(cudaEventSynchronize(t1));
            FGK_CUDA(cudaEventElapsedTime(&ms32, t0, t1));
            FGK_CUDA(cudaEventRecord(t0, s));
            if ((rc = mvm_q_f64(p, Pv + o, nrhs, W64 + o, s, nullptr))) break;
            FGK_CUDA(cudaEventRecord(t1, s));
            FGK_CUDA(cudaEventSynchronize(t1));
            FGK_CUDA(cudaEventElapsedTime(&ms64, t0, t1));
            min_gap[i] = ms32 > 0.f ? (int)std::min(1e6, std::ceil((double)ms64 / ms32)) : 0;
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (rc) break;
        k_to_f32_diag<<<b->nchunk, 256, 0, s>>>(Pv, P32, W32, b->probs, b->chunks, nrhs);
        FGK_LAUNCH_CHECK();
        {
            const uint64_t c0 = kernel_launch_count();
            FGK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int crc = batch_product(b, P32, W32, st.prob_active_next, s);
            if (!crc) {
                k_bdot<<<b->nchunk, kRedThreads, 0, s>>>(Pv, W32, sig2, b->chunks, b->prob_c0, nrhs, pw_part, st);
                add_kernel_launches(1);
                k_bupdate_xr<<<b->nchunk, kRedThreads, 0, s>>>(X, Rv, Pv, W32, sig2, b->chunks, b->prob_c0,
                                                               b->prob_nc, nrhs, pw_part, rr_part, st);
                add_kernel_launches(1);
                if (pcon) {
                    for (int i = 0; i < n && !crc; ++i) {
                        const size_t o = (size_t)b->voff[i] * nrhs;
                        crc = pc_apply(pcs[i], Rv + o, nrhs, Zv + o, nullptr, s, st.prob_active + i);
                    }
                    k_chunk_rz<<<b->nchunk, kRedThreads, 0, s>>>(Rv, Zv, b->chunks, nrhs, st.prob_active, rz_part);
                    add_kernel_launches(1);
                }
                k_bupdate_p<<<b->nchunk, kRedThreads, 0, s>>>(Pv, P32, W32, pcon ? Zv : Rv, b->probs, b->chunks,
                                                              b->prob_c0, b->prob_nc, nrhs, rr_part,
                                                              pcon ? rz_part : nullptr, st);
                add_kernel_launches(1);
            }
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            graph_nodes = kernel_launch_count() - c0;
            add_kernel_launches(-(int64_t)graph_nodes);
            if (crc) {
                rc = crc;
                break;
            }
            FGK_CUDA(ce);
            FGK_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
        }
        std::vector<int> snap_act(C), snap_iters(C);
        std::vector<double> snap_rho(C), snap_rr(C);
        int hbreak = 0;
        while (true) {
            bool all = true;
            for (int c = 0; c < C; ++c) all = all && confirmed[c];
            if (all) {
                converged = true;
                break;
            }
            if (iters_total >= maxit) break;
            const int k = std::min(check_every, maxit - iters_total);
            for (int it = 0; it < k; ++it) FGK_CUDA(cudaGraphLaunch(gexec, s));
            add_kernel_launches((int64_t)graph_nodes * k);
            FGK_CUDA(cudaMemcpyAsync(snap_act.data(), st.active_next, C * 4, cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaMemcpyAsync(snap_rho.data(), st.rho_next, C * 8, cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaMemcpyAsync(snap_rr.data(), st.rr, C * 8, cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaMemcpyAsync(snap_iters.data(), st.iters, C * 4, cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaMemcpyAsync(&hbreak, st.breakdown, 4, cudaMemcpyDeviceToHost, s));
            FGK_CUDA(cudaStreamSynchronize(s));
            const int before = *std::max_element(hiters.begin(), hiters.end());
            hiters = snap_iters;
            const int after = *std::max_element(hiters.begin(), hiters.end());
            iters_total += after - before;
            n32 += after - before;
            // FP32 breakdowns: decide with FP64 scans; restart the column if
            // p^T A p is positive there, else stop with a breakdown
            std::vector<int> broken(n, 0);
            if (hbreak) {
                FGK_CUDA(cudaMemcpyAsync(hbd.data(), st.bd, (size_t)C * 4, cudaMemcpyDeviceToHost, s));
                FGK_CUDA(cudaStreamSynchronize(s));
                for (int c = 0; c < C; ++c)
                    if (hbd[c]) broken[c / nrhs] = 1;
                for (int i = 0; i < n && !rc; ++i)
                    if (broken[i]) {
                        const size_t o = (size_t)b->voff[i] * nrhs;
                        rc = mvm_q_f64(b->plans[i], Pv + o, nrhs, W64 + o, s, nullptr);
                        ++n64;
                    }
                if (rc) break;
                k_chunk_pap<<<b->nchunk, kRedThreads, 0, s>>>(Pv, W64, sig2, b->chunks, nrhs, nrm_part);
                FGK_LAUNCH_CHECK();
                k_prob_sums<<<grid_for((int64_t)C * 32, 256), 256, 0, s>>>(nrm_part, b->prob_c0, b->prob_nc, n, nrhs,
                                                                         nrm);
                FGK_LAUNCH_CHECK();
                FGK_CUDA(cudaMemcpyAsync(hnorm.data(), nrm, (size_t)C * 8, cudaMemcpyDeviceToHost, s));
                FGK_CUDA(cudaStreamSynchronize(s));
                for (int c = 0; c < C; ++c)
                    if (hbd[c] && !(hnorm[c] > 0.0)) breakdown = true;
                for (int i = 0; i < n; ++i)
                    if (broken[i] && ++restarts[i] > kMaxRestarts && limit_prob < 0) limit_prob = i;
                if (limit_prob >= 0) breakdown = true;
                if (breakdown) break;
            }
            bool any = false;
            std::vector<int> todo;
            for (int i = 0; i < n; ++i) {
                bool claims = false, dropped = false;
                for (int j = 0; j < nrhs; ++j) {
                    const int c = i * nrhs + j;
                    if (confirmed[c]) continue;
                    if (!snap_act[c]) claims = true;
                    if (snap_rr[c] <= delta * delta * rho_ref[c]) dropped = true;
                }
                if (broken[i] || claims || (dropped && iters_total - last_repl[i] >= gap[i])) todo.push_back(i);
            }
            if (todo.empty()) continue;
            for (int c = 0; c < C; ++c) {
                hrho[c] = snap_rho[c];
                hrr[c] = snap_rr[c];
                hact[c] = snap_act[c];
            }
            if ((rc = residuals(todo))) break;
            if (pcon && (rc = precondition())) break;  // z and r^T z of the replaced residuals
            // restart p = z (z = r without preconditioners) on the columns whose
            // direction no longer fits the replaced residual (as fgk_cg_solve):
            // every replaced column with a preconditioner; without one, an FP32
            // breakdown, a column that had stopped, or a true residual above
            // twice the recursive one
            std::vector<int> rs(C, 0);
            bool any_rs = false;
            for (int i : todo) {
                last_repl[i] = iters_total;
                bool drift = false;
                for (int j = 0; j < nrhs; ++j) {
                    const int c = i * nrhs + j;
                    const bool dj = !confirmed[c] && rnorm[c] > 2.0 * std::sqrt(snap_rr[c]);
                    drift = drift || dj;
                    rs[c] = !confirmed[c] && (pcon || (hbreak && hbd[c]) || !snap_act[c] || dj) &&
                            !(rnorm[c] <= tol * bnorm[c]);
                    any_rs = any_rs || rs[c];
                }
                gap[i] = drift ? 0 : min_gap[i];
            }
            if (any_rs) {
                FGK_CUDA(cudaMemcpyAsync(st.bd, rs.data(), (size_t)C * 4, cudaMemcpyHostToDevice, s));
                k_brestart<<<b->nchunk, 256, 0, s>>>(Pv, pcon ? Zv : Rv, b->chunks, nrhs, st.bd);
                FGK_LAUNCH_CHECK();
                k_to_f32_diag<<<b->nchunk, 256, 0, s>>>(Pv, P32, W32, b->probs, b->chunks, nrhs);
                FGK_LAUNCH_CHECK();
            }
            if (any_rs || hbreak) {
                FGK_CUDA(cudaMemsetAsync(st.bd, 0, (size_t)C * 4, s));
                FGK_CUDA(cudaMemsetAsync(st.breakdown, 0, 16, s));
                FGK_CUDA(cudaStreamSynchronize(s));  // rs is a host vector
            }
            for (int i : todo) {
                for (int j = 0; j < nrhs; ++j) {
                    const int c = i * nrhs + j;
                    if (!confirmed[c] && rnorm[c] <= tol * bnorm[c]) confirmed[c] = 1;
                    hact[c] = !confirmed[c];
                    if (!confirmed[c]) {
                        hrr[c] = rnorm[c] * rnorm[c];
                        hrho[c] = pcon ? hrz[c] : hrr[c];
                        rho_ref[c] = hrr[c];
                    }
                }
                any = true;
            }
            if (rc) break;
            if (any && (rc = upload_state())) break;
        }
        if (rc) break;
        for (int i = 0; i < n && !rc; ++i)
            rc = from_q_order(b->plans[i], X + (size_t)b->voff[i] * nrhs, alpha[i], nrhs, 8, s);
        if (rc) break;
        FGK_CUDA(cudaStreamSynchronize(s));
    } while (0);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (void *q : mine) dev_free(q, s);
    cudaStreamSynchronize(s);
    cudaEventDestroy(ev);
    cudaStreamDestroy(s);
    if (info) {
        for (int i = 0; i < n; ++i) {
            double mx = 0.0;
            int it = 0;
            for (int j = 0; j < nrhs; ++j) {
                const int c = i * nrhs + j;
                const double r = bnorm[c] > 0 ? rnorm[c] / bnorm[c] : 0.0;
                mx = std::max(mx, r);
                it = std::max(it, hiters[c]);
                if (info[i].true_resid) info[i].true_resid[j] = r;
            }
            info[i].iterations = it;
            info[i].refinements = refinements;
            info[i].mvm_f32 = n32;
            info[i].mvm_f64 = n64;
            info[i].max_true_resid = mx;
            info[i].restarts = restarts[i];
            info[i].fp64_switch = 0;
        }
    }
    if (rc) return rc;
    if (breakdown && limit_prob >= 0) {
        set_error("fgk_batch_cg_solve: problem %d met p^T A p <= 0 with FP32 scans more than %d times; solve it "
                  "on its own (fgk_cg_solve continues with FP64 scans)",
                  limit_prob, kMaxRestarts);
        return FGK_ERR_BREAKDOWN;
    }
    if (breakdown) {
        set_error("fgk_batch_cg_solve: p^T A p <= 0 met; a system is not positive definite");
        return FGK_ERR_BREAKDOWN;
    }
    if (!converged) {
        set_error("fgk_batch_cg_solve: tolerance not reached within maxit = %d iterations", maxit);
        return FGK_NOT_CONVERGED;
    }
    return FGK_OK;
}

int fgk_batch_cg_solve(fgk_batch b, const double *const *y, const double *sigma2, double tol, int maxit,
                       double *const *alpha, fgk_cg_info *info, fgk_stream_t stream) {
    return batch_cg(b, nullptr, y, sigma2, tol, maxit, alpha, info, stream);
}

int fgk_batch_cg_solve_pc(fgk_batch b, const fgk_precond *pcs, const double *const *y, const double *sigma2,
                          double tol, int maxit, double *const *alpha, fgk_cg_info *info, fgk_stream_t stream) {
    if (!pcs) {
        set_error("fgk_batch_cg_solve_pc: pcs must not be NULL");
        return FGK_ERR_INVALID;
    }
    return batch_cg(b, pcs, y, sigma2, tol, maxit, alpha, info, stream);
}

}  // extern "C"
