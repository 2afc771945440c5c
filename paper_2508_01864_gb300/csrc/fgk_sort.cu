// K0: canonicalise and scale the coordinates; K1: stable radix sort of each
// scaled coordinate.
//
// The method first sorts the data (Sec. 2.1: the CDFs are taken in increasing
// order after a sort; Sec. 2.2.3: the sort outputs are stored for reuse).
// Here every coordinate is scaled, x'_k = x_k * sqrt(2 nu) / ell_k
// (eq. scaled_kernel, one lengthscale per dimension), -0 is mapped to +0, and
// the scaled values are sorted with ties broken by the original index
// (a stable sort of the points in index order).
//
// The sort is a least-significant-digit radix sort over the 64-bit
// order-preserving image of the double (8 passes of 8-bit digits).  All
// digit histograms come from one read of the keys; each pass is one kernel
// in which a tile ranks its keys stably in shared memory, publishes its
// per-digit counts, and obtains the counts of all earlier tiles by a
// decoupled look-back over the published words.  Passes whose digit is the
// same for every key are skipped.  Every look-back wait is bounded; on expiry
// the kernel records DEV_TIMEOUT in the plan's error word and stops waiting.
#include <algorithm>
#include <cstdlib>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortThreads * kSortIPT;
constexpr int kSortWarps = kSortThreads / 32;
// bound on the look-back's spins on one predecessor tile; fgk_build takes a
// smaller one from FGK_SORT_SPIN_LIMIT (a test hook that makes the wait
// expire, so that the expiry path is exercised)
constexpr int kSpinLimit = 1 << 24;

constexpr uint32_t ST_AGG = 1u << 30;
constexpr uint32_t ST_PRE = 2u << 30;
constexpr uint32_t ST_VAL = (1u << 30) - 1;

__device__ __forceinline__ uint64_t order_key(double x) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// K0: x'_k = x_k * a_k (+0.0 folds -0 into +0); non-finite input or output
// sets *bad.  Writes SoA scaled coordinates in the caller's order.
__global__ void k_canon_scale(const double *__restrict__ X, int64_t N, int d, double a0, double a1, double a2,
                              double *__restrict__ xs0, double *__restrict__ xs1, double *__restrict__ xs2,
                              int *__restrict__ bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double *out[3] = {xs0, xs1, xs2};
    double a[3] = {a0, a1, a2};
    for (int k = 0; k < d; ++k) {
        double x = X[i * d + k];
        double y = x * a[k] + 0.0;
        if (!isfinite(x) || !isfinite(y)) atomicOr(bad, 1);
        out[k][i] = y;
    }
}

__global__ void k_make_keys(const double *__restrict__ xs, int64_t N, uint64_t *__restrict__ keys,
                            int32_t *__restrict__ vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    keys[i] = order_key(xs[i]);
    vals[i] = (int32_t)i;
}

// all eight digit histograms in one pass
__global__ void k_histograms(const uint64_t *__restrict__ keys, int64_t N, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
#pragma unroll
        for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
        uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// exclusive scan of each pass's histogram (one block of 256 threads)
__global__ void k_digit_offsets(const uint32_t *__restrict__ hist, uint32_t *__restrict__ offs) {
    __shared__ uint32_t s[256];
    for (int p = 0; p < 8; ++p) {
        uint32_t v = hist[p * 256 + threadIdx.x];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        offs[p * 256 + threadIdx.x] = s[threadIdx.x] - v;
        __syncthreads();
    }
}

// One LSD pass.  Tiles are taken in order from *tile_counter so that every
// tile a look-back waits on has already been started by a running CTA.
// Once a wait has expired (the error word is set) the CTAs that start later
// take no tile and return: every tile still looks back only at tiles taken
// before it, and the host abandons the sort.  A tile whose wait expired
// stops summing its predecessors, so its offsets are at most the true ones
// and its writes stay inside the output.
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout, int64_t N, int shift, const uint32_t *__restrict__ digit_off,
    uint32_t *__restrict__ status, uint32_t *__restrict__ tile_counter, int *__restrict__ err, int spin_limit) {
    __shared__ uint16_t cnt[kSortIPT][kSortWarps][256];  // per (round, warp, digit); later exclusive offsets
    __shared__ uint32_t tile_excl[256];
    __shared__ uint32_t s_tile;
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_stop = *((volatile int *)err) != 0;
        if (!s_stop) s_tile = atomicAdd(tile_counter, 1u);
    }
    for (int i = tid; i < kSortIPT * kSortWarps * 256; i += kSortThreads) (&cnt[0][0][0])[i] = 0;
    __syncthreads();
    if (s_stop) return;
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kSortTile;

    uint64_t key[kSortIPT];
    int32_t val[kSortIPT];
    uint32_t dig[kSortIPT];
    uint32_t lrank[kSortIPT];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + tid;
        bool ok = i < N;
        key[r] = ok ? kin[i] : 0;
        val[r] = ok ? vin[i] : 0;
        dig[r] = ok ? (uint32_t)((key[r] >> shift) & 255) : 0x1000u + lane;  // unique sentinel
        uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        lrank[r] = __popc(peers & lt_mask);
        if (ok && (peers & lt_mask) == 0) cnt[r][warp][dig[r]] = (uint16_t)__popc(peers);
    }
    __syncthreads();
    // exclusive offsets over (round, warp) per digit; thread = digit
    {
        uint32_t run = 0;
        for (int r = 0; r < kSortIPT; ++r)
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = cnt[r][w][tid];
                cnt[r][w][tid] = (uint16_t)run;
                run += c;
            }
        // publish this tile's count, then look back for the earlier tiles'
        uint32_t *st = status + (size_t)tile * 256;
        if (tile == 0) {
            __stcg(&st[tid], ST_PRE | run);
            tile_excl[tid] = 0;
        } else {
            __stcg(&st[tid], ST_AGG | run);
            uint32_t excl = 0;
            int64_t j = (int64_t)tile - 1;
            int spins = 0;
            while (j >= 0) {
                uint32_t w = *((volatile uint32_t *)(status + (size_t)j * 256 + tid));
                if ((w & ~ST_VAL) == 0) {
                    if (++spins > spin_limit) {
                        atomicExch(err, DEV_TIMEOUT);
                        break;
                    }
                    continue;
                }
                excl += w & ST_VAL;
                if ((w & ~ST_VAL) == ST_PRE) break;
                --j;
            }
            __threadfence();
            __stcg(&st[tid], ST_PRE | (excl + run));
            tile_excl[tid] = excl;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortIPT; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + tid;
        if (i < N) {
            uint32_t dg = dig[r];
            uint32_t dst = digit_off[dg] + tile_excl[dg] + cnt[r][warp][dg] + lrank[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
    }
}

__global__ void k_invert(const int32_t *__restrict__ perm, int64_t N, int32_t *__restrict__ rank) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) rank[perm[i]] = (int32_t)i;
}

__global__ void k_gather_f64(const double *__restrict__ src, const int32_t *__restrict__ idx, int64_t N,
                             double *__restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[idx[i]];
}

__global__ void k_gather_rows(const double *__restrict__ X, const int32_t *__restrict__ idx, int64_t N, int d,
                              double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t s = idx[i];
    for (int k = 0; k < d; ++k) out[i * d + k] = X[s * d + k];
}

}  // namespace

// Stable sort of one scaled coordinate: perm_out[position] = point.
static int radix_sort(Plan *p, const double *xs, int32_t *perm_out, cudaStream_t s) {
    const int64_t N = p->N;
    const int ntiles = (int)((N + kSortTile - 1) / kSortTile);
    size_t bytes = 2 * N * sizeof(uint64_t) + N * sizeof(int32_t) + 8 * 256 * 4 * 2 + 8 * 4 +
                   (size_t)ntiles * 256 * 4 + 256;
    char *w = (char *)dev_alloc(bytes, s);
    if (!w) {
        set_error("device allocation of %zu bytes for the sort failed", bytes);
        return FGK_ERR_OOM;
    }
    uint64_t *k0 = (uint64_t *)w;
    uint64_t *k1 = k0 + N;
    int32_t *v1 = (int32_t *)(k1 + N);
    uint32_t *hist = (uint32_t *)(v1 + N);
    uint32_t *offs = hist + 8 * 256;
    uint32_t *counters = offs + 8 * 256;
    uint32_t *status = counters + 8;
    int32_t *v0 = perm_out;  // ping-pong with the output buffer

    k_make_keys<<<grid_for(N, 256), 256, 0, s>>>(xs, N, k0, v0);
    FGK_LAUNCH_CHECK();
    FGK_CUDA(cudaMemsetAsync(hist, 0, 8 * 256 * 4, s));
    k_histograms<<<std::min<unsigned>(grid_for(N, 256), 1024u), 256, 0, s>>>(k0, N, hist);
    FGK_LAUNCH_CHECK();
    k_digit_offsets<<<1, 256, 0, s>>>(hist, offs);
    FGK_LAUNCH_CHECK();
    uint32_t hhost[8 * 256];
    FGK_CUDA(cudaMemcpyAsync(hhost, hist, sizeof(hhost), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaStreamSynchronize(s));

    uint64_t *kin = k0, *kout = k1;
    int32_t *vin = v0, *vout = v1;
    for (int pass = 0; pass < 8; ++pass) {
        bool trivial = false;
        for (int dg = 0; dg < 256; ++dg)
            if (hhost[pass * 256 + dg] == (uint32_t)N) trivial = true;
        if (trivial) continue;
        FGK_CUDA(cudaMemsetAsync(status, 0, (size_t)ntiles * 256 * 4, s));
        FGK_CUDA(cudaMemsetAsync(counters + pass, 0, 4, s));
        k_sort_pass<<<ntiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, N, 8 * pass, offs + pass * 256, status,
                                                     counters + pass, p->dev_err, p->sort_spin_limit);
        FGK_LAUNCH_CHECK();
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (vin != perm_out) FGK_CUDA(cudaMemcpyAsync(perm_out, vin, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    dev_free(w, s);
    return FGK_OK;
}

int build_sort(Plan *p, const double *X) {
    cudaStream_t s = p->stream;
    const int64_t N = p->N;
    const int d = p->d;
    double *xs = (double *)dev_alloc(sizeof(double) * N * d + 64, s);
    if (!xs) {
        set_error("device allocation for the scaled coordinates failed");
        return FGK_ERR_OOM;
    }
    int *bad = p->dev_err;
    FGK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_canon_scale<<<grid_for(N, 256), 256, 0, s>>>(X, N, d, p->a[0], p->a[1], p->a[2], xs, xs + N, xs + 2 * N,
                                                    bad);
    FGK_LAUNCH_CHECK();
    int hbad = 0;
    FGK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        dev_free(xs, s);
        FGK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        set_error("fgk_build: X holds a NaN or an infinity (or x * sqrt(2nu)/ell overflows)");
        return FGK_ERR_NONFINITE;
    }
    {
        const char *lim = getenv("FGK_SORT_SPIN_LIMIT");
        p->sort_spin_limit = lim ? std::max(1, atoi(lim)) : kSpinLimit;
    }
    for (int k = 0; k < d; ++k) {
        FGK_TRY(plan_alloc(p, (void **)&p->perm[k], N * sizeof(int32_t)));
        FGK_TRY(radix_sort(p, xs + k * N, p->perm[k], s));
    }
    // an expired look-back leaves the permutations invalid: stop before using them
    {
        const int rc = check_dev_error(p, "radix sort");
        if (rc != FGK_OK) {
            dev_free(xs, s);
            return rc;
        }
    }
    FGK_TRY(plan_alloc(p, (void **)&p->rank1, N * sizeof(int32_t)));
    k_invert<<<grid_for(N, 256), 256, 0, s>>>(p->perm[0], N, p->rank1);
    FGK_LAUNCH_CHECK();
    for (int k = 0; k < d; ++k) {
        FGK_TRY(plan_alloc(p, (void **)&p->xq[k], N * sizeof(double)));
        k_gather_f64<<<grid_for(N, 256), 256, 0, s>>>(xs + k * N, p->perm[0], N, p->xq[k]);
        FGK_LAUNCH_CHECK();
    }
    FGK_TRY(plan_alloc(p, (void **)&p->xraw_q, N * d * sizeof(double)));
    k_gather_rows<<<grid_for(N, 256), 256, 0, s>>>(X, p->perm[0], N, d, p->xraw_q);
    FGK_LAUNCH_CHECK();
    dev_free(xs, s);
    return check_dev_error(p, "radix sort");
}

}  // namespace fgk
