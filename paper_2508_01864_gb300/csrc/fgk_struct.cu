// K2: the dominance structure (Sec. 2.2.3: the sorted subsets of every node
// of the divide and conquer are computed once and stored, so that taking a
// product needs no sort).
//
// A level lists every point once, in aligned power-of-two segments, each
// segment ordered by the sweep coordinate (the last one).  With q the
// point's position in x'_1 order and L = ceil(log2 N):
//   d = 2: level l has segments of 2^(L-l) consecutive q; the role of a point
//          is bit (L-1-l) of q (low or high half of the segment in x'_1).
//   d = 3: outer level l1 groups 2^(L-l1) consecutive q; inside an outer
//          segment the points are ranked by x'_2 (local rank lr2) and inner
//          level l2 splits those ranks the same way, role r2 = bit
//          (L-l1-1-l2) of lr2.
// Two distinct points meet at exactly one level with complementary roles in
// every split dimension, so every pair of the kernel sum is visited once
// (the divide and conquer of Bentley that the paper cites, with the sorting
// steps replaced by these stored orders).
//
// Construction: level l+1 is level l with every segment stably split by
// its role bit (zero half first).  The zero half of a segment of size S
// holding c entries has min(S/2, c) entries, so the destination of an entry
// is its segment start plus a segmented exclusive count.
//
// Per entry the level also stores the gap dl of the sweep coordinate to the
// previous entry of its segment and, for each split dimension, the offset
// |x' - split| to the segment's split value (the last point of its low half,
// clamped to the segment's last point), in FP64 and rounded to FP32.
#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kPartThreads = 256;
constexpr int kPartEPT = 4;
constexpr int kPartTile = kPartThreads * kPartEPT;
constexpr uint32_t kQMask = 0x3fffffffu;

__global__ void k_gather_q(const int32_t *__restrict__ perm_d, const int32_t *__restrict__ rank1, int64_t N,
                           uint32_t *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) out[i] = (uint32_t)rank1[perm_d[i]];
}

__device__ __forceinline__ uint32_t part_bit(uint32_t q, const uint32_t *key_src, int bitpos) {
    uint32_t k = key_src ? key_src[q] : q;
    return (k >> bitpos) & 1u;
}

// zeros per tile of kPartTile entries
__global__ void k_tile_zero_counts(const uint32_t *__restrict__ in, int64_t N, const uint32_t *__restrict__ key_src,
                                   int bitpos, uint32_t *__restrict__ tile_zero) {
    __shared__ uint32_t s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kPartTile;
    uint32_t c = 0;
    for (int e = 0; e < kPartEPT; ++e) {
        int64_t i = base + threadIdx.x * kPartEPT + e;
        if (i < N) c += 1u - part_bit(in[i] & kQMask, key_src, bitpos);
    }
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) tile_zero[blockIdx.x] = s;
}

// exclusive scan of tile counts inside each segment longer than a tile
__global__ void k_seg_tile_scan(uint32_t *__restrict__ tile_zero, int64_t ntiles, int64_t tiles_per_seg) {
    int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t t0 = sg * tiles_per_seg;
    if (t0 >= ntiles) return;
    int64_t t1 = min(t0 + tiles_per_seg, ntiles);
    uint32_t run = 0;
    for (int64_t t = t0; t < t1; ++t) {
        uint32_t c = tile_zero[t];
        tile_zero[t] = run;
        run += c;
    }
}

// stable split of each segment (size 2^log2S >= kPartEPT) by the bit
__global__ void __launch_bounds__(kPartThreads) k_partition(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                            int64_t N, int log2S, const uint32_t *__restrict__ key_src,
                                                            int bitpos, const uint32_t *__restrict__ tile_off,
                                                            int *__restrict__ err) {
    __shared__ uint32_t s_val[kPartThreads];
    __shared__ uint8_t s_flag[kPartThreads];
    const int64_t S = int64_t(1) << log2S;
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
    const int tid = threadIdx.x;
    const int64_t first = base + (int64_t)tid * kPartEPT;
    uint32_t q[kPartEPT], b[kPartEPT];
    uint32_t zeros = 0;
    for (int e = 0; e < kPartEPT; ++e) {
        int64_t i = first + e;
        q[e] = i < N ? (in[i] & kQMask) : 0;
        b[e] = i < N ? part_bit(q[e], key_src, bitpos) : 1;
        zeros += (i < N) ? 1u - b[e] : 0u;
    }
    // segmented inclusive scan over threads; a segment starts where first % S == 0
    uint32_t v = zeros;
    uint8_t f = (first % S) == 0;
    s_val[tid] = v;
    s_flag[tid] = f;
    __syncthreads();
    for (int off = 1; off < kPartThreads; off <<= 1) {
        uint32_t pv = 0;
        uint8_t pf = 0;
        if (tid >= off) {
            pv = s_val[tid - off];
            pf = s_flag[tid - off];
        }
        __syncthreads();
        if (tid >= off && !f) {
            v += pv;
            f |= pf;
        }
        s_val[tid] = v;
        s_flag[tid] = f;
        __syncthreads();
    }
    uint32_t e0 = v - zeros;  // zeros before my first entry, within my segment and tile
    // add the zeros of the segment's earlier tiles when the segment spans tiles
    if (S > kPartTile) e0 += tile_off[blockIdx.x];
    for (int e = 0; e < kPartEPT; ++e) {
        int64_t i = first + e;
        if (i >= N) break;
        int64_t seg0 = i & ~(S - 1);
        int64_t within = i - seg0;
        int64_t dst = b[e] ? seg0 + S / 2 + (within - e0) : seg0 + e0;
        if (dst < seg0 || dst >= N || dst >= seg0 + S)
            atomicExch(err, DEV_INTERNAL);  // the zero-half size assumption failed
        else
            out[dst] = q[e];
        e0 += 1u - b[e];
    }
}

// local rank of x'_2 inside each outer segment, from the outer order
__global__ void k_local_rank(const uint32_t *__restrict__ outer, int64_t N, int log2S1, uint32_t *__restrict__ lr2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N) lr2[outer[i] & kQMask] = (uint32_t)(i & ((int64_t(1) << log2S1) - 1));
}

__global__ void k_attrs_d1(const double *__restrict__ x1q, int64_t N, uint32_t *__restrict__ lq,
                           double *__restrict__ dl64, float *__restrict__ dl32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    lq[i] = (uint32_t)i;
    double g = i > 0 ? x1q[i] - x1q[i - 1] : 0.0;
    dl64[i] = g;
    dl32[i] = (float)g;
}

__global__ void k_attrs_d2(const double *__restrict__ x1q, const double *__restrict__ x2q, int64_t N, int L,
                           int lev, uint32_t *__restrict__ lq, double *__restrict__ dl64, float *__restrict__ dl32,
                           double *__restrict__ off64, float *__restrict__ off32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int log2S = L - lev;
    const int64_t S = int64_t(1) << log2S;
    uint32_t q = lq[i] & kQMask;
    uint32_t r1 = (q >> (L - 1 - lev)) & 1u;
    double g = 0.0;
    if (i % S) g = x2q[q] - x2q[lq[i - 1] & kQMask];
    int64_t seg0 = i & ~(S - 1);
    int64_t split = min(seg0 + S / 2 - 1, N - 1);
    double o = fabs(x1q[q] - x1q[split]);
    lq[i] = q | (r1 << 31);
    dl64[i] = g;
    dl32[i] = (float)g;
    off64[i] = o;
    off32[i] = (float)o;
}

// level (l1, l2) of d = 3: lq holds the inner order; pi is the outer order
__global__ void k_attrs_d3(const double *__restrict__ x1q, const double *__restrict__ x2q,
                           const double *__restrict__ x3q, const uint32_t *__restrict__ pi,
                           const uint32_t *__restrict__ lr2, int64_t N, int L, int l1, int l2,
                           uint32_t *__restrict__ lq, double *__restrict__ dl64, float *__restrict__ dl32,
                           double *__restrict__ off1_64, float *__restrict__ off1_32, double *__restrict__ off2_64,
                           float *__restrict__ off2_32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int log2S1 = L - l1;
    const int log2S = L - l1 - l2;
    const int64_t S1 = int64_t(1) << log2S1, S = int64_t(1) << log2S;
    uint32_t q = lq[i] & kQMask;
    uint32_t lr = lr2[q];
    uint32_t r1 = (q >> (L - 1 - l1)) & 1u;
    uint32_t r2 = (lr >> (log2S - 1)) & 1u;
    double g = 0.0;
    if (i % S) g = x3q[q] - x3q[lq[i - 1] & kQMask];
    int64_t o0 = i & ~(S1 - 1);
    int64_t cnt1 = min(S1, N - o0);
    int64_t split1 = min(o0 + S1 / 2 - 1, N - 1);
    int64_t h0 = (i - o0) & ~(S - 1);  // inner segment start, in local ranks
    int64_t split2 = o0 + min(h0 + S / 2 - 1, cnt1 - 1);
    double o1 = fabs(x1q[q] - x1q[split1]);
    double o2 = fabs(x2q[q] - x2q[pi[split2] & kQMask]);
    lq[i] = q | (r1 << 31) | (r2 << 30);
    dl64[i] = g;
    dl32[i] = (float)g;
    off1_64[i] = o1;
    off1_32[i] = (float)o1;
    off2_64[i] = o2;
    off2_32[i] = (float)o2;
}

struct PartWS {
    uint32_t *tile = nullptr;
    int64_t ntiles = 0;
};

// out = in with every segment (size 2^log2S) stably split by the bit
int partition(const uint32_t *in, uint32_t *out, int64_t N, int log2S, const uint32_t *key_src, int bitpos,
              PartWS &ws, int *err, cudaStream_t s) {
    const int64_t S = int64_t(1) << log2S;
    if (S > kPartTile) {
        k_tile_zero_counts<<<ws.ntiles, kPartThreads, 0, s>>>(in, N, key_src, bitpos, ws.tile);
        FGK_LAUNCH_CHECK();
        int64_t tps = S / kPartTile;
        int64_t nseg = (ws.ntiles + tps - 1) / tps;
        k_seg_tile_scan<<<grid_for(nseg, 128), 128, 0, s>>>(ws.tile, ws.ntiles, tps);
        FGK_LAUNCH_CHECK();
    }
    k_partition<<<ws.ntiles, kPartThreads, 0, s>>>(in, out, N, log2S, key_src, bitpos, ws.tile, err);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

}  // namespace

// e^{-x} of every entry of nblk blocks of ldN values (the levels of the FP64
// gaps or of one offset dimension), 1 for the padding past N in each block:
// the FP64 scans read these instead of taking an FP64 exponential per entry
// and product
__global__ void k_decays(const double *__restrict__ x, int64_t nblk, int64_t N, int64_t ldN,
                         double *__restrict__ ex) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nblk * ldN) return;
    ex[e] = (e % ldN) < N ? exp(-x[e]) : 1.0;
}

static int build_decays(Plan *p) {
    cudaStream_t s = p->stream;
    const int64_t nb = p->nlev, nbo = (int64_t)(p->d - 1) * p->nlev;
    FGK_TRY(plan_alloc(p, (void **)&p->lv_edl64, (size_t)nb * p->ldN * sizeof(double)));
    k_decays<<<grid_for(nb * p->ldN, 256), 256, 0, s>>>(p->lv_dl64, nb, p->N, p->ldN, p->lv_edl64);
    FGK_LAUNCH_CHECK();
    if (nbo > 0) {
        FGK_TRY(plan_alloc(p, (void **)&p->lv_eoff64, (size_t)nbo * p->ldN * sizeof(double)));
        k_decays<<<grid_for(nbo * p->ldN, 256), 256, 0, s>>>(p->lv_off64, nbo, p->N, p->ldN, p->lv_eoff64);
        FGK_LAUNCH_CHECK();
    }
    return FGK_OK;
}

int build_levels(Plan *p) {
    cudaStream_t s = p->stream;
    const int64_t N = p->N;
    const int d = p->d, L = p->L;
    const int nlev = p->nlev;
    const int64_t ldN = p->ldN;  // level stride (padded for aligned vector loads)
    const size_t E = (size_t)nlev * ldN;
    FGK_TRY(plan_alloc(p, (void **)&p->lv_q, E * sizeof(uint32_t)));
    FGK_TRY(plan_alloc(p, (void **)&p->lv_dl32, E * sizeof(float)));
    FGK_TRY(plan_alloc(p, (void **)&p->lv_dl64, E * sizeof(double)));
    if (d >= 2) {
        FGK_TRY(plan_alloc(p, (void **)&p->lv_off32, (size_t)(d - 1) * E * sizeof(float)));
        FGK_TRY(plan_alloc(p, (void **)&p->lv_off64, (size_t)(d - 1) * E * sizeof(double)));
    }
    p->lev_log2S.assign(nlev, 0);
    if (d == 1) {
        p->lev_log2S[0] = L;
        k_attrs_d1<<<grid_for(N, 256), 256, 0, s>>>(p->xq[0], N, p->lv_q, p->lv_dl64, p->lv_dl32);
        FGK_LAUNCH_CHECK();
        return build_decays(p);
    }
    PartWS ws;
    ws.ntiles = (N + kPartTile - 1) / kPartTile;
    size_t tmp_bytes = ws.ntiles * sizeof(uint32_t) + 64;
    if (d == 3) tmp_bytes += 5 * N * sizeof(uint32_t) + 64;
    char *tmp = (char *)dev_alloc(tmp_bytes, s);
    if (!tmp) {
        set_error("device allocation of %zu bytes for the structure build failed", tmp_bytes);
        return FGK_ERR_OOM;
    }
    ws.tile = (uint32_t *)tmp;
    if (d == 2) {
        uint32_t *lv0 = p->lv_q;
        k_gather_q<<<grid_for(N, 256), 256, 0, s>>>(p->perm[1], p->rank1, N, lv0);
        FGK_LAUNCH_CHECK();
        for (int l = 0; l < L; ++l) {
            p->lev_log2S[l] = L - l;
            uint32_t *cur = p->lv_q + (size_t)l * ldN;
            if (l + 1 < L) FGK_TRY(partition(cur, cur + ldN, N, L - l, nullptr, L - 1 - l, ws, p->dev_err, s));
            k_attrs_d2<<<grid_for(N, 256), 256, 0, s>>>(p->xq[0], p->xq[1], N, L, l, cur, p->lv_dl64 + (size_t)l * ldN,
                                                         p->lv_dl32 + (size_t)l * ldN, p->lv_off64 + (size_t)l * ldN,
                                                         p->lv_off32 + (size_t)l * ldN);
            FGK_LAUNCH_CHECK();
        }
    } else {
        uint32_t *buf = (uint32_t *)(tmp + ws.ntiles * sizeof(uint32_t) + 32);
        buf = (uint32_t *)(((uintptr_t)buf + 15) & ~uintptr_t(15));
        uint32_t *pi_cur = buf, *pi_nxt = buf + N, *rho_cur = buf + 2 * N, *rho_nxt = buf + 3 * N, *lr2 = buf + 4 * N;
        k_gather_q<<<grid_for(N, 256), 256, 0, s>>>(p->perm[1], p->rank1, N, pi_cur);
        FGK_LAUNCH_CHECK();
        k_gather_q<<<grid_for(N, 256), 256, 0, s>>>(p->perm[2], p->rank1, N, rho_cur);
        FGK_LAUNCH_CHECK();
        int lev = 0;
        for (int l1 = 0; l1 < L; ++l1) {
            const int log2S1 = L - l1;
            k_local_rank<<<grid_for(N, 256), 256, 0, s>>>(pi_cur, N, log2S1, lr2);
            FGK_LAUNCH_CHECK();
            // inner chain starts from the x'_3 order split into outer segments
            FGK_CUDA(cudaMemcpyAsync(p->lv_q + (size_t)lev * ldN, rho_cur, N * sizeof(uint32_t),
                                     cudaMemcpyDeviceToDevice, s));
            for (int l2 = 0; l2 < L - l1; ++l2) {
                const int log2S = L - l1 - l2;
                p->lev_log2S[lev + l2] = log2S;
                uint32_t *cur = p->lv_q + (size_t)(lev + l2) * ldN;
                if (l2 + 1 < L - l1)
                    FGK_TRY(partition(cur, cur + ldN, N, log2S, lr2, log2S - 1, ws, p->dev_err, s));
                size_t o = (size_t)(lev + l2) * ldN;
                k_attrs_d3<<<grid_for(N, 256), 256, 0, s>>>(
                    p->xq[0], p->xq[1], p->xq[2], pi_cur, lr2, N, L, l1, l2, cur, p->lv_dl64 + o, p->lv_dl32 + o,
                    p->lv_off64 + o, p->lv_off32 + o, p->lv_off64 + E + o, p->lv_off32 + E + o);
                FGK_LAUNCH_CHECK();
            }
            lev += L - l1;
            if (l1 + 1 < L) {
                FGK_TRY(partition(pi_cur, pi_nxt, N, log2S1, nullptr, L - 1 - l1, ws, p->dev_err, s));
                FGK_TRY(partition(rho_cur, rho_nxt, N, log2S1, nullptr, L - 1 - l1, ws, p->dev_err, s));
                std::swap(pi_cur, pi_nxt);
                std::swap(rho_cur, rho_nxt);
            }
        }
    }
    dev_free(tmp, s);
    return build_decays(p);
}

}  // namespace fgk
