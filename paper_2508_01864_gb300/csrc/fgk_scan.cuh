// K3/K4: bidirectional segmented scans of the exponentially weighted
// polynomial moments, one level of the dominance structure per grid row.
//
// What is computed.  With scaled coordinates the Matérn kernel is
// k(r) = sum_{p<P} c_p r^p e^{-r}, P = nu + 1/2, c = (1), (1,1), (1,1,1/3)
// (eqs. matern_1_2, matern_3_2, matern_5_2 after eq. scaled_kernel).  At one
// level, a source i and a query j of complementary roles in the same segment
// are at distance r = sum_k (o_k(i) + o_k(j)) + D(i,j) for the L1 kernel,
// where o_k are the stored split offsets and D the sweep-coordinate distance,
// and the product kernel factorises as prod_k k(o_k(i) + o_k(j)) * k(D).
// The kernel sum over all sources before (forward) or after (backward) a
// query in the sweep order is the weighted ECDF of eq. ECDFdelta taken over
// that level, and the paper evaluates it by fast sum updating (Sec. 2.1,
// eq. fast_exact_decomposition_1d): one pass, each new source added to
// running sums.  The paper's running sums carry weights exp(+a x) x^p
// (eq. matern_weights), which overflow and cancel in finite precision; here
// the running sums are kept relative to the current sweep position instead:
//
//   M[a][q] = sum_{sources} v w_a(o) D^q e^{-D},
//
// so every factor lies in [0, 1] or is a non-negative binomial weight:
//   step by a gap g:   M[a][q] <- e^{-g} sum_{t<=q} C(q,t) g^{q-t} M[a][t]
//   insert a source:   M[a][0] += v * prod_k o_k^{a_k} e^{-o_k}   (product)
//                      M[0][q] += v * s^q e^{-s},  s = sum_k o_k   (L1)
//   read a query:      sum_a prod_k u_{a_k}(o_k) sum_q c_q M[a][q] (product)
//                      sum_q u_q(s) M[0][q]                         (L1)
// with u_q(s) = e^{-s} sum_{p>=q} c_p C(p,q) s^{p-q}.  These are the same
// sums as eqs. matern_12_decomposition, matern_32_decomposition,
// matern_52_decomposition (L1) and eq. product_decomposition, Proposition 2
// (product), with the orthants delta realised as the two sweep directions
// times the complementary role channels.
//
// Parallel form.  A run of entries acts on the moments as the affine map
// M -> A(T) M + M_run, where T is the run's summed gap and A(T) the step
// matrix above; maps compose associatively,
//   (T1, M1) then (T2, M2) = (T1 + T2, A(T2) M1 + M2),
// so a segment is scanned in parallel: each thread folds kScanEPT entries,
// threads of one segment combine by warp shuffles and shared memory, and
// segments longer than a tile receive the aggregate of their earlier
// (forward) or later (backward) tiles from a separate carry pass.  The decay
// of a run is recomputed as e^{-T} from its summed gap T whenever runs are
// composed, never carried as a product of per-entry factors: a factor near 1
// holds the decay 1 - e^{-g} to only ~eps/g relative accuracy, and a product
// of thousands of them would turn that into a visible error in the distance.
#pragma once

#include <type_traits>

#include "fgk_internal.cuh"

namespace fgk {

constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

enum { SCAN_AGG = 0, SCAN_OUT = 1 };

template <int P, int NOFF, int KIND>
struct Traits {
    static constexpr int NA = (KIND == FGK_PRODUCT && NOFF > 0 && P > 1) ? ipow_c(P, NOFF) : 1;
    static constexpr int MOM = NA * P;
    static constexpr int NCH = 1 << NOFF;
    static constexpr int AG = 1 + MOM;  // summed gap T, then the moments
};

template <class R>
struct ScanArgs {
    const uint32_t *lv_q;
    const R *lv_dl;
    const R *lv_off;  // (d-1) blocks of nlev x N
    int64_t N;
    int nlev;
    const WorkItem *items;
    const void *V;  // q order, N x nrhs
    int vin_f64;
    int nrhs;
    R *Y;          // q order, N x nrhs, accumulated atomically
    R *agg;        // SCAN_AGG: tile aggregates out; SCAN_OUT: carries in
    R s2;
    int *err;
    const int *gate;  // NULL, or a device int: 0 = skip the whole product
};

template <class R>
__device__ __forceinline__ R exp_neg(R x);
template <>
__device__ __forceinline__ float exp_neg<float>(float x) { return __expf(-x); }
template <>
__device__ __forceinline__ double exp_neg<double>(double x) { return exp(-x); }

// one group of P moments stepped by (T, E = e^{-T})
template <class R, int P>
__device__ __forceinline__ void step_group(R *m, R T, R E) {
    if constexpr (P == 1) {
        m[0] *= E;
    } else if constexpr (P == 2) {
        const R ET = E == R(0) ? R(0) : E * T;
        m[1] = E * m[1] + ET * m[0];
        m[0] *= E;
    } else {
        const R ET = E == R(0) ? R(0) : E * T;
        const R ET2 = E == R(0) ? R(0) : ET * T;
        m[2] = E * m[2] + R(2) * ET * m[1] + ET2 * m[0];
        m[1] = E * m[1] + ET * m[0];
        m[0] *= E;
    }
}

template <class R, int P, int MOM>
__device__ __forceinline__ void step_all(R *M, R T, R E) {
#pragma unroll
    for (int a = 0; a < MOM / P; ++a) step_group<R, P>(M + a * P, T, E);
}

// coefficients u_j(o) = e^{-o} sum_{p>=j} c_p C(p,j) o^{p-j}
template <class R, int P>
__device__ __forceinline__ void ucoef(R o, R eo, R *u) {
    if constexpr (P == 1) {
        u[0] = eo;
    } else if constexpr (P == 2) {
        u[0] = eo * (R(1) + o);
        u[1] = eo;
    } else {
        const R third = R(1) / R(3);
        u[0] = eo * (R(1) + o + third * o * o);
        u[1] = eo * (R(1) + R(2) * third * o);
        u[2] = eo * third;
    }
}

template <class R, int P>
__device__ __forceinline__ R csum(const R *m) {
    if constexpr (P == 1) return m[0];
    else if constexpr (P == 2) return m[0] + m[1];
    else return m[0] + m[1] + m[2] * (R(1) / R(3));
}

template <class R, int P, int NOFF, int KIND>
__device__ __forceinline__ void insert_src(R *M, R v, const R *o, const R *eo) {
    using Tr = Traits<P, NOFF, KIND>;
    if constexpr (NOFF == 0) {
        M[0] += v;
    } else if constexpr (Tr::NA == 1) {
        R s = o[0], es = eo[0];
        if constexpr (NOFF == 2) {
            s += o[1];
            es *= eo[1];
        }
        R w = v * es;
        M[0] += w;
        if constexpr (P > 1) {
            w *= s;
            M[1] += w;
        }
        if constexpr (P > 2) {
            w *= s;
            M[2] += w;
        }
    } else {
        R f[NOFF][P];
#pragma unroll
        for (int k = 0; k < NOFF; ++k) {
            f[k][0] = eo[k];
#pragma unroll
            for (int j = 1; j < P; ++j) f[k][j] = f[k][j - 1] * o[k];
        }
#pragma unroll
        for (int a = 0; a < Tr::NA; ++a) {
            R w = v;
            int rem = a;
#pragma unroll
            for (int k = 0; k < NOFF; ++k) {
                w *= f[k][rem % P];
                rem /= P;
            }
            M[a * P] += w;
        }
    }
}

template <class R, int P, int NOFF, int KIND>
__device__ __forceinline__ R read_query(const R *M, const R *o, const R *eo) {
    using Tr = Traits<P, NOFF, KIND>;
    if constexpr (NOFF == 0) {
        return csum<R, P>(M);
    } else if constexpr (Tr::NA == 1) {
        R s = o[0], es = eo[0];
        if constexpr (NOFF == 2) {
            s += o[1];
            es *= eo[1];
        }
        R u[P];
        ucoef<R, P>(s, es, u);
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < P; ++q) acc += u[q] * M[q];
        return acc;
    } else {
        R u[NOFF][P];
#pragma unroll
        for (int k = 0; k < NOFF; ++k) ucoef<R, P>(o[k], eo[k], u[k]);
        R acc = R(0);
#pragma unroll
        for (int a = 0; a < Tr::NA; ++a) {
            R c = R(1);
            int rem = a;
#pragma unroll
            for (int k = 0; k < NOFF; ++k) {
                c *= u[k][rem % P];
                rem /= P;
            }
            acc += c * csum<R, P>(M + a * P);
        }
        return acc;
    }
}

// x = prev then x   (prev precedes x in the walk direction): the moments of
// prev are stepped across x's span T (decay e^{-T}) and added to x's.
template <class R, int P, int AG>
__device__ __forceinline__ void compose_after(R *x, const R *prev) {
    R tmp[AG - 1];
#pragma unroll
    for (int m = 0; m < AG - 1; ++m) tmp[m] = prev[1 + m];
    step_all<R, P, AG - 1>(tmp, x[0], exp_neg<R>(x[0]));
#pragma unroll
    for (int m = 0; m < AG - 1; ++m) x[1 + m] += tmp[m];
    x[0] += prev[0];
}

template <class R, int AG>
__device__ __forceinline__ void set_identity(R *x) {
#pragma unroll
    for (int m = 0; m < AG; ++m) x[m] = R(0);
}

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <class R, int P, int NOFF, int KIND>
struct SmemLayout {
    using Tr = Traits<P, NOFF, KIND>;
    static constexpr int NW = kScanThreads / 32;
    static constexpr size_t q_off = 0;
    static constexpr size_t dl_off = align_up(q_off + sizeof(uint32_t) * (kTile + 1), 16);
    static constexpr size_t edl_off = align_up(dl_off + sizeof(R) * (kTile + 1), 16);
    static constexpr size_t o_off = align_up(edl_off + sizeof(R) * (kTile + 1), 16);
    static constexpr size_t eo_off = align_up(o_off + sizeof(R) * kTile * NOFF, 16);
    static constexpr size_t w_off = align_up(eo_off + sizeof(R) * kTile * NOFF, 16);
    static constexpr size_t wex_off = align_up(w_off + sizeof(R) * NW * Tr::AG, 16);
    static constexpr size_t bytes = align_up(wex_off + sizeof(R) * NW * Tr::AG, 16);
};

template <class R, int P, int NOFF, int KIND, int MODE>
__global__ void __launch_bounds__(kScanThreads) k_level_scan(ScanArgs<R> A) {
    using Tr = Traits<P, NOFF, KIND>;
    using Lay = SmemLayout<R, P, NOFF, KIND>;
    constexpr int MOM = Tr::MOM, NCH = Tr::NCH, AG = Tr::AG, EPT = kScanEPT, NT = kScanThreads;
    constexpr int NW = NT / 32;
    constexpr int LOG2EPT = (EPT == 8) ? 3 : (EPT == 4 ? 2 : (EPT == 16 ? 4 : 0));
    static_assert((1 << LOG2EPT) == EPT, "EPT must be 4, 8 or 16");

    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *s_q = (uint32_t *)(smem + Lay::q_off);
    R *s_dl = (R *)(smem + Lay::dl_off);
    R *s_edl = (R *)(smem + Lay::edl_off);
    R *s_o = (R *)(smem + Lay::o_off);
    R *s_eo = (R *)(smem + Lay::eo_off);
    R *s_w = (R *)(smem + Lay::w_off);
    R *s_wex = (R *)(smem + Lay::wex_off);

    if (A.gate && *A.gate == 0) return;
    const WorkItem wi = A.items[blockIdx.x];
    const int64_t N = A.N;
    const int64_t base = (int64_t)wi.tile * kTile;
    const int cnt = (int)(N - base < (int64_t)kTile ? N - base : (int64_t)kTile);
    const int log2S = wi.log2S;
    const int64_t S = int64_t(1) << log2S;
    const size_t lo = (size_t)wi.level * N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i <= kTile; i += NT) {
        const int64_t pos = base + i;
        R g = R(0);
        if (pos < N && (i < kTile || (pos & (S - 1)) != 0)) g = A.lv_dl[lo + pos];
        s_dl[i] = g;
        s_edl[i] = exp_neg<R>(g);
        if (i < kTile) {
            s_q[i] = pos < N ? A.lv_q[lo + pos] : 0u;
#pragma unroll
            for (int k = 0; k < NOFF; ++k) {
                R o = pos < N ? A.lv_off[((size_t)k * A.nlev + wi.level) * N + pos] : R(0);
                s_o[k * kTile + i] = o;
                s_eo[k * kTile + i] = exp_neg<R>(o);
            }
        }
    }
    __syncthreads();

    const int j0 = tid * EPT;
    const bool multi = log2S < LOG2EPT;  // several segments inside one thread's entries
    // scan group (in threads) for segments no longer than a tile
    const int G = multi ? 1 : (int)((S >> LOG2EPT) < (int64_t)NT ? (S >> LOG2EPT) : (int64_t)NT);
    const bool is_long = S > kTile;

    for (int r = 0; r < A.nrhs; ++r) {
        R v[EPT], out[EPT];
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            const int j = j0 + i;
            out[i] = R(0);
            v[i] = R(0);
            if (j < cnt) {
                const size_t idx = (size_t)(s_q[j] & 0x3fffffffu) * A.nrhs + r;
                v[i] = A.vin_f64 ? (R)((const double *)A.V)[idx] : (R)((const float *)A.V)[idx];
            }
        }
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int vlane = dir == 0 ? lane : 31 - lane;
            const int vwarp = dir == 0 ? warp : NW - 1 - warp;
#pragma unroll 1
            for (int c = 0; c < NCH; ++c) {
                const int qrole = c ^ (NCH - 1);
                R excl[AG];
                set_identity<R, AG>(excl);
                if (!multi) {
                    // 1. fold this thread's entries
                    R cur[AG];
                    set_identity<R, AG>(cur);
#pragma unroll
                    for (int ii = 0; ii < EPT; ++ii) {
                        const int i = dir == 0 ? ii : EPT - 1 - ii;
                        const int j = j0 + i;
                        const R g = dir == 0 ? s_dl[j] : s_dl[j + 1];
                        const R eg = dir == 0 ? s_edl[j] : s_edl[j + 1];
                        step_all<R, P, MOM>(cur + 1, g, eg);
                        cur[0] += g;
                        if (j < cnt) {
                            const int role = NOFF == 0 ? 0 : (int)(s_q[j] >> (32 - NOFF));
                            if (role == c) {
                                R o[NOFF > 0 ? NOFF : 1], eo[NOFF > 0 ? NOFF : 1];
#pragma unroll
                                for (int k = 0; k < NOFF; ++k) {
                                    o[k] = s_o[k * kTile + j];
                                    eo[k] = s_eo[k * kTile + j];
                                }
                                insert_src<R, P, NOFF, KIND>(cur + 1, v[i], o, eo);
                            }
                        }
                    }
                    // 2. inclusive scan across the threads of the segment (virtual lanes)
                    const int GW = G < 32 ? G : 32;
                    R inc[AG];
#pragma unroll
                    for (int m = 0; m < AG; ++m) inc[m] = cur[m];
                    for (int dlt = 1; dlt < GW; dlt <<= 1) {
                        R prev[AG];
#pragma unroll
                        for (int m = 0; m < AG; ++m)
                            prev[m] = dir == 0 ? __shfl_up_sync(0xffffffffu, inc[m], dlt)
                                               : __shfl_down_sync(0xffffffffu, inc[m], dlt);
                        if ((vlane & (GW - 1)) >= dlt) compose_after<R, P, AG>(inc, prev);
                    }
                    // exclusive within the warp group
                    {
                        R prev[AG];
#pragma unroll
                        for (int m = 0; m < AG; ++m)
                            prev[m] = dir == 0 ? __shfl_up_sync(0xffffffffu, inc[m], 1)
                                               : __shfl_down_sync(0xffffffffu, inc[m], 1);
                        if ((vlane & (GW - 1)) != 0) {
#pragma unroll
                            for (int m = 0; m < AG; ++m) excl[m] = prev[m];
                        }
                    }
                    if (G > 32 || MODE == SCAN_AGG) {
                        // warp totals -> exclusive prefix over the warps of each group
                        if (vlane == 31) {
#pragma unroll
                            for (int m = 0; m < AG; ++m) s_w[vwarp * AG + m] = inc[m];
                        }
                        __syncthreads();
                        if (tid == 0) {
                            const int GWn = G > 32 ? G / 32 : 1;
                            R run[AG];
                            set_identity<R, AG>(run);
                            if (MODE == SCAN_OUT && is_long) {
                                const R *cin = A.agg + ((((size_t)wi.agg * 2 + dir) * A.nrhs + r) * NCH + c) * AG;
#pragma unroll
                                for (int m = 0; m < AG; ++m) run[m] = cin[m];
                            }
                            for (int w = 0; w < NW; ++w) {
                                if (!is_long && (w % GWn) == 0) set_identity<R, AG>(run);
#pragma unroll
                                for (int m = 0; m < AG; ++m) s_wex[w * AG + m] = run[m];
                                R t[AG];
#pragma unroll
                                for (int m = 0; m < AG; ++m) t[m] = s_w[w * AG + m];
                                compose_after<R, P, AG>(t, run);
#pragma unroll
                                for (int m = 0; m < AG; ++m) run[m] = t[m];
                            }
                            if (MODE == SCAN_AGG) {
                                R *aout = A.agg + ((((size_t)wi.agg * 2 + dir) * A.nrhs + r) * NCH + c) * AG;
#pragma unroll
                                for (int m = 0; m < AG; ++m) aout[m] = run[m];
                            }
                        }
                        __syncthreads();
                        if (MODE == SCAN_OUT && G > 32) {
                            R wex[AG];
#pragma unroll
                            for (int m = 0; m < AG; ++m) wex[m] = s_wex[vwarp * AG + m];
                            compose_after<R, P, AG>(excl, wex);
                        }
                        __syncthreads();
                    }
                }
                if (MODE == SCAN_AGG) continue;
                // 3. walk again from the carried-in moments and read the queries
                R st[MOM];
#pragma unroll
                for (int m = 0; m < MOM; ++m) st[m] = excl[1 + m];
#pragma unroll
                for (int ii = 0; ii < EPT; ++ii) {
                    const int i = dir == 0 ? ii : EPT - 1 - ii;
                    const int j = j0 + i;
                    if (multi) {
                        const bool seg_start = dir == 0 ? (j & (S - 1)) == 0 : ((j + 1) & (S - 1)) == 0;
                        if (seg_start) {
#pragma unroll
                            for (int m = 0; m < MOM; ++m) st[m] = R(0);
                        }
                    }
                    const R g = dir == 0 ? s_dl[j] : s_dl[j + 1];
                    const R eg = dir == 0 ? s_edl[j] : s_edl[j + 1];
                    step_all<R, P, MOM>(st, g, eg);
                    if (j < cnt) {
                        const int role = NOFF == 0 ? 0 : (int)(s_q[j] >> (32 - NOFF));
                        R o[NOFF > 0 ? NOFF : 1], eo[NOFF > 0 ? NOFF : 1];
#pragma unroll
                        for (int k = 0; k < NOFF; ++k) {
                            o[k] = s_o[k * kTile + j];
                            eo[k] = s_eo[k * kTile + j];
                        }
                        if (role == qrole) out[i] += read_query<R, P, NOFF, KIND>(st, o, eo);
                        if (role == c) insert_src<R, P, NOFF, KIND>(st, v[i], o, eo);
                    }
                }
            }
        }
        if (MODE == SCAN_OUT) {
#pragma unroll
            for (int i = 0; i < EPT; ++i) {
                const int j = j0 + i;
                if (j < cnt) atomicAdd(A.Y + (size_t)(s_q[j] & 0x3fffffffu) * A.nrhs + r, A.s2 * out[i]);
            }
        }
    }
}

// Exclusive scan of the tile aggregates of every long segment, in both
// directions: carry[tile] = composition of the tiles before it (forward) or
// after it (backward).  One thread per (segment, direction, rhs, channel).
template <class R, int P, int NOFF, int KIND>
__global__ void k_carry_scan(const R *__restrict__ agg, R *__restrict__ carry, const int32_t *__restrict__ segs,
                             int nseg, int nrhs, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    using Tr = Traits<P, NOFF, KIND>;
    constexpr int AG = Tr::AG, NCH = Tr::NCH;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nseg * 2 * nrhs * NCH;
    if (t >= total) return;
    const int c = (int)(t % NCH);
    const int r = (int)((t / NCH) % nrhs);
    const int dir = (int)((t / ((int64_t)NCH * nrhs)) % 2);
    const int sg = (int)(t / ((int64_t)NCH * nrhs * 2));
    const int a0 = segs[2 * sg], nt = segs[2 * sg + 1];
    R run[AG];
    set_identity<R, AG>(run);
    for (int k = 0; k < nt; ++k) {
        const int slot = a0 + (dir == 0 ? k : nt - 1 - k);
        const size_t off = ((((size_t)slot * 2 + dir) * nrhs + r) * NCH + c) * AG;
        R x[AG];
#pragma unroll
        for (int m = 0; m < AG; ++m) {
            x[m] = agg[off + m];
            carry[off + m] = run[m];
        }
        compose_after<R, P, AG>(x, run);
#pragma unroll
        for (int m = 0; m < AG; ++m) run[m] = x[m];
    }
}

template <class R>
__global__ void k_diag_init(const void *__restrict__ V, int vin_f64, int64_t n, R s2, R *__restrict__ Y,
                            const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const R v = vin_f64 ? (R)((const double *)V)[i] : (R)((const float *)V)[i];
    Y[i] = s2 * v;
}

template <class R, int P, int NOFF, int KIND>
int run_levels(Plan *p, const void *Vq, bool vin64, int nrhs, R *Yq, R *ws, cudaStream_t s, const int *gate) {
    using Tr = Traits<P, NOFF, KIND>;
    using Lay = SmemLayout<R, P, NOFF, KIND>;
    static bool attr_set = false;
    if (!attr_set) {
        FGK_CUDA(cudaFuncSetAttribute(k_level_scan<R, P, NOFF, KIND, SCAN_AGG>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes));
        FGK_CUDA(cudaFuncSetAttribute(k_level_scan<R, P, NOFF, KIND, SCAN_OUT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes));
        attr_set = true;
    }
    ScanArgs<R> A;
    A.lv_q = p->lv_q;
    A.lv_dl = std::is_same<R, float>::value ? (const R *)p->lv_dl32 : (const R *)p->lv_dl64;
    A.lv_off = std::is_same<R, float>::value ? (const R *)p->lv_off32 : (const R *)p->lv_off64;
    A.N = p->N;
    A.nlev = p->nlev;
    A.V = Vq;
    A.vin_f64 = vin64 ? 1 : 0;
    A.nrhs = nrhs;
    A.Y = Yq;
    A.s2 = (R)p->s2;
    A.err = p->dev_err;
    A.gate = gate;
    const size_t per_slot = (size_t)2 * nrhs * Tr::NCH * Tr::AG;
    R *agg = ws;
    R *carry = ws + (size_t)p->n_long * per_slot;
    if (p->n_long > 0) {
        A.items = p->long_items;
        A.agg = agg;
        k_level_scan<R, P, NOFF, KIND, SCAN_AGG><<<p->n_long, kScanThreads, Lay::bytes, s>>>(A);
        FGK_LAUNCH_CHECK();
        const int64_t nthr = (int64_t)p->n_long_segments * 2 * nrhs * Tr::NCH;
        k_carry_scan<R, P, NOFF, KIND><<<grid_for(nthr, 128), 128, 0, s>>>(agg, carry, p->long_seg,
                                                                           p->n_long_segments, nrhs, gate);
        FGK_LAUNCH_CHECK();
    }
    if (p->n_items > 0) {
        A.items = p->items;
        A.agg = carry;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (scan_timing_enabled() && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
            cs == cudaStreamCaptureStatusNone) {
            FGK_CUDA(cudaEventCreate(&e0));
            FGK_CUDA(cudaEventCreate(&e1));
            FGK_CUDA(cudaEventRecord(e0, s));
        }
        k_level_scan<R, P, NOFF, KIND, SCAN_OUT><<<p->n_items, kScanThreads, Lay::bytes, s>>>(A);
        FGK_LAUNCH_CHECK();
        if (e0) {
            FGK_CUDA(cudaEventRecord(e1, s));
            scan_timing_record(e0, e1);
        }
    }
    return FGK_OK;
}

template <class R>
size_t scan_ws_elems(const Plan *p, int nrhs) {
    // generous: the largest AG (product, P = 3, d = 3: 1 + 27) and 4 channels
    return (size_t)2 * p->n_long * 2 * nrhs * 4 * 29 + 64;
}

// dispatch over (P, d-1, kind); nu = 1/2 or d = 1 make both kinds the same kernel
template <class R>
int run_levels_dispatch(Plan *p, const void *Vq, bool vin64, int nrhs, R *Yq, R *ws, cudaStream_t s,
                        const int *gate) {
    const int P = p->P, NOFF = p->d - 1;
    const int kind = (P == 1 || NOFF == 0) ? FGK_L1 : p->kind;
    const int key = (P * 3 + NOFF) * 2 + kind;
    switch (key) {
#define FGK_CASE(PP, NO, KK) \
    case (PP * 3 + NO) * 2 + KK: return run_levels<R, PP, NO, KK>(p, Vq, vin64, nrhs, Yq, ws, s, gate);
        FGK_CASE(1, 0, FGK_L1)
        FGK_CASE(2, 0, FGK_L1)
        FGK_CASE(3, 0, FGK_L1)
        FGK_CASE(1, 1, FGK_L1)
        FGK_CASE(2, 1, FGK_L1)
        FGK_CASE(3, 1, FGK_L1)
        FGK_CASE(2, 1, FGK_PRODUCT)
        FGK_CASE(3, 1, FGK_PRODUCT)
        FGK_CASE(1, 2, FGK_L1)
        FGK_CASE(2, 2, FGK_L1)
        FGK_CASE(3, 2, FGK_L1)
        FGK_CASE(2, 2, FGK_PRODUCT)
        FGK_CASE(3, 2, FGK_PRODUCT)
#undef FGK_CASE
    default:
        break;
    }
    set_error("no scan kernel for P=%d d=%d kind=%d", P, p->d, p->kind);
    return FGK_ERR_INTERNAL;
}

}  // namespace fgk
