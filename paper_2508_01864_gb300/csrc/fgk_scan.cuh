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

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "fgk_internal.cuh"

namespace fgk {

constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

// readout coefficients per factor of the generic-coefficient scans: up to six
// moments (the nu = 9/2 kernel has five, its lengthscale derivative six)
constexpr int kMaxCoef = 6;

enum { SCAN_AGG = 0, SCAN_OUT = 1 };

// resident CTAs per SM the scan kernels are compiled for (register budget)
#ifndef FGK_SCAN_MINB
#define FGK_SCAN_MINB 2
#endif
// the same for the FP64 scans (bound by GB300's FP64 pipe rather than by latency)
#ifndef FGK_SCAN_MINB_F64
#define FGK_SCAN_MINB_F64 FGK_SCAN_MINB
#endif

// Channels: a source of role c feeds the queries of the complementary role
// c ^ (NCH-1), so a pass handles one complementary pair {cA, cB} (d = 2: one
// pair; d = 3: two pairs; d = 1: one self-paired channel).  A pass carries,
// per direction, the summed gap T and the moments of its CP channels.
template <int P, int NOFF, int KIND>
struct Traits {
    static constexpr int NA = (KIND == FGK_PRODUCT && NOFF > 0 && P > 1) ? ipow_c(P, NOFF) : 1;
    static constexpr int MOM = NA * P;                 // moments per channel
    static constexpr int NCH = 1 << NOFF;              // role channels
    static constexpr int CP = NOFF == 0 ? 1 : 2;       // channels per pass
    static constexpr int NPASS = NOFF == 2 ? 2 : 1;    // channel-pair passes
    // The product kernel's moments fall into NA groups (one per power pattern
    // of the offsets) that the step never mixes, so groups can be scanned in
    // separate passes; a pass carries GP groups of P moments per channel.
    static constexpr int GP = (NA > 1 && CP * NA * P > 12) ? 1 : NA;
    static constexpr int NGP = NA / GP;                // group passes
    static constexpr int GM = GP * P;                  // moments per channel in a pass
    static constexpr int SM = CP * GM;                 // moments per pass and direction
    static constexpr int AG = 1 + SM;                  // aggregate: T, moments
    static constexpr int NDIR = SM <= 8 ? 2 : 1;       // directions walked together
    static constexpr int NPT = NPASS * NGP;            // passes per right-hand side
    static constexpr int NWC = NOFF == 0 ? 1 : (NA == 1 ? P : GP);  // per-entry coefficients of a pass
};


template <class R>
struct ScanArgs {
    const uint32_t *lv_q;
    const R *lv_dl;
    const R *lv_off;  // (d-1) blocks of nlev x ldN
    // FP64 only: the decays e^{-gap} and e^{-offset} of every entry, stored by
    // the structure build (1 past each level's end); NULL: computed per entry
    const R *lv_edl;
    const R *lv_eoff;
    int64_t N;
    int64_t ldN;
    int nlev;
    const WorkItem *items;
    // the work item of block k, without a load per block: k / ntiles indexes
    // lv_map (level | log2S << 16, the long-segment levels first), the tile is
    // k mod ntiles, and the first n_long blocks are the long-segment tiles with
    // aggregate slot k
    const uint32_t *lv_map;
    int ntiles;
    int n_long;
    const R *V;  // q order, N x nrhs, in the scan precision
    int nrhs;
    R *Y;      // q order, N x nrhs: accumulated atomically when rows == NULL
    // per-level output rows (q order, N x nrhs each, level l at l * row_stride):
    // every (level, point, column) slot is written exactly once per product by
    // a plain store, and k_level_sum adds the levels in a fixed order
    R *rows;
    int64_t row_stride;
    R *agg;    // SCAN_AGG: tile aggregates out; SCAN_OUT: carries in
    R s2;
    int *err;
    const int *gate;  // NULL, or a device int: 0 = skip the whole product
    // readout coefficients of the generic-coefficient scans (GEN): the
    // kernel factor sum_p cf[k][p] r^p e^{-r} of split dimension k (offset
    // block k), cf[d-1] for the sweep dimension, cf[0] for the L1 kernel's
    // radial factor
    R cf[kMaxD][kMaxCoef];
};

template <class R>
__device__ __forceinline__ R exp_neg(R x);
template <>
__device__ __forceinline__ float exp_neg<float>(float x) { return __expf(-x); }
template <>
__device__ __forceinline__ double exp_neg<double>(double x) { return exp(-x); }

__host__ __device__ constexpr int binom_c(int n, int k) {
    return (k < 0 || k > n) ? 0 : (k == 0 || k == n) ? 1 : binom_c(n - 1, k - 1) + binom_c(n - 1, k);
}

// one group of P moments stepped by (T, E = e^{-T})
template <class R, int P>
__device__ __forceinline__ void step_group(R *m, R T, R E) {
    if constexpr (P == 1) {
        m[0] *= E;
    } else if constexpr (P == 2) {
        const R ET = E == R(0) ? R(0) : E * T;
        m[1] = E * m[1] + ET * m[0];
        m[0] *= E;
    } else if constexpr (P == 3) {
        const R ET = E == R(0) ? R(0) : E * T;
        const R ET2 = E == R(0) ? R(0) : ET * T;
        m[2] = E * m[2] + R(2) * ET * m[1] + ET2 * m[0];
        m[1] = E * m[1] + ET * m[0];
        m[0] *= E;
    } else {
        // any order: m_q <- sum_{t<=q} C(q,t) E T^{q-t} m_t, from the highest q
        // down so that every m_t read is still the old one; the powers
        // E T^k are formed by repeated multiplication (each stays bounded by
        // max_T T^k e^{-T}, so nothing overflows before it is scaled)
        R ETk[P];
        ETk[0] = E;
#pragma unroll
        for (int k = 1; k < P; ++k) ETk[k] = E == R(0) ? R(0) : ETk[k - 1] * T;
#pragma unroll
        for (int q = P - 1; q >= 0; --q) {
            R acc = ETk[0] * m[q];
#pragma unroll
            for (int t = 0; t < q; ++t) acc += R(binom_c(q, t)) * ETk[q - t] * m[t];
            m[q] = acc;
        }
    }
}

template <class R, int P, int MOM>
__device__ __forceinline__ void step_all(R *M, R T, R E) {
#pragma unroll
    for (int a = 0; a < MOM / P; ++a) step_group<R, P>(M + a * P, T, E);
}

// One group of P moments kept relative to an anchor behind the current
// position (m~ = e^{+X} m, X the distance from the anchor): a step by G
// shifts only the polynomial part, m~_q <- sum_{t<=q} C(q,t) G^{q-t} m~_t.
template <class R, int P>
__device__ __forceinline__ void astep_group(R *m, R G) {
    if constexpr (P == 2) {
        m[1] = fma(G, m[0], m[1]);
    } else if constexpr (P == 3) {
        const R gm0 = G * m[0];
        m[2] = fma(G, fma(R(2), m[1], gm0), m[2]);
        m[1] += gm0;
    } else if constexpr (P > 3) {
        R Gk[P];
        Gk[0] = R(1);
#pragma unroll
        for (int k = 1; k < P; ++k) Gk[k] = Gk[k - 1] * G;
#pragma unroll
        for (int q = P - 1; q >= 1; --q) {
            R acc = m[q];
#pragma unroll
            for (int t = 0; t < q; ++t) acc += R(binom_c(q, t)) * Gk[q - t] * m[t];
            m[q] = acc;
        }
    }
}

template <class R, int P, int MOM>
__device__ __forceinline__ void astep_all(R *M, R G) {
#pragma unroll
    for (int a = 0; a < MOM / P; ++a) astep_group<R, P>(M + a * P, G);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp_approx(double x) { return 1.0 / x; }

// a thread's anchored walk is used when the gaps between its entries sum to
// at most this (scaled units): e^{+X} <= e^{20} ~ 5e8, so an anchored moment
// reaches the FP32 range limit only for operands near 1e29, where the product
// itself overflows FP32 anyway
constexpr float kAnchorSpan = 20.0f;

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

// o^e and u_e(o) = e^{-o} sum_{p>=e} c_p C(p,e) o^{p-e} for a run-time e < P
template <class R, int P>
__device__ __forceinline__ R pow_sel(R o, int e) {
    return e == 0 ? R(1) : (e == 1 ? o : o * o);
}
template <class R, int P>
__device__ __forceinline__ R ucoef_sel(R o, R eo, int e) {
    if constexpr (P == 2) {
        return e == 0 ? eo * (R(1) + o) : eo;
    } else {
        const R third = R(1) / R(3);
        return e == 0 ? eo * (R(1) + o + third * o * o) : (e == 1 ? eo * (R(1) + R(2) * third * o) : eo * third);
    }
}

// Generic readout coefficients (GEN scans: the lengthscale derivatives, whose
// factors have runtime coefficients and one order more).
template <class R>
__device__ __forceinline__ R pow_rt(R o, int e) {  // o^e, 0 <= e < kMaxCoef
    R r = R(1);
#pragma unroll
    for (int k = 1; k < kMaxCoef; ++k) r = k <= e ? r * o : r;
    return r;
}
// u_j(o) = e^{-o} sum_{p>=j} cf[p] C(p,j) o^{p-j}, all j < P
template <class R, int P>
__device__ __forceinline__ void ucoef_gen(R o, R eo, const R *cf, R *u) {
    R op[P];
    op[0] = R(1);
#pragma unroll
    for (int q = 1; q < P; ++q) op[q] = op[q - 1] * o;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        R acc = R(0);
#pragma unroll
        for (int q = j; q < P; ++q) acc += cf[q] * R(binom_c(q, j)) * op[q - j];
        u[j] = eo * acc;
    }
}
// the same for one run-time j = e
template <class R, int P>
__device__ __forceinline__ R ucoef_sel_gen(R o, R eo, int e, const R *cf) {
    R acc = R(0);
#pragma unroll
    for (int q = 0; q < P; ++q) {
        R c = R(0);
#pragma unroll
        for (int j = 0; j <= q; ++j)
            if (j == e) c = cf[q] * R(binom_c(q, j)) * pow_rt<R>(o, q - j);
        acc += c;
    }
    return eo * acc;
}
template <class R, int P>
__device__ __forceinline__ R csum_gen(const R *m, const R *cf) {
    R acc = R(0);
#pragma unroll
    for (int q = 0; q < P; ++q) acc += cf[q] * m[q];
    return acc;
}

// Per-entry coefficients of one pass (groups a0 .. a0+GP-1), from the
// entry's offsets o and e^{-o}:
//   insertion w: L1   w[q] = e^{-s} s^q (s = sum of offsets), added to M[q];
//                product w[g] = prod_k o_k^{a_k} e^{-o_k}, added to M[g][0];
//   readout   u: L1   u[q] = u_q(s); product u[g] = prod_k u_{a_k}(o_k).
// d = 1 needs neither (v is added to M[0], the query reads sum_q c_q M[q]).
template <class R, int P, int NOFF, int KIND, bool GEN = false>
__device__ __forceinline__ void pass_coef(int a0, const R *o, const R *eo, R *w, R *u, const R (*cf)[kMaxCoef] = nullptr) {
    using Tr = Traits<P, NOFF, KIND>;
    if constexpr (NOFF == 0) {
        w[0] = R(1);
        u[0] = R(1);
    } else if constexpr (Tr::NA == 1) {
        R s = o[0], es = eo[0];
        if constexpr (NOFF == 2) {
            s += o[1];
            es *= eo[1];
        }
        w[0] = es;
#pragma unroll
        for (int q = 1; q < P; ++q) w[q] = w[q - 1] * s;
        if constexpr (GEN)
            ucoef_gen<R, P>(s, es, cf[0], u);
        else
            ucoef<R, P>(s, es, u);
    } else {
#pragma unroll
        for (int g = 0; g < Tr::GP; ++g) {
            const int a = a0 + g;
            const int e0 = NOFF == 1 ? a : a % P;
            R ww, uu;
            if constexpr (GEN) {
                ww = eo[0] * pow_rt<R>(o[0], e0);
                uu = ucoef_sel_gen<R, P>(o[0], eo[0], e0, cf[0]);
            } else {
                ww = eo[0] * pow_sel<R, P>(o[0], e0);
                uu = ucoef_sel<R, P>(o[0], eo[0], e0);
            }
            if constexpr (NOFF == 2) {
                const int e1 = a / P;
                if constexpr (GEN) {
                    ww *= eo[1] * pow_rt<R>(o[1], e1);
                    uu *= ucoef_sel_gen<R, P>(o[1], eo[1], e1, cf[1]);
                } else {
                    ww *= eo[1] * pow_sel<R, P>(o[1], e1);
                    uu *= ucoef_sel<R, P>(o[1], eo[1], e1);
                }
            }
            w[g] = ww;
            u[g] = uu;
        }
    }
}

template <class R, int P, int NOFF, int KIND>
__device__ __forceinline__ void add_pass(R *M, R v, const R *w) {
    using Tr = Traits<P, NOFF, KIND>;
    if constexpr (NOFF == 0) {
        M[0] += v;
    } else if constexpr (Tr::NA == 1) {
#pragma unroll
        for (int q = 0; q < P; ++q) M[q] += v * w[q];
    } else {
#pragma unroll
        for (int g = 0; g < Tr::GP; ++g) M[g * P] += v * w[g];
    }
}

template <class R, int P, int NOFF, int KIND, bool GEN = false>
__device__ __forceinline__ R read_pass(const R *M, const R *u, const R (*cf)[kMaxCoef] = nullptr) {
    using Tr = Traits<P, NOFF, KIND>;
    if constexpr (NOFF == 0) {
        if constexpr (GEN)
            return csum_gen<R, P>(M, cf[0]);
        else
            return csum<R, P>(M);
    } else if constexpr (Tr::NA == 1) {
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < P; ++q) acc += u[q] * M[q];
        return acc;
    } else {
        R acc = R(0);
#pragma unroll
        for (int g = 0; g < Tr::GP; ++g) {
            if constexpr (GEN)
                acc += u[g] * csum_gen<R, P>(M + g * P, cf[NOFF]);
            else
                acc += u[g] * csum<R, P>(M + g * P);
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

// One CTA = one tile of kTile consecutive entries of one level; each thread
// owns kScanEPT consecutive entries, held in registers.  Per right-hand side
// and channel pair: fold each thread's entries in both directions, scan the
// folds across the threads of each segment (warp shuffles, then the warp
// totals through shared memory), and walk the entries again from the
// carried-in moments, reading queries and inserting sources.  Segments
// longer than a tile receive their carry from the aggregate pass
// (MODE == SCAN_AGG writes each tile's totals; k_carry_scan scans them).
// ROWS: the output pass stores into the level rows (A.rows); otherwise it adds
// into Y atomically (the batched products).
//
// Anchored fold and walk (FP32).  Within one thread's entries the moments
// may be kept relative to the thread's first entry in walk order instead of
// the current one, m~ = e^{+X} M with X the distance walked since that entry:
// a step by a gap G then only shifts the polynomial part (astep_group, no
// decay), a source enters scaled by e^{+X}, a query's read is scaled by
// e^{-X}, and the fold's total is scaled back by e^{-X} once.  e^{-X} is the
// running product of the entries' decays e^{-g} (the factors the plain walk
// multiplies by), e^{+X} its reciprocal.  A warp takes this form when each of
// its threads' gaps sum to at most kAnchorSpan; the step into the first entry
// is always the plain one.
// The arithmetic of one tile, from this thread's entries (q, gaps, offsets,
// their decays e^{-gap}, e^{-offset}, the first column's operands, and for
// lane 31 the gap into the entry after its last one and its decay) already in
// registers; entries past the level's end carry q = 0, zero gaps and offsets,
// unit decays and zero operands.
template <class R, int P, int NOFF, int KIND, int MODE, bool GEN = false, bool ROWS = true>
__device__ __forceinline__ void scan_compute(const ScanArgs<R> &A, const WorkItem wi, int r0, int r1,
                                             const uint32_t (&q)[kScanEPT], const R (&g)[kScanEPT],
                                             const R (&o)[NOFF > 0 ? NOFF : 1][kScanEPT],
                                             const R (&vpre)[kScanEPT], R gn31,
                                             const R (&eg)[kScanEPT], const R (&eo)[NOFF > 0 ? NOFF : 1][kScanEPT],
                                             R egn31) {
    using Tr = Traits<P, NOFF, KIND>;
    constexpr int GM = Tr::GM, CP = Tr::CP, SMM = Tr::SM, AG = Tr::AG, NCH = Tr::NCH;
    constexpr int NGP = Tr::NGP, NPT = Tr::NPT, NWC = Tr::NWC;
    constexpr int ND = Tr::NDIR, NDP = 2 / ND;  // directions per walk, direction passes
    constexpr int EPT = kScanEPT, NT = kScanThreads, NW = NT / 32;
    constexpr int LOG2EPT = (EPT == 8) ? 3 : (EPT == 4 ? 2 : (EPT == 16 ? 4 : 0));
    constexpr int NO = NOFF > 0 ? NOFF : 1;
    constexpr bool ANCH = std::is_same<R, float>::value && !GEN && NOFF < 2;
    static_assert((1 << LOG2EPT) == EPT, "EPT must be 4, 8 or 16");
    static_assert(EPT == 8, "vector loads assume 8 entries per thread");
    __shared__ R s_w[ND][NW][AG];
    __shared__ R s_pre[ND][NW][AG];  // SCAN_OUT: exclusive prefixes of the warp totals
    __shared__ R s_car[2][AG];       // SCAN_OUT, long segments: the tile's carries (both directions)

    const int64_t N = A.N;
    const int64_t base = (int64_t)wi.tile * kTile;
    const int log2S = wi.log2S;
    const int64_t S = int64_t(1) << log2S;
    const size_t lo = (size_t)wi.level * A.ldN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j0 = tid * EPT;
    const int64_t p0 = base + j0;
    const int nvalid = (int)(N - p0 < 0 ? 0 : (N - p0 > EPT ? EPT : N - p0));

    // gap into my last entry when walking backward: the next entry's forward gap
    R gn = __shfl_down_sync(0xffffffffu, g[0], 1);
    R egn = __shfl_down_sync(0xffffffffu, eg[0], 1);
    if (lane == 31) {
        gn = gn31;
        egn = egn31;
    }
    // the gaps between this thread's entries (the same in both walk directions)
    R span = R(0);
#pragma unroll
    for (int i = 1; i < EPT; ++i) span += g[i];
    bool fast = false;
    if constexpr (ANCH) fast = __all_sync(0xffffffffu, span <= R(kAnchorSpan));

    const bool multi = log2S < LOG2EPT;  // whole segments inside one thread
    const int G = multi ? 1 : (int)((S >> LOG2EPT) < (int64_t)NT ? (S >> LOG2EPT) : (int64_t)NT);
    const int GW = G < 32 ? G : 32;
    const bool is_long = S > kTile;

    R v[EPT];  // this column's operands; the next column's are gathered at the end of the loop body
#pragma unroll
    for (int i = 0; i < EPT; ++i) v[i] = vpre[i];
    for (int r = r0; r < r1; ++r) {
        R out[EPT];
#pragma unroll
        for (int i = 0; i < EPT; ++i) out[i] = R(0);
#pragma unroll 1
        for (int pq = 0; pq < NPT; ++pq) {
            const int pp = pq / NGP;       // channel pair
            const int a0 = NGP == 1 ? 0 : (pq % NGP) * Tr::GP;  // first offset-power group of the pass
            const int cA = pp;
            const int cB = NOFF == 0 ? 0 : (cA ^ (NCH - 1));
            // a long tile's carries (both directions), read now and parked in shared
            // memory before the first barrier below, so the load is hidden by the fold
            R cpf = R(0);
            if constexpr (MODE == SCAN_OUT) {
                if (is_long && tid < 2 * AG) {
                    const int cdir = tid / AG;
                    cpf = A.agg[((((size_t)wi.agg * 2 + cdir) * A.nrhs + r) * NPT + pq) * AG + (tid - cdir * AG)];
                }
            }
#pragma unroll
            for (int dp = 0; dp < NDP; ++dp) {
                R ex[ND][AG];
#pragma unroll
                for (int dd = 0; dd < ND; ++dd) set_identity<R, AG>(ex[dd]);
                if (!multi) {
                    // 1. fold this thread's entries
                    R inc[ND][AG];
#pragma unroll
                    for (int dd = 0; dd < ND; ++dd) set_identity<R, AG>(inc[dd]);
                    auto fold = [&](auto anch) {
                        constexpr bool AN = decltype(anch)::value;
                        R Rr[ND];
#pragma unroll
                        for (int dd = 0; dd < ND; ++dd) Rr[dd] = R(1);
#pragma unroll
                        for (int ii = 0; ii < EPT; ++ii) {
#pragma unroll
                            for (int dd = 0; dd < ND; ++dd) {
                                const int dir = ND == 2 ? dd : dp;
                                const int i = dir == 0 ? ii : EPT - 1 - ii;
                                const R gg = dir == 0 ? g[i] : (i < EPT - 1 ? g[i + 1] : gn);
                                const R ee = dir == 0 ? eg[i] : (i < EPT - 1 ? eg[i + 1] : egn);
                                R vi = v[i];
                                if constexpr (AN) {
                                    // the first entry starts from the identity: nothing to step
                                    if (ii > 0) {
                                        astep_all<R, P, SMM>(inc[dd] + 1, gg);
                                        Rr[dd] *= ee;
                                        vi *= rcp_approx(Rr[dd]);
                                    }
                                } else {
                                    step_all<R, P, SMM>(inc[dd] + 1, gg, ee);
                                    inc[dd][0] += gg;
                                }
                                const int role = NOFF == 0 ? 0 : (int)(q[i] >> (32 - NOFF));
                                R oi[NO], eoi[NO], w[NWC], u[NWC];
#pragma unroll
                                for (int k = 0; k < NO; ++k) {
                                    oi[k] = NOFF ? o[k][i] : R(0);
                                    eoi[k] = NOFF ? eo[k][i] : R(1);
                                }
                                pass_coef<R, P, NOFF, KIND, GEN>(a0, oi, eoi, w, u, A.cf);
                                add_pass<R, P, NOFF, KIND>(inc[dd] + 1, role == cA ? vi : R(0), w);
                                if constexpr (CP == 2) add_pass<R, P, NOFF, KIND>(inc[dd] + 1 + GM, role == cB ? vi : R(0), w);
                            }
                        }
                        if constexpr (AN) {
#pragma unroll
                            for (int dd = 0; dd < ND; ++dd) {
                                const int dir = ND == 2 ? dd : dp;
#pragma unroll
                                for (int m = 0; m < SMM; ++m) inc[dd][1 + m] *= Rr[dd];
                                inc[dd][0] = (dir == 0 ? g[0] : gn) + span;
                            }
                        }
                    };
                    if constexpr (ANCH) {
                        if (fast)
                            fold(std::true_type{});
                        else
                            fold(std::false_type{});
                    } else {
                        fold(std::false_type{});
                    }
                    // 2. inclusive scan over the threads of each segment (virtual lanes)
                    for (int dlt = 1; dlt < GW; dlt <<= 1) {
#pragma unroll
                        for (int dd = 0; dd < ND; ++dd) {
                            const int dir = ND == 2 ? dd : dp;
                            const int vlane = dir == 0 ? lane : 31 - lane;
                            R prev[AG];
#pragma unroll
                            for (int m = 0; m < AG; ++m)
                                prev[m] = dir == 0 ? __shfl_up_sync(0xffffffffu, inc[dd][m], dlt)
                                                   : __shfl_down_sync(0xffffffffu, inc[dd][m], dlt);
                            if ((vlane & (GW - 1)) >= dlt) compose_after<R, P, AG>(inc[dd], prev);
                        }
                    }
#pragma unroll
                    for (int dd = 0; dd < ND; ++dd) {
                        const int dir = ND == 2 ? dd : dp;
                        const int vlane = dir == 0 ? lane : 31 - lane;
                        R prev[AG];
#pragma unroll
                        for (int m = 0; m < AG; ++m)
                            prev[m] = dir == 0 ? __shfl_up_sync(0xffffffffu, inc[dd][m], 1)
                                               : __shfl_down_sync(0xffffffffu, inc[dd][m], 1);
                        if ((vlane & (GW - 1)) != 0) {
#pragma unroll
                            for (int m = 0; m < AG; ++m) ex[dd][m] = prev[m];
                        }
                    }
                    // 3. across warps: the warp totals go through shared memory;
                    //    AGG: one thread composes the tile's total; OUT: one warp
                    //    per direction scans them (segmented by the segment's
                    //    warps, after the tile's carry) and every thread composes
                    //    its warp's exclusive prefix
                    if (G > 32 || MODE == SCAN_AGG) {
#pragma unroll
                        for (int dd = 0; dd < ND; ++dd) {
                            const int dir = ND == 2 ? dd : dp;
                            const int vlane = dir == 0 ? lane : 31 - lane;
                            const int vwarp = dir == 0 ? warp : NW - 1 - warp;
                            if (vlane == 31) {
#pragma unroll
                                for (int m = 0; m < AG; ++m) s_w[dd][vwarp][m] = inc[dd][m];
                            }
                        }
                        if (MODE == SCAN_OUT && dp == 0 && is_long && tid < 2 * AG) {
                            const int cdir = tid / AG;
                            s_car[cdir][tid - cdir * AG] = cpf;
                        }
                        __syncthreads();
#pragma unroll
                        for (int dd = 0; dd < ND; ++dd) {
                            const int dir = ND == 2 ? dd : dp;
                            if (MODE == SCAN_AGG) {
                                if (tid == dd * 32) {  // the tile's total
                                    const size_t cslot = ((((size_t)wi.agg * 2 + dir) * A.nrhs + r) * NPT + pq) * AG;
                                    R run[AG];
                                    set_identity<R, AG>(run);
                                    for (int w2 = 0; w2 < NW; ++w2) {
                                        R t[AG];
#pragma unroll
                                        for (int m = 0; m < AG; ++m) t[m] = s_w[dd][w2][m];
                                        compose_after<R, P, AG>(t, run);
#pragma unroll
                                        for (int m = 0; m < AG; ++m) run[m] = t[m];
                                    }
#pragma unroll
                                    for (int m = 0; m < AG; ++m) A.agg[cslot + m] = run[m];
                                }
                            } else if (warp == dd) {
                                // Warp dd: the exclusive prefix of the warp totals (in walk
                                // order) within each segment's group of warps, by a
                                // segmented shuffle scan over lanes 0..NW-1, preceded by
                                // the tile's carry for a long segment.
                                const int grp = is_long ? NW : (G > 32 ? G / 32 : 1);
                                R x[AG];
#pragma unroll
                                for (int m = 0; m < AG; ++m) x[m] = lane < NW ? s_w[dd][lane][m] : R(0);
                                for (int dlt = 1; dlt < grp; dlt <<= 1) {
                                    R prev[AG];
#pragma unroll
                                    for (int m = 0; m < AG; ++m) prev[m] = __shfl_up_sync(0xffffffffu, x[m], dlt);
                                    if ((lane & (grp - 1)) >= dlt) compose_after<R, P, AG>(x, prev);
                                }
                                R e[AG];
#pragma unroll
                                for (int m = 0; m < AG; ++m) e[m] = __shfl_up_sync(0xffffffffu, x[m], 1);
                                if ((lane & (grp - 1)) == 0) set_identity<R, AG>(e);
                                if (is_long) {
                                    R carry[AG];
#pragma unroll
                                    for (int m = 0; m < AG; ++m) carry[m] = s_car[dir][m];
                                    compose_after<R, P, AG>(e, carry);
                                }
                                if (lane < NW) {
#pragma unroll
                                    for (int m = 0; m < AG; ++m) s_pre[dd][lane][m] = e[m];
                                }
                            }
                        }
                        if (MODE == SCAN_OUT) {
                            __syncthreads();
#pragma unroll
                            for (int dd = 0; dd < ND; ++dd) {
                                const int dir = ND == 2 ? dd : dp;
                                const int vwarp = dir == 0 ? warp : NW - 1 - warp;
                                R pre[AG];
#pragma unroll
                                for (int m = 0; m < AG; ++m) pre[m] = s_pre[dd][vwarp][m];
                                compose_after<R, P, AG>(ex[dd], pre);
                            }
                        }
                        __syncthreads();
                    }
                }
                if constexpr (MODE == SCAN_OUT) {
                    // 4. walk again from the carried-in moments; read, then insert
                    R st[ND][SMM];
#pragma unroll
                    for (int dd = 0; dd < ND; ++dd)
#pragma unroll
                        for (int m = 0; m < SMM; ++m) st[dd][m] = ex[dd][1 + m];
                    auto walk = [&](auto anch) {
                        constexpr bool AN = decltype(anch)::value;
                        R Rr[ND];
#pragma unroll
                        for (int dd = 0; dd < ND; ++dd) Rr[dd] = R(1);
#pragma unroll
                        for (int ii = 0; ii < EPT; ++ii) {
#pragma unroll
                            for (int dd = 0; dd < ND; ++dd) {
                                const int dir = ND == 2 ? dd : dp;
                                const int i = dir == 0 ? ii : EPT - 1 - ii;
                                if (multi) {
                                    const int jj = j0 + i;
                                    const bool seg_start = dir == 0 ? (jj & (S - 1)) == 0 : ((jj + 1) & (S - 1)) == 0;
                                    if (seg_start) {
#pragma unroll
                                        for (int m = 0; m < SMM; ++m) st[dd][m] = R(0);
                                    }
                                }
                                const R gg = dir == 0 ? g[i] : (i < EPT - 1 ? g[i + 1] : gn);
                                const R ee = dir == 0 ? eg[i] : (i < EPT - 1 ? eg[i + 1] : egn);
                                R vi = v[i];
                                if (AN && ii > 0) {
                                    astep_all<R, P, SMM>(st[dd], gg);
                                    Rr[dd] *= ee;
                                    vi *= rcp_approx(Rr[dd]);
                                } else {
                                    step_all<R, P, SMM>(st[dd], gg, ee);
                                }
                                R oi[NO], eoi[NO], w[NWC], u[NWC];
#pragma unroll
                                for (int k = 0; k < NO; ++k) {
                                    oi[k] = NOFF ? o[k][i] : R(0);
                                    eoi[k] = NOFF ? eo[k][i] : R(1);
                                }
                                pass_coef<R, P, NOFF, KIND, GEN>(a0, oi, eoi, w, u, A.cf);
                                // padding entries read into slots that are never stored and
                                // insert zero
                                if constexpr (CP == 1) {
                                    const R rd = read_pass<R, P, NOFF, KIND, GEN>(st[dd], u, A.cf);
                                    out[i] = AN ? fma(Rr[dd], rd, out[i]) : out[i] + rd;
                                    add_pass<R, P, NOFF, KIND>(st[dd], vi, w);
                                } else {
                                    const int role = (int)(q[i] >> (32 - NOFF));
                                    const bool sa = role == cA, sb = role == cB;
                                    R msel[GM];
#pragma unroll
                                    for (int m = 0; m < GM; ++m) msel[m] = sa ? st[dd][GM + m] : st[dd][m];
                                    R rd = read_pass<R, P, NOFF, KIND, GEN>(msel, u, A.cf);
                                    if constexpr (NOFF == 2) rd = (sa || sb) ? rd : R(0);
                                    out[i] = AN ? fma(Rr[dd], rd, out[i]) : out[i] + rd;
                                    add_pass<R, P, NOFF, KIND>(st[dd], sa ? vi : R(0), w);
                                    add_pass<R, P, NOFF, KIND>(st[dd] + GM, sb ? vi : R(0), w);
                                }
                            }
                        }
                    };
                    if constexpr (ANCH) {
                        if (fast)
                            walk(std::true_type{});
                        else
                            walk(std::false_type{});
                    } else {
                        walk(std::false_type{});
                    }
                }
            }
        }
        if constexpr (MODE == SCAN_OUT) {
#pragma unroll
            for (int i = 0; i < EPT; ++i) {
                if (i >= nvalid) continue;
                const size_t t = (size_t)(q[i] & 0x3fffffffu) * A.nrhs + r;
                if constexpr (ROWS)
                    A.rows[(size_t)wi.level * A.row_stride + t] = A.s2 * out[i];
                else
                    atomicAdd(A.Y + t, A.s2 * out[i]);
            }
        }
        if (r + 1 < r1) {
#pragma unroll
            for (int i = 0; i < EPT; ++i)
                v[i] = i < nvalid ? A.V[(size_t)(q[i] & 0x3fffffffu) * A.nrhs + r + 1] : R(0);
        }
    }
}

template <class R, int P, int NOFF, int KIND, int MODE, bool GEN = false, bool ROWS = true>
__device__ __forceinline__ void scan_tile(const ScanArgs<R> &A, const WorkItem wi, int r0, int r1) {
    constexpr int EPT = kScanEPT;
    constexpr int NO = NOFF > 0 ? NOFF : 1;
    static_assert(EPT == 8, "vector loads assume 8 entries per thread");

    const int64_t N = A.N;
    const int64_t base = (int64_t)wi.tile * kTile;
    const size_t lo = (size_t)wi.level * A.ldN;
    const int tid = threadIdx.x, lane = tid & 31;
    const int j0 = tid * EPT;
    const int64_t p0 = base + j0;
    const int nvalid = (int)(N - p0 < 0 ? 0 : (N - p0 > EPT ? EPT : N - p0));

    // ---- this thread's entries (the level stride keeps 8-entry groups aligned)
    uint32_t q[EPT];
    R g[EPT], o[NO][EPT];
    R vpre[EPT];  // the first column's operands (0 on padding: the fold inserts padding entries as
                  // zero-weight sources)
    if (nvalid > 0) {
        const uint4 *qp = reinterpret_cast<const uint4 *>(A.lv_q + lo + p0);
        const uint4 qa = qp[0], qb = qp[1];
        q[0] = qa.x; q[1] = qa.y; q[2] = qa.z; q[3] = qa.w;
        q[4] = qb.x; q[5] = qb.y; q[6] = qb.z; q[7] = qb.w;
        if constexpr (sizeof(R) == 4) {
            const float4 *gp = reinterpret_cast<const float4 *>(A.lv_dl + lo + p0);
            const float4 ga = gp[0], gb = gp[1];
            g[0] = ga.x; g[1] = ga.y; g[2] = ga.z; g[3] = ga.w;
            g[4] = gb.x; g[5] = gb.y; g[6] = gb.z; g[7] = gb.w;
#pragma unroll
            for (int k = 0; k < NOFF; ++k) {
                const float4 *op = reinterpret_cast<const float4 *>(A.lv_off + ((size_t)k * A.nlev) * A.ldN + lo + p0);
                const float4 oa = op[0], ob = op[1];
                o[k][0] = oa.x; o[k][1] = oa.y; o[k][2] = oa.z; o[k][3] = oa.w;
                o[k][4] = ob.x; o[k][5] = ob.y; o[k][6] = ob.z; o[k][7] = ob.w;
            }
        } else {
            const double2 *gp = reinterpret_cast<const double2 *>(A.lv_dl + lo + p0);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const double2 x = gp[h];
                g[2 * h] = x.x;
                g[2 * h + 1] = x.y;
            }
#pragma unroll
            for (int k = 0; k < NOFF; ++k) {
                const double2 *op = reinterpret_cast<const double2 *>(A.lv_off + ((size_t)k * A.nlev) * A.ldN + lo + p0);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const double2 x = op[h];
                    o[k][2 * h] = x.x;
                    o[k][2 * h + 1] = x.y;
                }
            }
        }
    }
    // the gate word is read while the entries are in flight and tested below
    const int gate_on = A.gate ? *A.gate : 1;
    if (nvalid < EPT) {  // past the level's end: identity steps, no role, no weight
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            if (i >= nvalid) {
                q[i] = 0;
                g[i] = R(0);
#pragma unroll
                for (int k = 0; k < NOFF; ++k) o[k][i] = R(0);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i)
        vpre[i] = (i < nvalid && r0 < r1) ? A.V[(size_t)(q[i] & 0x3fffffffu) * A.nrhs + r0] : R(0);
    R gn31 = R(0), egn31 = R(1);
    R eg[EPT], eo[NO][EPT];
    if (sizeof(R) == 8 && A.lv_edl) {
        // FP64: the stored decays (an FP64 exponential per entry and offset would
        // be most of the product's FP64 work on GB300); 1 past the level's end
        if (nvalid > 0) {
            const double2 *ep = reinterpret_cast<const double2 *>(A.lv_edl + lo + p0);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const double2 x = ep[h];
                eg[2 * h] = (R)x.x;
                eg[2 * h + 1] = (R)x.y;
            }
#pragma unroll
            for (int k = 0; k < NOFF; ++k) {
                const double2 *op = reinterpret_cast<const double2 *>(A.lv_eoff + ((size_t)k * A.nlev) * A.ldN + lo + p0);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const double2 x = op[h];
                    eo[k][2 * h] = (R)x.x;
                    eo[k][2 * h + 1] = (R)x.y;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            if (i >= nvalid) {
                eg[i] = R(1);
#pragma unroll
                for (int k = 0; k < NOFF; ++k) eo[k][i] = R(1);
            }
        }
        if (lane == 31) {
            const int64_t pn = p0 + EPT;
            if (pn < N) {
                gn31 = A.lv_dl[lo + pn];
                egn31 = A.lv_edl[lo + pn];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            eg[i] = exp_neg<R>(g[i]);
#pragma unroll
            for (int k = 0; k < NOFF; ++k) eo[k][i] = exp_neg<R>(o[k][i]);
        }
        if (lane == 31) {
            const int64_t pn = p0 + EPT;
            gn31 = pn < N ? A.lv_dl[lo + pn] : R(0);
            egn31 = exp_neg<R>(gn31);
        }
    }
    if (!gate_on) return;  // uniform over the CTA
    scan_compute<R, P, NOFF, KIND, MODE, GEN, ROWS>(A, wi, r0, r1, q, g, o, vpre, gn31, eg, eo, egn31);
}

// the work item of list position k (block rows of ntiles tiles per level, the
// long-segment levels first; their tiles own aggregate slot k)
template <class R>
__device__ __forceinline__ WorkItem item_of(const ScanArgs<R> &A, int k) {
    const int slot = k / A.ntiles;
    const uint32_t lm = __ldg(A.lv_map + slot);
    WorkItem wi;
    wi.level = (int)(lm & 0xffffu);
    wi.log2S = (int)(lm >> 16);
    wi.tile = k - slot * A.ntiles;
    wi.agg = k < A.n_long ? k : -1;
    wi.seg_tile0 = 0;
    wi.seg_ntiles = 0;
    return wi;
}

template <class R, int P, int NOFF, int KIND, int MODE, bool GEN = false>
__global__ void __launch_bounds__(kScanThreads, GEN ? 1 : (sizeof(R) == 8 ? FGK_SCAN_MINB_F64 : FGK_SCAN_MINB))
    k_level_scan(ScanArgs<R> A) {
    scan_tile<R, P, NOFF, KIND, MODE, GEN>(A, item_of(A, blockIdx.x), 0, A.nrhs);
}

// one warp: exclusive carries of one long segment (tiles a0 .. a0+nt-1 of the
// aggregate slots) for direction dir, right-hand side r and pass pq
template <class R, int P, int NOFF, int KIND>
__device__ __forceinline__ void carry_warp(const R *__restrict__ agg, R *__restrict__ carry, int a0, int nt, int dir,
                                           int r, int pq, int nrhs) {
    using Tr = Traits<P, NOFF, KIND>;
    constexpr int AG = Tr::AG, NPT = Tr::NPT;
    const int lane = threadIdx.x & 31;
    R run[AG];
    set_identity<R, AG>(run);
    for (int k0 = 0; k0 < nt; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < nt;
        const int slot = a0 + (dir == 0 ? k : nt - 1 - k);
        const size_t off = ((((size_t)(valid ? slot : a0) * 2 + dir) * nrhs + r) * NPT + pq) * AG;
        R inc[AG];
#pragma unroll
        for (int m = 0; m < AG; ++m) inc[m] = valid ? agg[off + m] : R(0);
        for (int dlt = 1; dlt < 32; dlt <<= 1) {
            R prev[AG];
#pragma unroll
            for (int m = 0; m < AG; ++m) prev[m] = __shfl_up_sync(0xffffffffu, inc[m], dlt);
            if (lane >= dlt) compose_after<R, P, AG>(inc, prev);
        }
        R ex[AG];
#pragma unroll
        for (int m = 0; m < AG; ++m) ex[m] = __shfl_up_sync(0xffffffffu, inc[m], 1);
        if (lane == 0) set_identity<R, AG>(ex);
        compose_after<R, P, AG>(ex, run);
        if (valid) {
#pragma unroll
            for (int m = 0; m < AG; ++m) carry[off + m] = ex[m];
        }
        R last[AG];
#pragma unroll
        for (int m = 0; m < AG; ++m) last[m] = __shfl_sync(0xffffffffu, inc[m], 31);
        compose_after<R, P, AG>(last, run);
#pragma unroll
        for (int m = 0; m < AG; ++m) run[m] = last[m];
    }
}

// Exclusive scan of the tile aggregates of every long segment in both
// directions: one warp per (segment, direction, rhs, pass).
template <class R, int P, int NOFF, int KIND>
__global__ void k_carry_scan(const R *__restrict__ agg, R *__restrict__ carry, const int32_t *__restrict__ segs,
                             int nseg, int nrhs, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    constexpr int NPT = Traits<P, NOFF, KIND>::NPT;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t total = (int64_t)nseg * 2 * nrhs * NPT;
    if (wid >= total) return;  // uniform per warp
    const int pq = (int)(wid % NPT);
    const int r = (int)((wid / NPT) % nrhs);
    const int dir = (int)((wid / ((int64_t)NPT * nrhs)) % 2);
    const int sg = (int)(wid / ((int64_t)NPT * nrhs * 2));
    carry_warp<R, P, NOFF, KIND>(agg, carry, segs[2 * sg], segs[2 * sg + 1], dir, r, pq, nrhs);
}

template <class R>
__global__ void k_diag_init(const R *__restrict__ V, int64_t n, R s2, R *__restrict__ Y, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Y[i] = s2 * V[i];
}

// S5: Y = base + sum over levels of the level rows, the levels added in
// ascending order (the same order on every call, so a product is
// reproducible bit for bit); base = s2 V (the self-pairs, which no level
// holds) when V is given, else the Y already there.  Rows are stride apart
// (a multiple of 16 bytes), so each thread reads 16 bytes of every level at
// once: the independent loads of all levels are in flight together.
template <class R>
__global__ void k_level_sum(const R *__restrict__ rows, int nlev, int64_t n, int64_t stride,
                            const R *__restrict__ V, R s2, R *__restrict__ Y, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    constexpr int W = 16 / sizeof(R);  // elements per 16-byte load
    using Vec = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    const int64_t nv = n / W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
        R acc[W];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = V ? s2 * V[t * W + w] : Y[t * W + w];
#pragma unroll 6
        for (int l = 0; l < nlev; ++l) {
            const Vec x = reinterpret_cast<const Vec *>(rows + (size_t)l * stride)[t];
            const R *xv = reinterpret_cast<const R *>(&x);
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] += xv[w];
        }
#pragma unroll
        for (int w = 0; w < W; ++w) Y[t * W + w] = acc[w];
    }
    // the tail past the last full vector
    for (int64_t e = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        R acc = V ? s2 * V[e] : Y[e];
        for (int l = 0; l < nlev; ++l) acc += rows[(size_t)l * stride + e];
        Y[e] = acc;
    }
}

// Scratch of one product, in elements of the scan precision: the level rows
// (n_levels x N x nrhs), then the tile aggregates and the tile carries of
// the long segments (n_long tiles x 2 directions x nrhs x passes x aggregate
// size each).  The pass count and aggregate size follow Traits.
inline size_t scan_pass_elems(int P, int noff, int kind) {
    int na = 1;
    if (kind == FGK_PRODUCT && noff > 0 && P > 1)
        for (int k = 0; k < noff; ++k) na *= P;
    const size_t cp = noff == 0 ? 1 : 2;
    const size_t npass = noff == 2 ? 2 : 1;
    const size_t gp = (na > 1 && cp * na * P > 12) ? 1 : na;
    const size_t ngp = na / gp;
    const size_t ag = 1 + cp * gp * P;
    return npass * ngp * ag;
}
// level rows: stride = N nrhs rounded up to 16 bytes' worth of elements
inline size_t scan_row_stride(const Plan *p, int nrhs) { return ((size_t)p->N * nrhs + 3) / 4 * 4; }
inline size_t scan_rows_elems(const Plan *p, int nrhs) {
    return ((size_t)p->nlev * scan_row_stride(p, nrhs) + 63) / 64 * 64;
}
inline size_t scan_ws_elems_for(const Plan *p, int nrhs, int P, int kind) {
    const size_t slot = (size_t)2 * nrhs * scan_pass_elems(P, p->d - 1, kind);
    return scan_rows_elems(p, nrhs) + 2 * (size_t)p->n_long * slot + 64;
}

// One product's level scans: aggregate pass and carry scan over the long
// segments, output pass over every tile (each writing its level row), then
// the fixed-order level sum into Yq.  init_diag: Yq = s2 Vq + levels; else
// Yq += levels.
// preload: only make the runtime load the kernels this product would launch
// (their attributes are queried), so that a later product loads nothing.
template <class R, int P, int NOFF, int KIND, int MODE, bool GEN>
int launch_scan(const ScanArgs<R> &A, int nitems, cudaStream_t s) {
    k_level_scan<R, P, NOFF, KIND, MODE, GEN><<<nitems, kScanThreads, 0, s>>>(A);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

template <class R, int P, int NOFF, int KIND, bool GEN = false>
int run_levels(Plan *p, const R *Vq, int nrhs, R *Yq, R *ws, cudaStream_t s, const int *gate, bool init_diag,
               const double (*cf)[kMaxCoef] = nullptr, bool preload = false) {
    using Tr = Traits<P, NOFF, KIND>;
    if (preload) {
        // Also make sure the context's per-thread stack holds the largest
        // frame (spilled registers) of these kernels: a launch whose frame
        // exceeds cudaLimitStackSize (1 KiB by default) is not safe.
        cudaFuncAttributes fa[4];
        FGK_CUDA(cudaFuncGetAttributes(&fa[0], k_level_scan<R, P, NOFF, KIND, SCAN_AGG, GEN>));
        FGK_CUDA(cudaFuncGetAttributes(&fa[1], k_level_scan<R, P, NOFF, KIND, SCAN_OUT, GEN>));
        FGK_CUDA(cudaFuncGetAttributes(&fa[2], k_carry_scan<R, P, NOFF, KIND>));
        FGK_CUDA(cudaFuncGetAttributes(&fa[3], k_level_sum<R>));
        size_t need = 0, have = 0;
        for (const auto &a : fa) need = std::max(need, a.localSizeBytes);
        FGK_CUDA(cudaDeviceGetLimit(&have, cudaLimitStackSize));
        if (need > have) FGK_CUDA(cudaDeviceSetLimit(cudaLimitStackSize, (need + 255) / 256 * 256));
        return FGK_OK;
    }
    ScanArgs<R> A;
    for (int k = 0; k < kMaxD; ++k)
        for (int q = 0; q < kMaxCoef; ++q) A.cf[k][q] = cf ? (R)cf[k][q] : R(0);
    A.lv_q = p->lv_q;
    A.lv_dl = std::is_same<R, float>::value ? (const R *)p->lv_dl32 : (const R *)p->lv_dl64;
    A.lv_off = std::is_same<R, float>::value ? (const R *)p->lv_off32 : (const R *)p->lv_off64;
    A.lv_edl = std::is_same<R, float>::value ? nullptr : (const R *)p->lv_edl64;
    A.lv_eoff = std::is_same<R, float>::value ? nullptr : (const R *)p->lv_eoff64;
    A.N = p->N;
    A.ldN = p->ldN;
    A.nlev = p->nlev;
    A.V = Vq;
    A.nrhs = nrhs;
    A.Y = Yq;
    A.rows = ws;
    A.row_stride = (int64_t)scan_row_stride(p, nrhs);
    A.s2 = (R)p->s2;
    A.err = p->dev_err;
    A.gate = gate;
    A.lv_map = p->lv_map;
    A.ntiles = p->ntiles;
    A.n_long = p->n_long;
    const size_t per_slot = (size_t)2 * nrhs * Tr::NPT * Tr::AG;
    R *agg = ws + scan_rows_elems(p, nrhs);
    R *carry = agg + (size_t)p->n_long * per_slot;
    if (p->n_long > 0) {
        A.items = p->long_items;
        A.agg = agg;
        FGK_TRY((launch_scan<R, P, NOFF, KIND, SCAN_AGG, GEN>(A, p->n_long, s)));
        const int64_t nthr = (int64_t)p->n_long_segments * 2 * nrhs * Tr::NPT * 32;
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
        FGK_TRY((launch_scan<R, P, NOFF, KIND, SCAN_OUT, GEN>(A, p->n_items, s)));
        if (e0) {
            FGK_CUDA(cudaEventRecord(e1, s));
            scan_timing_record(e0, e1);
        }
    }
    const int64_t n = p->N * nrhs;
    const unsigned blocks = (unsigned)std::min<int64_t>(grid_for(n / (16 / sizeof(R)) + 1, 256), 152 * 8);
    k_level_sum<R><<<blocks, 256, 0, s>>>(ws, p->nlev, n, (int64_t)scan_row_stride(p, nrhs),
                                          init_diag ? Vq : nullptr, (R)p->s2, Yq, gate);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

// the kernel's own scans: nu = 1/2 or d = 1 make both kinds the same kernel
inline int scan_kind(const Plan *p) { return (p->P == 1 || p->d == 1) ? FGK_L1 : p->kind; }

template <class R>
size_t scan_ws_elems(const Plan *p, int nrhs) {
    return scan_ws_elems_for(p, nrhs, p->P, scan_kind(p));
}

// Matérn coefficients c_p of k(r) = sum_p c_p r^p e^{-r} in scaled units
// (eqs. matern_1_2 ... matern_9_2; eq. matern_explicit gives them for any
// half-integer nu: c_p = (P-1)! (2P-2-p)! 2^p / ((2P-2)! p! (P-1-p)!))
inline void matern_coef(int P, double *c) {
    for (int q = 0; q < kMaxCoef; ++q) c[q] = 0.0;
    auto fact = [](int n) {
        double f = 1.0;
        for (int k = 2; k <= n; ++k) f *= k;
        return f;
    };
    for (int q = 0; q < P; ++q)
        c[q] = fact(P - 1) * fact(2 * P - 2 - q) * std::ldexp(1.0, q) / (fact(2 * P - 2) * fact(q) * fact(P - 1 - q));
}

// dispatch over (P, d-1, kind).  nu <= 5/2: the scans with the coefficients
// compiled in; nu = 7/2, 9/2: the generic-coefficient scans (fgk_dscan.cuh)
// with c in every factor.
template <class R>
int run_levels_gen_dispatch(Plan *p, int P4, int kind, const R *Vq, int nrhs, R *Yq, R *ws, cudaStream_t s,
                            const double (*cf)[kMaxCoef], const int *gate, bool init_diag, bool preload = false);

template <class R>
int run_levels_dispatch(Plan *p, const R *Vq, int nrhs, R *Yq, R *ws, cudaStream_t s, const int *gate,
                        bool init_diag, bool preload = false) {
    const int P = p->P, NOFF = p->d - 1;
    const int kind = scan_kind(p);
    if (P > 3) {
        double cf[kMaxD][kMaxCoef];
        for (int k = 0; k < kMaxD; ++k) matern_coef(P, cf[k]);
        return run_levels_gen_dispatch<R>(p, P, kind, Vq, nrhs, Yq, ws, s, cf, gate, init_diag, preload);
    }
    const int key = (P * 3 + NOFF) * 2 + kind;
    switch (key) {
#define FGK_CASE(PP, NO, KK)          \
    case (PP * 3 + NO) * 2 + KK:      \
        return run_levels<R, PP, NO, KK>(p, Vq, nrhs, Yq, ws, s, gate, init_diag, nullptr, preload);
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
