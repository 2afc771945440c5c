// The preconditioner of the CG solve (App. A.3): P = L L^T + sigma^2 I with L
// the rank-k pivoted Cholesky factor of K (Harbrecht et al., cited there),
// applied by the Woodbury formula, with log det P by Sylvester's theorem.
//
// Build (once per plan and sigma^2).  The residual diagonal starts at
// K_ii = s2.  Step m takes as pivot the largest residual diagonal entry (ties:
// the smallest original point index), forms the column of K at the pivot
// from the scaled coordinates, subtracts what columns 0..m-1 already explain
// (sum_t L_t L_t[pivot]), divides by the square root of the pivot's residual
// and lowers the residual diagonal by the square of the new column.  One
// launch per step: each CTA first reduces the previous step's per-CTA
// maxima (so every CTA agrees on the pivot without a host round trip), then
// updates its rows and publishes its own maximum.  A step whose largest
// residual is at most 1e-12 s2 (numerically exhausted; the paper leaves the
// case open) records the realised rank and changes nothing.
// L is stored in FP32 (columns of N entries, q order), and each new column
// is rounded to FP32 before anything else uses it: the later columns and the
// residual diagonal are those of the stored factor, so the factor is the
// exact pivoted-Cholesky recurrence of its own stored columns (the rounding of
// a column, ~2^-24 of it, is taken up by the next ones, far below the
// residual the rank leaves).  The sums of the build are float pairs of exact
// products (two-product, two-sum), the divisions and the residual diagonal
// FP64.  The apply and the Woodbury matrix I + L^T L / sigma^2 use the same
// FP32 values, so P is exactly the SPD matrix L L^T + sigma^2 I the apply
// inverts.
//
// Apply (Z = P^{-1} R, every CG iteration, inside the captured graph):
//   t = L^T R          k_pc_ltr (persistent CTAs, per-CTA partials) + k_pc_tsum
//   c = C^{-1} t / s^4  k_pc_cmul (C^{-1} formed at build from the Cholesky
//                       factor of C: a matrix-vector product spread over
//                       warps instead of two latency-bound triangular solves)
//   Z = R / s^2 - L c   k_pc_apply (+ per-CTA partial sums of R .* Z)
// Both passes over L stream it through shared memory with TMA tensor copies.
// which is the Woodbury form P^{-1} R = R/s^2 - L (I + L^T L/s^2)^{-1} L^T R / s^4.
// The two passes over L are FP32 arithmetic: GB300 issues FP64 at a small
// fraction of its FP32 rate, and one FP64 multiply-add per element of L made
// them FP64-bound (about 30x slower than its memory traffic).  FP64 accuracy
// is kept with error-free transformations: FP64 operands split into float
// pairs (hi + lo), products of floats made exact by a fused multiply-add
// (two-product), and running sums carried as float pairs by Knuth's
// two-sum; each block's pair is added in FP64.
#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime's driver entry point)

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "fgk_internal.cuh"

namespace fgk {

namespace {

constexpr int kPcThreads = 256;
constexpr int kPcMaxRank = 1024;
constexpr int kGramTile = 32;  // Gram tile side (columns)
constexpr double kExhausted = 1e-12;  // stop once the residual diagonal is at most this x s2

struct PivPart {
    double val;
    int64_t orig;
    int64_t q;
};

// an integer key with the order of the doubles (negative values flipped
// except for the sign bit; -0 sorts just below +0), so that the pivot
// comparisons, a dozen per row of every step, stay off GB300's slow FP64 pipe
__device__ __forceinline__ long long piv_key(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ bool piv_better(const PivPart &a, const PivPart &b) {
    const long long ka = piv_key(a.val), kb = piv_key(b.val);
    return ka > kb || (ka == kb && a.orig < b.orig);
}

__device__ __forceinline__ PivPart piv_none() { return PivPart{-INFINITY, INT64_MAX, -1}; }

// block-wide best of one PivPart per thread; result valid in every thread
__device__ __forceinline__ PivPart block_best(PivPart v) {
    __shared__ PivPart s_w[kPcThreads / 32];
    __shared__ PivPart s_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PivPart u;
        u.val = __shfl_xor_sync(0xffffffffu, v.val, o);
        u.orig = __shfl_xor_sync(0xffffffffu, v.orig, o);
        u.q = __shfl_xor_sync(0xffffffffu, v.q, o);
        if (piv_better(u, v)) v = u;
    }
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        PivPart b = s_w[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (piv_better(s_w[w], b)) b = s_w[w];
        s_out = b;
    }
    __syncthreads();
    const PivPart r = s_out;
    __syncthreads();
    return r;
}

// unit-lengthscale Matern polynomial part: k(r) = poly(r) e^{-r} with
// poly(r) = sum_{p<P} c_p r^p, c = (1), (1, 1), (1, 1, 1/3), (1, 1, 2/5, 1/15),
// (1, 1, 3/7, 2/21, 1/105) for nu = 1/2 .. 9/2 (eqs. matern_1_2 .. matern_9_2
// in scaled units; eq. matern_explicit), by Horner's rule
__device__ __forceinline__ double matern_poly(int two_nu, double r) {
    if (two_nu == 1) return 1.0;
    if (two_nu == 3) return 1.0 + r;
    if (two_nu == 5) return 1.0 + r * (1.0 + r * (1.0 / 3.0));
    if (two_nu == 7) return 1.0 + r * (1.0 + r * (2.0 / 5.0 + r * (1.0 / 15.0)));
    return 1.0 + r * (1.0 + r * (3.0 / 7.0 + r * (2.0 / 21.0 + r * (1.0 / 105.0))));
}

struct KernArgs {
    const double *x0, *x1, *x2;  // scaled coordinates in q order
    int d, two_nu, kind;
    double s2;
    // e^{+x} and e^{-x} of each scaled coordinate (block k of N per
    // dimension), 0 where |x| > kExpTableMax; NULL: no tables
    const double *ep, *em;
    int64_t N;
};

// |x| up to which the tables hold e^{+-x}: e^{700} < DBL_MAX and e^{-700} >
// DBL_MIN, so neither factor nor their product (at most 1) overflows
constexpr double kExpTableMax = 700.0;

__global__ void k_pc_exptab(KernArgs ka, double *__restrict__ ep, double *__restrict__ em) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ka.N) return;
    for (int k = 0; k < ka.d; ++k) {
        const double x = (k == 0 ? ka.x0 : (k == 1 ? ka.x1 : ka.x2))[i];
        const bool in = fabs(x) <= kExpTableMax;
        ep[(size_t)k * ka.N + i] = in ? exp(x) : 0.0;
        em[(size_t)k * ka.N + i] = in ? exp(-x) : 0.0;
    }
}

// K(x_i, x_p): both kinds share the exponential e^{-sum_k |u_k|} (L1: of the
// summed distance; product: the product of the per-dimension factors).  With
// the tables, e^{-|x_i - x_p|} = e^{-x_i} e^{+x_p} (x_i >= x_p) or e^{+x_i}
// e^{-x_p}: d multiplications instead of an FP64 exponential, whose long
// instruction sequence on GB300's FP64 pipe bounds each pivot step's row pass.
// pex[k] = e^{+x_p,k}, pex[3 + k] = e^{-x_p,k}; tab: the pivot is inside the
// tables (rows outside them take the exponential).
__device__ __forceinline__ double kern_q(const KernArgs &k, int64_t i, const double *xp, const double *pex,
                                         bool tab) {
    const double d0 = k.x0[i] - xp[0];
    const double d1 = k.d > 1 ? k.x1[i] - xp[1] : 0.0;
    const double d2 = k.d > 2 ? k.x2[i] - xp[2] : 0.0;
    const double u0 = fabs(d0), u1 = fabs(d1), u2 = fabs(d2);
    double e;
    bool done = false;
    if (tab) {
        // the signs and the table's zero markers tested on the integer pipe
        const double em0 = k.em[i], ep0 = k.ep[i];
        double f = __double2hiint(d0) >= 0 ? em0 * pex[0] : ep0 * pex[3];
        bool in = __double_as_longlong(em0) != 0;
        if (k.d > 1) {
            const double em1 = k.em[k.N + i], ep1 = k.ep[k.N + i];
            f *= __double2hiint(d1) >= 0 ? em1 * pex[1] : ep1 * pex[4];
            in = in && __double_as_longlong(em1) != 0;
        }
        if (k.d > 2) {
            const double em2 = k.em[2 * k.N + i], ep2 = k.ep[2 * k.N + i];
            f *= __double2hiint(d2) >= 0 ? em2 * pex[2] : ep2 * pex[5];
            in = in && __double_as_longlong(em2) != 0;
        }
        e = f;
        done = in;
    }
    if (!done) e = exp(-(u0 + u1 + u2));
    if (k.d == 1 || k.kind == FGK_L1) return k.s2 * matern_poly(k.two_nu, u0 + u1 + u2) * e;
    double v = matern_poly(k.two_nu, u0) * matern_poly(k.two_nu, u1);
    if (k.d == 3) v *= matern_poly(k.two_nu, u2);
    return k.s2 * v * e;
}

// float-pair arithmetic (value = hi + lo): Knuth's two-sum and the
// fused-multiply-add two-product, both exact
struct F2 {
    float hi, lo;
};

// (the _rn intrinsics are never contracted into fused multiply-adds, which
// would break the exactness these steps rely on)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += l * (xh + xl), l a float, x given as a float pair
__device__ __forceinline__ void f2_fma(F2 &acc, float l, float xh, float xl) {
    const float p = __fmul_rn(l, xh);
    const float pe = fmaf(l, xh, -p);  // l * xh = p + pe exactly
    float sum, err;
    two_sum(acc.hi, p, sum, err);
    acc.hi = sum;
    acc.lo += err + fmaf(l, xl, pe);
}

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    F2 r;
    float e;
    two_sum(a.hi, b.hi, r.hi, e);
    r.lo = e + a.lo + b.lo;
    return r;
}

__device__ __forceinline__ void split_f2(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

__global__ void k_pc_init(int64_t N, double s2, const int32_t *__restrict__ perm0, double *__restrict__ dres,
                          PivPart *__restrict__ part) {
    PivPart best = piv_none();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        dres[i] = s2;
        const PivPart c{s2, (int64_t)perm0[i], i};
        if (piv_better(c, best)) best = c;
    }
    best = block_best(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// step m of the pivoted Cholesky (see the file comment)
__global__ void __launch_bounds__(kPcThreads, 3) k_pc_step(int m, int64_t N, int64_t ldN, KernArgs ka,
                                                          const int32_t *__restrict__ perm0,
                          const PivPart *__restrict__ prev, int nprev, PivPart *__restrict__ next,
                          float *__restrict__ L, double *__restrict__ dres, int32_t *__restrict__ piv_q,
                          int *__restrict__ rank, double floor) {
    __shared__ float s_lp[kPcMaxRank];
    __shared__ double s_xp[3];
    __shared__ double s_pex[6];  // the pivot's e^{+x_k}, e^{-x_k}
    __shared__ double s_isq;     // 1 / sqrt(the pivot's residual)
    PivPart best = piv_none();
    for (int b = threadIdx.x; b < nprev; b += blockDim.x)
        if (piv_better(prev[b], best)) best = prev[b];
    best = block_best(best);
    if (!(best.val > floor)) {  // exhausted: rank m, nothing changes from here on
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) atomicMin(rank, m);
            next[blockIdx.x] = best;
        }
        return;
    }
    const int64_t piv = best.q;
    if (blockIdx.x == 0 && threadIdx.x == 0) piv_q[m] = (int32_t)piv;
    for (int t = threadIdx.x; t < m; t += blockDim.x) s_lp[t] = L[(size_t)t * ldN + piv];
    if (threadIdx.x == 0) {
        s_xp[0] = ka.x0[piv];
        s_xp[1] = ka.d > 1 ? ka.x1[piv] : 0.0;
        s_xp[2] = ka.d > 2 ? ka.x2[piv] : 0.0;
        for (int k = 0; k < 3; ++k) {
            s_pex[k] = (ka.ep && k < ka.d) ? ka.ep[(size_t)k * ka.N + piv] : 1.0;
            s_pex[3 + k] = (ka.em && k < ka.d) ? ka.em[(size_t)k * ka.N + piv] : 1.0;
        }
        // one square root and one division per CTA, not per thread: both are long
        // dependent sequences on GB300's FP64 pipe
        s_isq = 1.0 / sqrt(best.val);
    }
    __syncthreads();
    const bool tab = ka.ep != nullptr && s_pex[3] != 0.0 && s_pex[4] != 0.0 && s_pex[5] != 0.0;
    const double isq = s_isq;
    PivPart mine = piv_none();
    // two consecutive rows per thread (8-byte vector loads of L; the column
    // stride ldN is a multiple of 64, so row i0 + 1 < ldN is always inside the
    // column, and only rows below N are written)
    for (int64_t i0 = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i0 < N;
         i0 += 2 * (int64_t)gridDim.x * blockDim.x) {
        const bool two = i0 + 1 < N;
        // sum_t L_t[i] L_t[pivot]: each product of two FP32 values made exact
        // by the two-product, the running sums float pairs (two per row, even
        // and odd t, so that consecutive terms do not wait on each other)
        F2 acc0{0.f, 0.f}, acc1{0.f, 0.f}, acc0b{0.f, 0.f}, acc1b{0.f, 0.f};
        int t = 0;
#pragma unroll 4
        for (; t + 1 < m; t += 2) {
            const float2 a = *reinterpret_cast<const float2 *>(L + (size_t)t * ldN + i0);
            const float2 b = *reinterpret_cast<const float2 *>(L + (size_t)(t + 1) * ldN + i0);
            const float ph = s_lp[t], ph1 = s_lp[t + 1];
            f2_fma(acc0, a.x, ph, 0.f);
            f2_fma(acc1, a.y, ph, 0.f);
            f2_fma(acc0b, b.x, ph1, 0.f);
            f2_fma(acc1b, b.y, ph1, 0.f);
        }
        if (t < m) {
            const float2 a = *reinterpret_cast<const float2 *>(L + (size_t)t * ldN + i0);
            f2_fma(acc0, a.x, s_lp[t], 0.f);
            f2_fma(acc1, a.y, s_lp[t], 0.f);
        }
        acc0 = f2_add(acc0, acc0b);
        acc1 = f2_add(acc1, acc1b);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            const int64_t i = i0 + h;
            const F2 acc = h == 0 ? acc0 : acc1;
            const double kv = kern_q(ka, i, s_xp, s_pex, tab);
            const double dot = (double)acc.hi + (double)acc.lo;
            const float lf = (float)((kv - dot) * isq);
            L[(size_t)m * ldN + i] = lf;
            const double l = (double)lf;  // the stored value from here on
            const double dn = dres[i] - l * l;
            dres[i] = dn;
            const PivPart c{dn, (int64_t)perm0[i], i};
            if (piv_better(c, mine)) mine = c;
        }
    }
    mine = block_best(mine);
    if (threadIdx.x == 0) next[blockIdx.x] = mine;
}

// partial Gram blocks: Gp[z][a][b] = sum over rows of chunk z of L32[a][i] L32[b][i]
// (products of FP32 values are exact; float-pair sums over 256 rows, then
// FP64).  A CTA takes a 32 x 32 tile (ta <= tb) of column pairs, each thread
// a 2 x 2 block of it, over rows staged 64 at a time in shared memory: two
// 8-byte shared loads feed four exact multiply-adds.
constexpr int kGramRows = 64;   // rows staged per round
constexpr int kGramFlush = 4;   // rounds between the FP64 flushes of the float-pair sums

// acc += a * b, the product exact (two-product), the sum a float pair
__device__ __forceinline__ void f2_mac(F2 &acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);  // a * b = p + pe exactly
    float sum, err;
    two_sum(acc.hi, p, sum, err);
    acc.hi = sum;
    acc.lo += err + pe;
}

__global__ void __launch_bounds__(kPcThreads) k_pc_gram(const float *__restrict__ L, int64_t ldN, int64_t N, int r,
                                                        int64_t rows_per_z, double *__restrict__ Gp) {
    __shared__ __align__(16) float sa[kGramRows][kGramTile + 2];
    __shared__ __align__(16) float sb[kGramRows][kGramTile + 2];
    const int ta = blockIdx.x, tb = blockIdx.y;
    if (ta > tb) return;
    const int z = blockIdx.z;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;  // 16 x 16 threads, 2 x 2 entries each
    const int64_t i0 = (int64_t)z * rows_per_z, i1 = min(N, i0 + rows_per_z);
    double tot[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    F2 f[2][2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
    int round = 0;
    for (int64_t c0 = i0; c0 < i1; c0 += kGramRows, ++round) {
        for (int e = threadIdx.x; e < kGramTile * kGramRows; e += blockDim.x) {
            const int col = e / kGramRows, row = e % kGramRows;  // consecutive threads: consecutive rows
            const int64_t i = c0 + row;
            const int ca = ta * kGramTile + col, cb = tb * kGramTile + col;
            sa[row][col] = (i < i1 && ca < r) ? L[(size_t)ca * ldN + i] : 0.f;
            sb[row][col] = (i < i1 && cb < r) ? L[(size_t)cb * ldN + i] : 0.f;
        }
        __syncthreads();
        const int n = (int)(i1 - c0 < kGramRows ? i1 - c0 : kGramRows);
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
            const float2 a = *reinterpret_cast<const float2 *>(&sa[k][ty * 2]);
            const float2 b = *reinterpret_cast<const float2 *>(&sb[k][tx * 2]);
            f2_mac(f[0][0], a.x, b.x);
            f2_mac(f[0][1], a.x, b.y);
            f2_mac(f[1][0], a.y, b.x);
            f2_mac(f[1][1], a.y, b.y);
        }
        __syncthreads();
        if (round % kGramFlush == kGramFlush - 1 || c0 + kGramRows >= i1) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    tot[u][v] += (double)f[u][v].hi + (double)f[u][v].lo;
                    f[u][v] = F2{0.f, 0.f};
                }
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int a = ta * kGramTile + ty * 2 + u, b = tb * kGramTile + tx * 2 + v;
            if (a < r && b < r) Gp[((size_t)z * r + a) * r + b] = tot[u][v];
        }
}

// C = I + G / sigma2 (G summed over the z partials, mirrored) and its lower
// Cholesky factor F (row-major r x r, upper part untouched), blocked and
// right-looking over the whole GPU: per panel of kCholB columns, the
// diagonal block is factored by one CTA (k_chol_diag), the rows below it are
// solved against that block (k_chol_panel, one thread per row), and the
// trailing lower triangle takes the panel's rank-kCholB update in 32 x 32
// tiles (k_chol_update, one CTA per tile).  GB300 issues FP64 at about two
// multiply-adds per cycle per SM, so the factorisation of C (r^3 / 3
// multiply-adds) belongs on all SMs, not one.  log det P by Sylvester:
// N log sigma2 + 2 sum_j log F_jj (k_chol_logdet).  err = 1 if C is not
// positive definite.
constexpr int kCholB = 32;

__global__ void k_chol_init(const double *__restrict__ Gp, int nz, int r, double sigma2, double *__restrict__ C) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)r * r) return;
    const int i = (int)(e / r), l = (int)(e % r);
    if (l > i) return;
    double g = 0.0;
    for (int z = 0; z < nz; ++z) g += Gp[((size_t)z * r + l) * r + i];  // partial tiles hold l <= i
    C[(size_t)i * r + l] = (i == l ? 1.0 : 0.0) + g / sigma2;
}

// the diagonal block [j0, j0 + b) in place, right-looking (one CTA): per
// column one thread forms the pivot's square root and reciprocal (GB300's FP64
// square root and divide are long dependent chains on a slow pipe), the rows
// below are scaled by the reciprocal, and the block's remaining lower
// triangle takes the rank-1 update, one entry per thread
__global__ void __launch_bounds__(1024) k_chol_diag(double *__restrict__ C, int r, int j0, int *__restrict__ err) {
    __shared__ double a[kCholB][kCholB + 1];
    __shared__ double s_inv;
    __shared__ int s_bad;
    const int b = min(kCholB, r - j0);
    const int tid = threadIdx.x;
    const int ti = tid >> 5, tl = tid & 31;  // this thread's entry of the block
    if (tid == 0) s_bad = 0;
    if (ti < b && tl <= ti) a[ti][tl] = C[(size_t)(j0 + ti) * r + j0 + tl];
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (tid == 0) {
            const double v = a[j][j];
            const bool ok = v > 0.0;
            const double djj = ok ? sqrt(v) : 1.0;
            a[j][j] = djj;
            s_inv = 1.0 / djj;
            if (!ok) s_bad = 1;
        }
        __syncthreads();
        if (tid > j && tid < b) a[tid][j] *= s_inv;
        __syncthreads();
        if (ti < b && tl > j && tl <= ti) a[ti][tl] -= a[ti][j] * a[tl][j];
        __syncthreads();  // the next pivot reads an updated entry
    }
    if (ti < b && tl <= ti) C[(size_t)(j0 + ti) * r + j0 + tl] = a[ti][tl];
    if (tid == 0) {
        if (j0 == 0) *err = 0;
        if (s_bad) *err = 1;
    }
}

// rows i >= j0 + b: F[i][j0 .. j0+b) = C[i][j0 .. j0+b) F_diag^{-T}, forward
// substitution along the row (one thread per row; one-warp CTAs, so that the
// FP64 work of the rows spreads over many SMs)
constexpr int kCholPanelThreads = 32;

__global__ void __launch_bounds__(kCholPanelThreads) k_chol_panel(double *__restrict__ C, int r, int j0) {
    __shared__ double d[kCholB][kCholB + 1];
    __shared__ double rd[kCholB];  // reciprocals of the diagonal
    const int b = min(kCholB, r - j0);
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int k = e / b, t = e % b;
        if (t <= k) d[k][t] = C[(size_t)(j0 + k) * r + j0 + t];
    }
    if (threadIdx.x < b) rd[threadIdx.x] = 1.0 / C[(size_t)(j0 + threadIdx.x) * r + j0 + threadIdx.x];
    __syncthreads();
    const int i = j0 + b + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    double x[kCholB];
    double *row = C + (size_t)i * r + j0;
#pragma unroll
    for (int k = 0; k < kCholB; ++k) x[k] = k < b ? row[k] : 0.0;
#pragma unroll
    for (int k = 0; k < kCholB; ++k) {
        if (k < b) {
            // four partial sums: the FP64 chain of a row is a quarter as long
            double v0 = x[k], v1 = 0.0, v2 = 0.0, v3 = 0.0;
#pragma unroll
            for (int t = 0; t < k; t += 4) {
                v0 -= x[t] * d[k][t];
                if (t + 1 < k) v1 -= x[t + 1] * d[k][t + 1];
                if (t + 2 < k) v2 -= x[t + 2] * d[k][t + 2];
                if (t + 3 < k) v3 -= x[t + 3] * d[k][t + 3];
            }
            x[k] = ((v0 + v1) + (v2 + v3)) * rd[k];
        }
    }
#pragma unroll
    for (int k = 0; k < kCholB; ++k)
        if (k < b) row[k] = x[k];
}

// the trailing lower triangle, rows and columns from m0 = j0 + b: tile
// (blockIdx.y, blockIdx.x) of 32 x 32 entries, skipped above the diagonal
__global__ void __launch_bounds__(1024) k_chol_update(double *__restrict__ C, int r, int j0) {
    __shared__ double pi[32][kCholB + 1], pl[32][kCholB + 1];
    const int b = min(kCholB, r - j0);
    const int m0 = j0 + b;
    const int bi = blockIdx.y, bl = blockIdx.x;
    if (bl > bi) return;
    const int y = threadIdx.x / 32, x = threadIdx.x % 32;
    {
        const int k = threadIdx.x % 32, row = threadIdx.x / 32;
        const int ii = m0 + bi * 32 + row, ll = m0 + bl * 32 + row;
        pi[row][k] = (ii < r && k < b) ? C[(size_t)ii * r + j0 + k] : 0.0;
        pl[row][k] = (ll < r && k < b) ? C[(size_t)ll * r + j0 + k] : 0.0;
    }
    __syncthreads();
    const int i = m0 + bi * 32 + y, l = m0 + bl * 32 + x;
    if (i >= r || l > i) return;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kCholB; ++k) acc = fma(pi[y][k], pl[x][k], acc);
    C[(size_t)i * r + l] -= acc;
}

__global__ void k_chol_logdet(const double *__restrict__ C, int r, int64_t N, double sigma2,
                              double *__restrict__ logdet, double *__restrict__ rdiag) {
    __shared__ double part[32];
    double ld = 0.0;
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double f = C[(size_t)j * r + j];
        ld += 2.0 * log(f);
        rdiag[j] = 1.0 / f;  // for the columns of F^{-1}
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ld += __shfl_xor_sync(0xffffffffu, ld, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ld;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = (double)N * log(sigma2);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *logdet = t;
    }
}

// Columns of F^{-1} (F lower, row-major r x r) by forward substitution, one
// warp per column c: FinvT[c][i] = (F^{-1})[i][c] (zero for i < c).  The
// dots run across the lanes; the column being solved sits in shared memory.
__global__ void k_pc_finv(const double *__restrict__ F, const double *__restrict__ rdiag, int r,
                          double *__restrict__ FinvT) {
    __shared__ double s_x[4][kPcMaxRank];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 4 + w;
    if (c >= r) return;  // uniform per warp
    double *x = s_x[w];
    for (int i = c; i < r; ++i) {
        double part = 0.0;
        for (int k = c + lane; k < i; k += 32) part = fma(F[(size_t)i * r + k], x[k], part);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const double xi = ((i == c ? 1.0 : 0.0) - part) * rdiag[i];
        if (lane == 0) x[i] = xi;
        __syncwarp();
    }
    for (int i = lane; i < r; i += 32) FinvT[(size_t)c * r + i] = i < c ? 0.0 : x[i];
}

// C^{-1} = F^{-T} F^{-1}: Cinv[a][b] = sum_{k >= max(a, b)} Finv[k][a] Finv[k][b],
// one warp per entry a <= b (mirrored).
__global__ void k_pc_cinv(const double *__restrict__ FinvT, int r, double *__restrict__ Cinv) {
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= (int64_t)r * r) return;  // uniform per warp
    const int a = (int)(e / r), b = (int)(e % r);
    if (a > b) return;
    double acc = 0.0;
    for (int k = b + lane; k < r; k += 32) acc = fma(FinvT[(size_t)a * r + k], FinvT[(size_t)b * r + k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        Cinv[(size_t)a * r + b] = acc;
        Cinv[(size_t)b * r + a] = acc;
    }
}

__global__ void k_sum(const double *__restrict__ a, int64_t n, double *__restrict__ out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += a[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---- shared-memory staging of L by TMA
// The rows (q order) are cut into tiles of kTR; a persistent CTA takes the
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... and streams each tile's L in
// chunks of kMC rank indices: one 2-D tensor copy (cp.async.bulk.tensor,
// box kTR x kMC floats, 32 KB) per chunk, issued by thread 0 and completing
// on an mbarrier.  Two chunk buffers alternate, so the next chunk (of this
// tile or the next) is in flight while the current one is used.  Rows and
// rank indices outside L are filled with zeros by the copy.  Every wait is
// bounded; on expiry the CTA records DEV_TIMEOUT in the error word and
// returns.
constexpr int kTR = 256;      // rows per tile (= threads per CTA)
constexpr int kMC = 32;       // rank indices per chunk
constexpr int kSpinLimit = 1 << 22;
constexpr int kPcCtasPerSm = 3;  // persistent CTAs per SM of the passes over L

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory loads by 32-bit shared address (volatile: never moved above
// the barrier waits that make the data visible)
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ F2 lds_f2(uint32_t a) {
    F2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.hi), "=f"(v.lo) : "r"(a));
    return v;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The chunk sequence of one CTA within a pass, tile by tile (the apply) or
// rank block by rank block (t = L^T R).  The buffers and barrier phases
// follow the CTA's running chunk count g (passes included).
struct ChunkStream {
    float *buf;     // 2 x kMC x kTR floats
    uint64_t *bar;  // 2 mbarriers
    const CUtensorMap *map;
    int nchunk, ntile_cta;
    bool rank_major;  // false: chunk c = rank block c % nchunk of tile c / nchunk;
                      // true:  chunk c = rank block c / ntile_cta of tile c % ntile_cta

    __device__ __forceinline__ int tile_of(int c) const { return rank_major ? c % ntile_cta : c / nchunk; }
    __device__ __forceinline__ int block_of(int c) const { return rank_major ? c / ntile_cta : c % nchunk; }
    __device__ __forceinline__ int64_t tile_row0(int c) const {
        return ((int64_t)blockIdx.x + (int64_t)tile_of(c) * gridDim.x) * kTR;
    }
    __device__ __forceinline__ void issue(int g, int c) const {  // thread 0 only
        const int b = g & 1;
        mbar_expect_tx(bar + b, (uint32_t)(kMC * kTR * 4));
        tma_load_2d(buf + (size_t)b * kMC * kTR, map, (int)tile_row0(c), block_of(c) * kMC, bar + b);
    }
    // every thread waits for chunk c (the use count of its buffer gives the
    // parity); false (CTA-uniform) if a wait expired.  next_issued: chunk
    // c + 1 is in flight too.
    __device__ __forceinline__ bool wait(int c, int *s_bad, int *err, bool next_issued) const {
        const uint32_t parity = (uint32_t)((c >> 1) & 1);
        const bool ok = mbar_wait_bounded(bar + (c & 1), parity);
        if (!ok) atomicOr(s_bad, 1);
        __syncthreads();
        if (*s_bad) {
            if (threadIdx.x == 0) {
                atomicOr(err, DEV_TIMEOUT);
                // let late copies land before the CTA exits (bounded again)
                mbar_wait_bounded(bar + (c & 1), parity);
                if (next_issued) mbar_wait_bounded(bar + ((c + 1) & 1), (uint32_t)(((c + 1) >> 1) & 1));
            }
            return false;
        }
        return true;
    }
    __device__ __forceinline__ const float *chunk(int c) const { return buf + (size_t)(c & 1) * kMC * kTR; }
};

__device__ __forceinline__ int tiles_of_cta(int64_t N) {
    const int64_t ntile = (N + kTR - 1) / kTR;
    return blockIdx.x < ntile ? (int)((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
}

// t_part[b][m][j] = sum over the rows of CTA b's tiles of L[m][i] R[i][j].
// The CTA streams its chunks rank block by rank block: rank indices
// 0..kMC-1 of all its tiles, then the next kMC, and so on (chunk c is rank
// block c / ntile of the CTA's tile c % ntile).  Warp w owns the rank
// indices w, w + 8, w + 16, w + 24 of every block; lane l takes rows l,
// l + 32, ... of each tile and keeps one float-pair running sum per owned
// rank index and column across all the CTA's tiles, so sums cross lanes
// (shuffles) only once per rank block, after its last tile.  The rows of R
// for the next chunk are fetched into registers while the current chunk is
// summed, then put in shared memory as float pairs.  The split of an FP64
// row into its float pair is FP64 work (conversions on GB300's slow FP64
// pipe), so it is done once per row and pass: in the first rank block, whose
// chunks cover each of the CTA's tiles once, every thread keeps its rows'
// pairs in Rsp (N x ncols, the layout of R) and the later rank blocks load
// them from there (8 bytes, as for the FP64 row; each row is written and
// read back by the same thread).  Per-chunk splits had cost about 10 % of
// the pass at rank 350.
// NC: columns per pass (1, 2, 4 or 8); a pass with fewer real columns pads
// with zero columns.
template <int NC>
__global__ void __launch_bounds__(kTR, NC <= 4 ? kPcCtasPerSm : 2) k_pc_ltr(const __grid_constant__ CUtensorMap map, int r,
                                                 const double *__restrict__ R, int64_t N, int ncols,
                                                 double *__restrict__ t_part, F2 *__restrict__ Rsp,
                                                 int *__restrict__ err, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    constexpr int NW = kTR / 32, OWN = kMC / NW, RPL = kTR / 32;  // warps, rank indices per warp, rows per lane
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    F2 *Rs = reinterpret_cast<F2 *>(buf + 2 * kMC * kTR);  // kTR x NC
    uint64_t *bar = reinterpret_cast<uint64_t *>(Rs + kTR * NC);
    __shared__ int s_bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(bar);
        mbar_init(bar + 1);
        mbar_fence_init();
        s_bad = 0;
    }
    __syncthreads();  // barriers and s_bad initialised before any thread waits on them
    const int nchunk = (r + kMC - 1) / kMC;
    const int ntile = tiles_of_cta(N);
    const ChunkStream cs{buf, bar, &map, nchunk, ntile, true};
    const int total = nchunk * ntile;
    int c_base = 0;  // chunks streamed by earlier passes (barrier phases keep counting)
    for (int j0 = 0; j0 < ncols; j0 += NC) {
        const int nc = min(NC, ncols - j0);
        F2 acc[OWN][NC];
#pragma unroll
        for (int o = 0; o < OWN; ++o)
#pragma unroll
            for (int u = 0; u < NC; ++u) acc[o][u] = F2{0.f, 0.f};
        // this thread's row for the chunk about to be used, as raw 8 bytes: the
        // FP64 row of R in the first rank block (c < ntile), its float pair
        // from Rsp after that
        unsigned long long rn[NC];
#pragma unroll
        for (int u = 0; u < NC; ++u) rn[u] = 0ull;
        if (total > 0) {
            const int64_t i = cs.tile_row0(0) + threadIdx.x;
#pragma unroll
            for (int u = 0; u < NC; ++u)
                if (u < nc && i < N) rn[u] = reinterpret_cast<const unsigned long long *>(R)[i * ncols + j0 + u];
            if (threadIdx.x == 0) cs.issue(c_base, 0);
        }
        for (int c = 0; c < total; ++c) {
            const int cc = c_base + c;
            if (threadIdx.x == 0 && c + 1 < total) cs.issue(cc + 1, c + 1);
            if (c < ntile) {
                const int64_t i = cs.tile_row0(c) + threadIdx.x;
#pragma unroll
                for (int u = 0; u < NC; ++u) {
                    F2 f;
                    split_f2(__longlong_as_double((long long)rn[u]), f.hi, f.lo);
                    Rs[threadIdx.x * NC + u] = f;
                    if (u < nc && i < N) Rsp[i * ncols + j0 + u] = f;
                }
            } else {
#pragma unroll
                for (int u = 0; u < NC; ++u)
                    Rs[threadIdx.x * NC + u] =
                        F2{__uint_as_float((unsigned)(rn[u] & 0xffffffffull)), __uint_as_float((unsigned)(rn[u] >> 32))};
            }
            if (c + 1 < total) {
                const int64_t i = cs.tile_row0(c + 1) + threadIdx.x;
                if (c + 1 < ntile) {
#pragma unroll
                    for (int u = 0; u < NC; ++u)
                        rn[u] = (u < nc && i < N) ? reinterpret_cast<const unsigned long long *>(R)[i * ncols + j0 + u]
                                                  : 0ull;
                } else {
#pragma unroll
                    for (int u = 0; u < NC; ++u)
                        rn[u] = (u < nc && i < N) ? reinterpret_cast<const unsigned long long *>(Rsp)[i * ncols + j0 + u]
                                                  : 0ull;
                }
            }
            if (!cs.wait(cc, &s_bad, err, c + 1 < total)) return;  // (its barrier also publishes Rs)
            const uint32_t la = smem_u32(cs.chunk(cc)) + (uint32_t)(warp * kTR + lane) * 4u;
            const uint32_t ra = smem_u32(Rs) + (uint32_t)lane * NC * 8u;
            // (rank indices at or above r read the zeros the copy filled in)
#pragma unroll
            for (int k = 0; k < RPL; ++k) {
                F2 rv[NC];
#pragma unroll
                for (int u = 0; u < NC; ++u) rv[u] = lds_f2(ra + (uint32_t)((32 * k * NC + u) * 8));
#pragma unroll
                for (int o = 0; o < OWN; ++o) {
                    const float l = lds_f32(la + (uint32_t)((o * NW * kTR + 32 * k) * 4));
#pragma unroll
                    for (int u = 0; u < NC; ++u) f2_fma(acc[o][u], l, rv[u].hi, rv[u].lo);
                }
            }
            __syncthreads();  // every warp is done with this chunk's buffer and with Rs
            if (c % ntile == ntile - 1) {
                // The rank block's last tile: sum each accumulator over the 32
                // lanes through the buffer just consumed (each warp writes its
                // lanes' values to its own 4 KB, then every lane adds a slice
                // and a few shuffles finish), in groups of RG values per lane.
                const int m0 = (c / ntile) * kMC;
                constexpr int V = OWN * NC, RG = V < 16 ? V : 16, LPV = 32 / RG, SL = 32 / LPV;
                const uint32_t wa = smem_u32(cs.chunk(cc)) + (uint32_t)warp * 4096u;
#pragma unroll
                for (int g0 = 0; g0 < V; g0 += RG) {
#pragma unroll
                    for (int v = 0; v < RG; ++v) {
                        const F2 a = acc[(g0 + v) / NC][(g0 + v) % NC];
                        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(wa + (uint32_t)((v * 32 + lane) * 8)),
                                     "f"(a.hi), "f"(a.lo)
                                     : "memory");
                    }
                    __syncwarp();
                    const int v = lane / LPV, part = lane % LPV;  // value v, lanes part*SL .. part*SL+SL-1
                    F2 a = F2{0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < SL; ++e) a = f2_add(a, lds_f2(wa + (uint32_t)((v * 32 + part * SL + e) * 8)));
#pragma unroll
                    for (int sh = LPV / 2; sh > 0; sh >>= 1) {
                        F2 other;
                        other.hi = __shfl_xor_sync(0xffffffffu, a.hi, sh);
                        other.lo = __shfl_xor_sync(0xffffffffu, a.lo, sh);
                        a = f2_add(a, other);
                    }
                    const int o = (g0 + v) / NC, u = (g0 + v) % NC, m = m0 + warp + o * NW;
                    if (part == 0 && m < r && u < nc)
                        t_part[((size_t)blockIdx.x * r + m) * ncols + j0 + u] = (double)a.hi + (double)a.lo;
                    __syncwarp();
                }
#pragma unroll
                for (int o = 0; o < OWN; ++o)
#pragma unroll
                    for (int u = 0; u < NC; ++u) acc[o][u] = F2{0.f, 0.f};
                // order these generic-proxy writes before the bulk copy that
                // will refill the buffer, then free it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
            }
        }
        c_base += total;
        if (ntile == 0)  // a CTA without rows still owns its rows of partials
            for (int t = threadIdx.x; t < r * nc; t += blockDim.x)
                t_part[((size_t)blockIdx.x * r + t / nc) * ncols + j0 + t % nc] = 0.0;
    }
}

// t[m][j] = sum over the gridDim partials (one warp per entry)
__global__ void k_pc_tsum(const double *__restrict__ t_part, int nb, int r, int ncols, double *__restrict__ t,
                          const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= (int64_t)r * ncols) return;
    double acc = 0.0;
    for (int b = lane; b < nb; b += 32) acc += t_part[(size_t)b * r * ncols + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) t[e] = acc;
}

// c[a][j] = sum_b Cinv[a][b] t[b][j] / sigma2^2 (one warp per entry)
__global__ void k_pc_cmul(const double *__restrict__ t, int r, int ncols, const double *__restrict__ Cinv,
                          double sigma2, double *__restrict__ c, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= (int64_t)r * ncols) return;
    const int a = (int)(e / ncols), j = (int)(e % ncols);
    double acc = 0.0;
    for (int b = lane; b < r; b += 32) acc = fma(Cinv[(size_t)a * r + b], t[(size_t)b * ncols + j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) c[e] = acc / (sigma2 * sigma2);
}

// Z = R / sigma2 - L c (thread t: row t of the current tile) and per-CTA
// partial sums of R .* Z per column (rz_partial[b * ncols + j], gridDim rows).
// c is split into float pairs in shared memory per pass of up to kColsPass
// columns; L c is summed in float pairs.
template <int NC>
__global__ void __launch_bounds__(kTR, kPcCtasPerSm) k_pc_apply(const __grid_constant__ CUtensorMap map, int r,
                                                   const double *__restrict__ R, int64_t N, int ncols,
                                                   const double *__restrict__ c, double inv,
                                                   double *__restrict__ Z, double *__restrict__ rz_partial,
                                                   int *__restrict__ err, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *buf = reinterpret_cast<float *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(buf + 2 * kMC * kTR);
    F2 *cs2 = reinterpret_cast<F2 *>(bar + 2);  // r x NC
    __shared__ int s_bad;
    __shared__ double red[kTR / 32][NC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(bar);
        mbar_init(bar + 1);
        mbar_fence_init();
        s_bad = 0;
    }
    __syncthreads();  // barriers and s_bad initialised before any thread waits on them
    const int nchunk = (r + kMC - 1) / kMC;
    const int ntile = tiles_of_cta(N);
    const ChunkStream cs{buf, bar, &map, nchunk, ntile};
    const int total = nchunk * ntile;
    // inv = 1 / sigma2, formed once on the host (a division per thread would
    // put a few microseconds of FP64 work on every launch)
    int c_base = 0;
    for (int j0 = 0; j0 < ncols; j0 += NC) {
        const int nc = min(NC, ncols - j0);
        for (int t = threadIdx.x; t < r * NC; t += blockDim.x) {
            const int m = t / NC, u = t % NC;
            float hi = 0.f, lo = 0.f;
            if (u < nc) split_f2(c[(size_t)m * ncols + j0 + u], hi, lo);
            cs2[t] = F2{hi, lo};
        }
        __syncthreads();
        double rz[NC];
#pragma unroll
        for (int u = 0; u < NC; ++u) rz[u] = 0.0;
        // rank 0: no chunks, each tile is R / sigma2
        for (int tt = 0; tt < (nchunk > 0 ? 0 : ntile); ++tt) {
            const int64_t i = ((int64_t)blockIdx.x + (int64_t)tt * gridDim.x) * kTR + threadIdx.x;
#pragma unroll
            for (int u = 0; u < NC; ++u)
                if (u < nc && i < N) {
                    const int64_t t = i * ncols + j0 + u;
                    const double rv = R[t], z = rv * inv;
                    Z[t] = z;
                    rz[u] += rv * z;
                }
        }
        F2 acc[NC];
#pragma unroll
        for (int u = 0; u < NC; ++u) acc[u] = F2{0.f, 0.f};
        if (total > 0 && threadIdx.x == 0) cs.issue(c_base, 0);
        for (int c = 0; c < total; ++c) {
            const int cc = c_base + c;
            if (threadIdx.x == 0 && c + 1 < total) cs.issue(cc + 1, c + 1);
            if (!cs.wait(cc, &s_bad, err, c + 1 < total)) return;
            const float *Lc = cs.chunk(cc);
            const int m0 = (c % nchunk) * kMC, mc = min(kMC, r - m0);
            if (mc == kMC) {
                const uint32_t la = smem_u32(Lc) + threadIdx.x * 4u;
                const uint32_t ca = smem_u32(cs2 + m0 * NC);
#pragma unroll 8
                for (int mm = 0; mm < kMC; ++mm) {
                    const float l = lds_f32(la + (uint32_t)(mm * kTR * 4));
#pragma unroll
                    for (int u = 0; u < NC; ++u) {
                        const F2 cm = lds_f2(ca + (uint32_t)((mm * NC + u) * 8));
                        f2_fma(acc[u], l, cm.hi, cm.lo);
                    }
                }
            } else {
                for (int mm = 0; mm < mc; ++mm) {
                    const float l = Lc[mm * kTR + threadIdx.x];
                    const F2 *cm = cs2 + (m0 + mm) * NC;
#pragma unroll
                    for (int u = 0; u < NC; ++u) f2_fma(acc[u], l, cm[u].hi, cm[u].lo);
                }
            }
            __syncthreads();
            if (c % nchunk == nchunk - 1) {  // the tile is complete: its rows of Z
                const int64_t i = cs.tile_row0(c) + threadIdx.x;
#pragma unroll
                for (int u = 0; u < NC; ++u) {
                    if (u < nc && i < N) {
                        const int64_t t = i * ncols + j0 + u;
                        const double rv = R[t];
                        const double z = rv * inv - ((double)acc[u].hi + (double)acc[u].lo);
                        Z[t] = z;
                        rz[u] += rv * z;
                    }
                    acc[u] = F2{0.f, 0.f};
                }
            }
        }
        c_base += total;
        if (rz_partial) {
#pragma unroll
            for (int u = 0; u < NC; ++u) {
                double v = rz[u];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[warp][u] = v;
            }
            __syncthreads();
            if ((int)threadIdx.x < nc) {
                double tot = 0.0;
                for (int w = 0; w < kTR / 32; ++w) tot += red[w][threadIdx.x];
                rz_partial[(size_t)blockIdx.x * ncols + j0 + threadIdx.x] = tot;
            }
        }
        __syncthreads();
    }
}

// B[orig][j] = sum_m L[m][q] E_r[m][j] + sigma E_n[orig][j] (orig = perm0[q]), FP64
__global__ void k_pc_sample(const float *__restrict__ L, int64_t ldN, int r, int64_t N,
                            const int32_t *__restrict__ perm0, const double *__restrict__ Er,
                            const double *__restrict__ En, int nprobe, double sigma, double *__restrict__ B) {
    const int64_t n = N * nprobe;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / nprobe;
        const int j = (int)(t % nprobe);
        double acc = 0.0;
        for (int m = 0; m < r; ++m) acc = fma((double)L[(size_t)m * ldN + q], Er[(size_t)m * nprobe + j], acc);
        const int64_t o = (int64_t)perm0[q] * nprobe + j;
        B[o] = acc + sigma * En[o];
    }
}

// L in the caller's point order: out[orig * r + m] = L[m][q]
__global__ void k_pc_factor_out(const float *__restrict__ L, int64_t ldN, int r, int64_t N,
                                const int32_t *__restrict__ perm0, double *__restrict__ out) {
    const int64_t n = N * r;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / r;
        const int m = (int)(t % r);
        const size_t o = (size_t)m * ldN + q;
        out[(int64_t)perm0[q] * r + m] = (double)L[o];
    }
}

}  // namespace

struct Precond {
    Plan *plan = nullptr;
    int k_req = 0, rank = 0;
    double sigma2 = 0.0, logdet = 0.0, trace = 0.0;
    int64_t ldN = 0;
    double *dres = nullptr, *Cf = nullptr, *Cinv = nullptr, *t_part = nullptr, *cvec = nullptr,
           *scal = nullptr;
    F2 *rsp = nullptr;  // the float pairs of R's rows, N x cap_cols (written and read by k_pc_ltr)
    float *L32 = nullptr;  // the factor, k columns of ldN (q order)
    int32_t *piv_q = nullptr;
    int *ints = nullptr;  // [0] rank, [1] error flag
    int nb_ltr = 0, chunk = 0, cap_cols = 0;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    std::vector<void *> owned;
    double *tvec = nullptr;  // t = L^T R, r x cap_cols
    CUtensorMap tmap;        // L32 as a 2-D tensor (rows x rank), boxes of kTR x kMC
};

// scratch of the apply for up to ncols columns (grown before any capture)
int pc_reserve(Precond *pc, int ncols, cudaStream_t s) {
    if (ncols < 1 || ncols > kPcMaxCols) {
        set_error("preconditioner: ncols = %d is outside [1, %d]", ncols, kPcMaxCols);
        return FGK_ERR_INVALID;
    }
    if (ncols <= pc->cap_cols) return FGK_OK;
    const size_t kk = (size_t)std::max(pc->k_req, 1);
    const size_t nrow = (size_t)std::max<int64_t>(pc->plan->N, 1);
    void *t = dev_alloc((size_t)pc->nb_ltr * kk * ncols * 8, s);
    void *c = dev_alloc(kk * ncols * 8, s);
    void *tv = dev_alloc(kk * ncols * 8, s);
    void *rs = dev_alloc(nrow * ncols * 8, s);
    if (!t || !c || !tv || !rs) {
        if (t) dev_free(t, s);
        if (c) dev_free(c, s);
        if (tv) dev_free(tv, s);
        if (rs) dev_free(rs, s);
        set_error("preconditioner: scratch allocation failed");
        return FGK_ERR_OOM;
    }
    FGK_CUDA(cudaMemsetAsync(c, 0, kk * ncols * 8, s));
    for (auto &q : pc->owned)
        if (q == pc->t_part || q == pc->cvec || q == pc->tvec || q == pc->rsp) {
            dev_free(q, s);
            q = nullptr;
        }
    pc->owned.erase(std::remove(pc->owned.begin(), pc->owned.end(), nullptr), pc->owned.end());
    pc->t_part = (double *)t;
    pc->cvec = (double *)c;
    pc->tvec = (double *)tv;
    pc->rsp = (F2 *)rs;
    pc->owned.push_back(t);
    pc->owned.push_back(c);
    pc->owned.push_back(tv);
    pc->owned.push_back(rs);
    pc->bytes += (size_t)pc->nb_ltr * kk * (ncols - pc->cap_cols) * 8 + 2 * kk * (ncols - pc->cap_cols) * 8 +
                 nrow * (ncols - pc->cap_cols) * 8;
    pc->cap_cols = ncols;
    return FGK_OK;
}

double pc_sigma2(const Precond *pc) { return pc->sigma2; }
double pc_logdet(const Precond *pc) { return pc->logdet; }
int pc_rank(const Precond *pc) { return pc->rank; }
const Plan *pc_plan(const Precond *pc) { return pc->plan; }

static int cols_per_pass(int ncols) { return ncols >= 8 ? 8 : (ncols >= 3 ? (ncols == 3 || ncols == 4 ? 4 : 8) : ncols); }
static size_t ltr_smem(int r, int nc) {
    (void)r;
    return (size_t)2 * kMC * kTR * 4 + (size_t)kTR * nc * 8 + 2 * 8;
}
static size_t apply_smem(int r, int nc) { return (size_t)2 * kMC * kTR * 4 + 2 * 8 + (size_t)std::max(r, 1) * nc * 8; }

template <int NC>
static int set_pc_attrs(int k) {
    FGK_CUDA(cudaFuncSetAttribute(k_pc_ltr<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ltr_smem(k, NC)));
    FGK_CUDA(cudaFuncSetAttribute(k_pc_apply<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)apply_smem(k, NC)));
    return FGK_OK;
}

template <int NC>
static int launch_pc_ltr(const Precond *pc, int r, const double *R, int ncols, int *err, cudaStream_t s,
                         const int *gate);
template <int NC>
static int launch_pc_apply(const Precond *pc, int r, const double *R, int ncols, double *Z, double *rz_partial,
                           int *err, cudaStream_t s, const int *gate);

int pc_partial_blocks(const Precond *pc) { return pc->nb_ltr; }

int pc_apply(const Precond *pc, const double *R, int ncols, double *Z, double *rz_partial, cudaStream_t s,
             const int *gate) {
    if (ncols < 1 || ncols > pc->cap_cols) {
        set_error("preconditioner apply: ncols = %d is outside [1, %d] (internal)", ncols, pc->cap_cols);
        return FGK_ERR_INTERNAL;
    }
    const int r = pc->rank, nb = pc->nb_ltr;
    int *err = pc->ints + 2;
    const int nc = cols_per_pass(ncols);
    if (r > 0) {
        switch (nc) {
            case 1: FGK_TRY(launch_pc_ltr<1>(pc, r, R, ncols, err, s, gate)); break;
            case 2: FGK_TRY(launch_pc_ltr<2>(pc, r, R, ncols, err, s, gate)); break;
            case 4: FGK_TRY(launch_pc_ltr<4>(pc, r, R, ncols, err, s, gate)); break;
            default: FGK_TRY(launch_pc_ltr<8>(pc, r, R, ncols, err, s, gate)); break;
        }
        const unsigned nw_blocks = grid_for((int64_t)r * ncols * 32, 256);
        k_pc_tsum<<<nw_blocks, 256, 0, s>>>(pc->t_part, nb, r, ncols, pc->tvec, gate);
        FGK_LAUNCH_CHECK();
        k_pc_cmul<<<nw_blocks, 256, 0, s>>>(pc->tvec, r, ncols, pc->Cinv, pc->sigma2, pc->cvec, gate);
        FGK_LAUNCH_CHECK();
    }
    switch (nc) {
        case 1: return launch_pc_apply<1>(pc, r, R, ncols, Z, rz_partial, err, s, gate);
        case 2: return launch_pc_apply<2>(pc, r, R, ncols, Z, rz_partial, err, s, gate);
        case 4: return launch_pc_apply<4>(pc, r, R, ncols, Z, rz_partial, err, s, gate);
        default: return launch_pc_apply<8>(pc, r, R, ncols, Z, rz_partial, err, s, gate);
    }
}

// the driver's tensor-map encoder, fetched once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int encode_tiled(EncodeTiledFn *out) {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    if (!fn) {
        set_error("preconditioner: cuTensorMapEncodeTiled is not available");
        return FGK_ERR_CUDA;
    }
    *out = fn;
    return FGK_OK;
}

int pc_check(const Precond *pc, cudaStream_t s) {
    int e = 0;
    FGK_CUDA(cudaMemcpyAsync(&e, pc->ints + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaStreamSynchronize(s));
    if (e) {
        FGK_CUDA(cudaMemsetAsync(pc->ints + 2, 0, sizeof(int), s));
        set_error("preconditioner apply: a bounded wait for a bulk copy expired");
        return FGK_ERR_TIMEOUT;
    }
    return FGK_OK;
}

template <int NC>
static int launch_pc_ltr(const Precond *pc, int r, const double *R, int ncols, int *err, cudaStream_t s,
                         const int *gate) {
    TimedLaunch tl(kTimedPcLtr, s);
    k_pc_ltr<NC><<<pc->nb_ltr, kTR, ltr_smem(r, NC), s>>>(pc->tmap, r, R, pc->plan->N, ncols, pc->t_part,
                                                          pc->rsp, err, gate);
    FGK_LAUNCH_CHECK();
    tl.end();
    return FGK_OK;
}

template <int NC>
static int launch_pc_apply(const Precond *pc, int r, const double *R, int ncols, double *Z, double *rz_partial,
                           int *err, cudaStream_t s, const int *gate) {
    TimedLaunch tl(kTimedPcApply, s);
    k_pc_apply<NC><<<pc->nb_ltr, kTR, apply_smem(r, NC), s>>>(pc->tmap, r, R, pc->plan->N, ncols, pc->cvec,
                                                              1.0 / pc->sigma2, Z, rz_partial, err, gate);
    FGK_LAUNCH_CHECK();
    tl.end();
    return FGK_OK;
}

static void pc_release(Precond *pc, cudaStream_t s) {
    for (void *q : pc->owned) dev_free(q, s);
    pc->owned.clear();
}

static int pc_build(Precond *pc, cudaStream_t s) {
    Plan *p = pc->plan;
    const int64_t N = p->N, ldN = p->ldN;
    const int k = pc->k_req;
    auto take = [&](size_t bytes) -> void * {
        void *q = dev_alloc(bytes > 0 ? bytes : 16, s);
        if (q) {
            pc->owned.push_back(q);
            pc->bytes += bytes;
        }
        return q;
    };
    // the pivot steps: every row pair in one pass while that fits three CTAs
    // per SM (a thread left with a second pair makes every step wait for its
    // second pass over the factor), else three CTAs per SM, several passes
    int n_sm = 152;
    FGK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device));
    const int steps_blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>(3 * (int64_t)n_sm, (N + 2 * kPcThreads - 1) / (2 * kPcThreads)));
    pc->chunk = kTR;
    FGK_TRY(set_pc_attrs<1>(k));
    FGK_TRY(set_pc_attrs<2>(k));
    FGK_TRY(set_pc_attrs<4>(k));
    FGK_TRY(set_pc_attrs<8>(k));
    {
        // persistent CTAs of the two passes over L: as many as are resident
        // together for one column (at most kPcCtasPerSm per SM)
        int dev = 0, nsm = 0, occ_a = 0, occ_t = 0;
        FGK_CUDA(cudaGetDevice(&dev));
        FGK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        FGK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, k_pc_apply<1>, kTR, apply_smem(k, 1)));
        FGK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, k_pc_ltr<1>, kTR, ltr_smem(k, 1)));
        const int per_sm = std::max(1, std::min(kPcCtasPerSm, std::min(occ_a, occ_t)));
        pc->nb_ltr = (int)std::min<int64_t>((int64_t)per_sm * std::max(nsm, 1), (N + kTR - 1) / kTR);
    }
    pc->ldN = ldN;
    pc->L32 = (float *)take((size_t)k * ldN * 4);
    pc->dres = (double *)take((size_t)N * 8);
    pc->piv_q = (int32_t *)take((size_t)k * 4);
    pc->ints = (int *)take(16);
    PivPart *part0 = (PivPart *)take((size_t)steps_blocks * sizeof(PivPart));
    PivPart *part1 = (PivPart *)take((size_t)steps_blocks * sizeof(PivPart));
    pc->Cf = (double *)take((size_t)k * k * 8);
    pc->Cinv = (double *)take((size_t)k * k * 8);
    pc->scal = (double *)take(32);
    for (void *q : pc->owned)
        if (!q) {
            set_error("fgk_precond_build: device allocation failed");
            return FGK_ERR_OOM;
        }
    // Gram partials: chunks of rows for parallelism
    const int ntile = (k + kGramTile - 1) / kGramTile;
    const int nz = (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 4096));
    const int64_t rows_per_z = (N + nz - 1) / nz;
    double *Gp = (double *)take((size_t)nz * k * k * 8);
    if (!Gp) {
        set_error("fgk_precond_build: device allocation failed");
        return FGK_ERR_OOM;
    }

    FGK_CUDA(cudaMemsetAsync(pc->L32, 0, (size_t)k * ldN * 4, s));
    const int init[4] = {k, 0, 0, 0};
    FGK_CUDA(cudaMemcpyAsync(pc->ints, init, sizeof(init), cudaMemcpyHostToDevice, s));
    KernArgs ka{p->xq[0], p->xq[1], p->xq[2], p->d, p->two_nu, p->kind, p->s2, nullptr, nullptr, N};
    // the exponential tables of the kernel columns, for the pivot steps only
    double *exptab = (double *)dev_alloc((size_t)2 * p->d * N * 8, s);
    if (!exptab) {
        set_error("fgk_precond_build: device allocation failed");
        return FGK_ERR_OOM;
    }
    ka.ep = exptab;
    ka.em = exptab + (size_t)p->d * N;
    k_pc_exptab<<<grid_for(N, 256), 256, 0, s>>>(ka, exptab, exptab + (size_t)p->d * N);
    FGK_LAUNCH_CHECK();
    k_pc_init<<<steps_blocks, kPcThreads, 0, s>>>(N, p->s2, p->perm[0], pc->dres, part0);
    FGK_LAUNCH_CHECK();
    PivPart *bufs[2] = {part0, part1};
    for (int m = 0; m < k; ++m) {
        k_pc_step<<<steps_blocks, kPcThreads, 0, s>>>(m, N, ldN, ka, p->perm[0], bufs[m & 1], steps_blocks,
                                                      bufs[(m + 1) & 1], pc->L32, pc->dres, pc->piv_q, pc->ints,
                                                      kExhausted * p->s2);
        FGK_LAUNCH_CHECK();
    }
    dev_free(exptab, s);
    int hints[4];
    FGK_CUDA(cudaMemcpyAsync(hints, pc->ints, sizeof(hints), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaStreamSynchronize(s));
    const int r = std::min(k, hints[0]);
    pc->rank = r;
    k_sum<<<1, 1024, 0, s>>>(pc->dres, N, pc->scal);
    FGK_LAUNCH_CHECK();
    {  // L32 as a 2-D tensor for the apply's TMA copies (rank rows of ldN floats)
        EncodeTiledFn enc = nullptr;
        FGK_TRY(encode_tiled(&enc));
        const cuuint64_t dims[2] = {(cuuint64_t)ldN, (cuuint64_t)std::max(r, 1)};
        const cuuint64_t strides[1] = {(cuuint64_t)ldN * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kTR, (cuuint32_t)kMC};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult cr = enc(&pc->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pc->L32, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            set_error("fgk_precond_build: cuTensorMapEncodeTiled failed (%d)", (int)cr);
            return FGK_ERR_CUDA;
        }
    }
    if (r > 0) {
        k_pc_gram<<<dim3(ntile, ntile, nz), kPcThreads, 0, s>>>(pc->L32, ldN, N, r, rows_per_z, Gp);
        FGK_LAUNCH_CHECK();
        k_chol_init<<<grid_for((int64_t)r * r, 256), 256, 0, s>>>(Gp, nz, r, pc->sigma2, pc->Cf);
        FGK_LAUNCH_CHECK();
        for (int j0 = 0; j0 < r; j0 += kCholB) {
            const int b = std::min(kCholB, r - j0);
            k_chol_diag<<<1, 1024, 0, s>>>(pc->Cf, r, j0, pc->ints + 1);
            FGK_LAUNCH_CHECK();
            const int rest = r - j0 - b;
            if (rest > 0) {
                k_chol_panel<<<(rest + kCholPanelThreads - 1) / kCholPanelThreads, kCholPanelThreads, 0, s>>>(
                    pc->Cf, r, j0);
                FGK_LAUNCH_CHECK();
                const int nt = (rest + 31) / 32;
                k_chol_update<<<dim3(nt, nt), 1024, 0, s>>>(pc->Cf, r, j0);
                FGK_LAUNCH_CHECK();
            }
        }
        // the diagonal's reciprocals go to C^{-1}'s storage until k_pc_cinv fills it
        k_chol_logdet<<<1, 256, 0, s>>>(pc->Cf, r, N, pc->sigma2, pc->scal + 1, pc->Cinv);
        FGK_LAUNCH_CHECK();
        // Gp (nz * k * k >= k * k doubles) as the scratch of F^{-1}
        k_pc_finv<<<(r + 3) / 4, 128, 0, s>>>(pc->Cf, pc->Cinv, r, Gp);
        FGK_LAUNCH_CHECK();
        k_pc_cinv<<<grid_for((int64_t)r * r * 32, 256), 256, 0, s>>>(Gp, r, pc->Cinv);
        FGK_LAUNCH_CHECK();
    }
    double hs[2] = {0.0, 0.0};
    FGK_CUDA(cudaMemcpyAsync(hs, pc->scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaMemcpyAsync(hints, pc->ints, sizeof(hints), cudaMemcpyDeviceToHost, s));
    FGK_CUDA(cudaStreamSynchronize(s));
    pc->trace = hs[0];
    pc->logdet = r > 0 ? hs[1] : (double)N * std::log(pc->sigma2);
    if (r > 0 && hints[1]) {
        set_error("fgk_precond_build: I + L^T L / sigma2 is not positive definite (internal)");
        return FGK_ERR_INTERNAL;
    }
    // the Gram partials are only needed for the factorisation
    dev_free(Gp, s);
    pc->owned.pop_back();
    pc->bytes -= (size_t)nz * k * k * 8;
    return pc_reserve(pc, 1, s);
}

}  // namespace fgk

using namespace fgk;

struct fgk_precond_s : public fgk::Precond {};

fgk::Precond *fgk::pc_of(fgk_precond h) { return h; }

extern "C" {

int fgk_precond_build(fgk_handle h, int rank, double sigma2, fgk_stream_t stream, fgk_precond *out) {
    clear_error();
    if (out) *out = nullptr;
    if (!h || !out || rank < 0 || rank > kPcMaxRank || !(sigma2 > 0.0) || !std::isfinite(sigma2)) {
        set_error("fgk_precond_build: need h, out, 0 <= rank <= %d and a finite sigma2 > 0", kPcMaxRank);
        return FGK_ERR_INVALID;
    }
    fgk_precond_s *pc = new fgk_precond_s();
    pc->plan = h;
    pc->k_req = (int)std::min<int64_t>(rank, h->N);
    pc->sigma2 = sigma2;
    cudaStream_t s = (cudaStream_t)stream;
    pc->stream = s;
    const int rc = pc_build(pc, s);
    if (rc) {
        pc_release(pc, s);
        delete pc;
        return rc;
    }
    *out = pc;
    return FGK_OK;
}

int fgk_precond_info(fgk_precond pc, fgk_precond_report *rep, int64_t *pivots) {
    clear_error();
    if (!pc || !rep) {
        set_error("fgk_precond_info: NULL argument");
        return FGK_ERR_INVALID;
    }
    rep->rank_requested = pc->k_req;
    rep->rank = pc->rank;
    rep->sigma2 = pc->sigma2;
    rep->trace_resid = pc->trace;
    rep->logdet = pc->logdet;
    rep->device_bytes = pc->bytes;
    if (pivots && pc->rank > 0) {
        std::vector<int32_t> q(pc->rank), perm(pc->plan->N);
        FGK_CUDA(cudaMemcpy(q.data(), pc->piv_q, pc->rank * 4, cudaMemcpyDeviceToHost));
        FGK_CUDA(cudaMemcpy(perm.data(), pc->plan->perm[0], pc->plan->N * 4, cudaMemcpyDeviceToHost));
        for (int m = 0; m < pc->rank; ++m) pivots[m] = perm[q[m]];
    }
    return FGK_OK;
}

int fgk_precond_factor(fgk_precond pc, double *L, fgk_stream_t stream) {
    clear_error();
    if (!pc || !L) {
        set_error("fgk_precond_factor: NULL argument");
        return FGK_ERR_INVALID;
    }
    if (pc->rank == 0) return FGK_OK;
    const int64_t n = pc->plan->N * pc->rank;
    k_pc_factor_out<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(pc->L32, pc->ldN, pc->rank, pc->plan->N,
                                                                         pc->plan->perm[0], L);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

int fgk_precond_sample(fgk_precond pc, const double *E_r, const double *E_n, int nprobe, double *B,
                       fgk_stream_t stream) {
    clear_error();
    if (!pc || !E_n || !B || (pc->rank > 0 && !E_r) || nprobe < 1 || nprobe > kPcMaxCols) {
        set_error("fgk_precond_sample: need pc, E_r (rank > 0), E_n, B and 1 <= nprobe <= %d", kPcMaxCols);
        return FGK_ERR_INVALID;
    }
    const int64_t n = pc->plan->N * nprobe;
    k_pc_sample<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(pc->L32, pc->ldN, pc->rank, pc->plan->N,
                                                                    pc->plan->perm[0], E_r, E_n, nprobe,
                                                                    std::sqrt(pc->sigma2), B);
    FGK_LAUNCH_CHECK();
    return FGK_OK;
}

int fgk_precond_apply(fgk_precond pc, const double *R, int ncols, double *Z, fgk_stream_t stream) {
    clear_error();
    if (!pc || !R || !Z || ncols < 1 || ncols > kPcMaxCols) {
        set_error("fgk_precond_apply: need pc, R, Z and 1 <= ncols <= %d", kPcMaxCols);
        return FGK_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Plan *p = pc->plan;
    const size_t bytes = (size_t)p->N * ncols * 8;
    double *Rq = (double *)dev_alloc(bytes, s), *Zq = (double *)dev_alloc(bytes, s);
    int rc = FGK_OK;
    if (!Rq || !Zq) {
        set_error("fgk_precond_apply: device allocation failed");
        rc = FGK_ERR_OOM;
    }
    if (!rc) rc = pc_reserve(pc, ncols, s);
    if (!rc) rc = to_q_order(p, R, Rq, ncols, 8, s);
    if (!rc) rc = pc_apply(pc, Rq, ncols, Zq, nullptr, s);
    if (!rc) rc = pc_check(pc, s);
    if (!rc) rc = from_q_order(p, Zq, Z, ncols, 8, s);
    if (Rq) dev_free(Rq, s);
    if (Zq) dev_free(Zq, s);
    return rc;
}

int fgk_precond_destroy(fgk_precond pc) {
    clear_error();
    if (!pc) return FGK_OK;
    pc_release(pc, pc->stream);
    cudaStreamSynchronize(pc->stream);
    delete pc;
    return FGK_OK;
}

}  // extern "C"
