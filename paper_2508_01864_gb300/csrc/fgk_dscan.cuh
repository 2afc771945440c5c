// Level scans with runtime readout coefficients and one moment more than the
// kernel's: the products with the lengthscale derivatives of K.
//
// With scaled distances r_k = sqrt(2 nu) |x_k - x'_k| / ell_k the Matérn
// factor is k(r) = sum_{p<P} c_p r^p e^{-r}, and dr_k / d log ell_k = -r_k, so
//   d k(r_k) / d log ell_k = -r_k k'(r_k) = h(r_k) = sum_{q<=P} h_q r^q e^{-r},
//   h_q = c_{q-1} - q c_q:  h = (0, 1), (0, 0, 1), (0, 0, 1/3, 1/3)
// for nu = 1/2, 3/2, 5/2 (the gradient formulas of App. C.1 times ell).
// Product kernel: dK/d log ell_m = s2 prod_{k != m} k(r_k) h(r_m), a product
// kernel whose factor m is h and the others c (padded with c_P = 0).  L1
// kernel, every lengthscale scaled together: d/d log ell k(R) = h(R), a
// radial kernel with coefficients h.  Both run the scans of fgk_scan.cuh
// with P + 1 moments and these coefficients; self-pairs contribute h(0) = 0.
#pragma once

#include "fgk_scan.cuh"

namespace fgk {

// P4 moments (2..5) with coefficients cf; kind as given (the product kernel
// with nu = 1/2 is not reduced to L1 here: a derivative factor differs per
// dimension)
template <class R>
int run_levels_gen_dispatch(Plan *p, int P4, int kind, const R *Vq, int nrhs, R *Yq, R *ws, cudaStream_t s,
                            const double (*cf)[kMaxCoef], const int *gate, bool init_diag, bool preload) {
    const int NOFF = p->d - 1;
    const int kk = NOFF == 0 ? FGK_L1 : kind;
    const int key = (P4 * 3 + NOFF) * 2 + kk;
    switch (key) {
#define FGK_GCASE(PP, NO, KK)     \
    case (PP * 3 + NO) * 2 + KK:  \
        return run_levels<R, PP, NO, KK, true>(p, Vq, nrhs, Yq, ws, s, gate, init_diag, cf, preload);
        FGK_GCASE(2, 0, FGK_L1)
        FGK_GCASE(3, 0, FGK_L1)
        FGK_GCASE(4, 0, FGK_L1)
        FGK_GCASE(5, 0, FGK_L1)
        FGK_GCASE(2, 1, FGK_L1)
        FGK_GCASE(3, 1, FGK_L1)
        FGK_GCASE(4, 1, FGK_L1)
        FGK_GCASE(5, 1, FGK_L1)
        FGK_GCASE(2, 1, FGK_PRODUCT)
        FGK_GCASE(3, 1, FGK_PRODUCT)
        FGK_GCASE(4, 1, FGK_PRODUCT)
        FGK_GCASE(5, 1, FGK_PRODUCT)
        FGK_GCASE(2, 2, FGK_L1)
        FGK_GCASE(3, 2, FGK_L1)
        FGK_GCASE(4, 2, FGK_L1)
        FGK_GCASE(2, 2, FGK_PRODUCT)
        FGK_GCASE(3, 2, FGK_PRODUCT)
        FGK_GCASE(4, 2, FGK_PRODUCT)
#undef FGK_GCASE
    default:
        break;
    }
    set_error("no generic-coefficient scan kernel for %d moments, d=%d, kind=%d", P4, p->d, kind);
    return FGK_ERR_INTERNAL;
}

// Y_q = s2 (dK/d log ell_dim) V_q in q order (dim in [0, d); the caller sums
// dims for the common scale of the product kernel, and passes dim = -1 for
// the L1 kernel's common scale).  Y_q is accumulated: the caller zeroes it.
template <class R>
int dlogell_q(Plan *p, int dim, const R *Vq, int nrhs, R *Yq, cudaStream_t s) {
    // c of the kernel (P moments) and h_q = c_{q-1} - q c_q (P + 1 moments)
    const int P = p->P;
    if (P + 1 > 5 || (P + 1 == 5 && p->d == 3)) {
        set_error("fgk_matvec_dlogell: the lengthscale derivative is built for nu <= 7/2 at d <= 2 and nu <= 5/2 "
                  "at d = 3 (it needs %d moments here)", P + 1);
        return FGK_ERR_INVALID;
    }
    double c[kMaxCoef], h[kMaxCoef];
    matern_coef(P, c);
    for (int q = 0; q < kMaxCoef; ++q) h[q] = (q > 0 ? c[q - 1] : 0.0) - q * c[q];
    double cf[kMaxD][kMaxCoef] = {};
    const bool radial = p->d == 1 || dim < 0;
    for (int k = 0; k < kMaxD; ++k)
        for (int q = 0; q < kMaxCoef; ++q) cf[k][q] = (radial ? (k == 0) : (k == dim)) ? h[q] : c[q];
    if (p->nlev == 0) return FGK_OK;
    const int kind = radial ? FGK_L1 : FGK_PRODUCT;
    FGK_TRY(ensure_ws(p, scan_ws_elems_for(p, nrhs, P + 1, kind) * sizeof(R), s));
    return run_levels_gen_dispatch<R>(p, P + 1, kind, Vq, nrhs, Yq, (R *)p->ws.p, s, cf, nullptr, false);
}

}  // namespace fgk
