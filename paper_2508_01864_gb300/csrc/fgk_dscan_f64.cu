// double instantiation of the lengthscale-gradient scans (fgk_dscan.cuh).
#include "fgk_dscan.cuh"

namespace fgk {

int dlogell_q_f64(Plan *p, int dim, const double *Vq, int nrhs, double *Yq, cudaStream_t s) {
    return dlogell_q<double>(p, dim, Vq, nrhs, Yq, s);
}

// used by the nu = 7/2, 9/2 products of fgk_scan_*.cu
template int run_levels_gen_dispatch<double>(Plan *, int, int, const double *, int, double *, double *, cudaStream_t,
                                           const double (*)[kMaxCoef], const int *, bool, bool);

}  // namespace fgk
