// float instantiation of the lengthscale-gradient scans (fgk_dscan.cuh).
#include "fgk_dscan.cuh"

namespace fgk {

int dlogell_q_f32(Plan *p, int dim, const float *Vq, int nrhs, float *Yq, cudaStream_t s) {
    return dlogell_q<float>(p, dim, Vq, nrhs, Yq, s);
}

// used by the nu = 7/2, 9/2 products of fgk_scan_*.cu
template int run_levels_gen_dispatch<float>(Plan *, int, int, const float *, int, float *, float *, cudaStream_t,
                                           const double (*)[kMaxCoef], const int *, bool, bool);

}  // namespace fgk
