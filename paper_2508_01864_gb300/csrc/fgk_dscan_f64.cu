// double instantiation of the lengthscale-gradient scans (fgk_dscan.cuh).
#include "fgk_dscan.cuh"

namespace fgk {

int dlogell_q_f64(Plan *p, int dim, const double *Vq, int nrhs, double *Yq, cudaStream_t s) {
    return dlogell_q<double>(p, dim, Vq, nrhs, Yq, s);
}

}  // namespace fgk
