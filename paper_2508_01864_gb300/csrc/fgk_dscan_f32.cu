// float instantiation of the lengthscale-gradient scans (fgk_dscan.cuh).
#include "fgk_dscan.cuh"

namespace fgk {

int dlogell_q_f32(Plan *p, int dim, const float *Vq, int nrhs, float *Yq, cudaStream_t s) {
    return dlogell_q<float>(p, dim, Vq, nrhs, Yq, s);
}

}  // namespace fgk
