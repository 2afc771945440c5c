// FP32 instantiation of the level scans (the path used inside mixed-precision
// CG): FP32 vectors, moments and outputs.
#include "fgk_scan.cuh"

namespace fgk {

int mvm_q_f32(Plan *p, const float *Vq, int nrhs, float *Yq, cudaStream_t s, const int *gate, bool init_diag) {
    const int64_t n = p->N * nrhs;
    if (init_diag) {
        k_diag_init<float><<<grid_for(n, 256), 256, 0, s>>>(Vq, n, (float)p->s2, Yq, gate);
        FGK_LAUNCH_CHECK();
    }
    if (p->nlev == 0) return FGK_OK;
    FGK_TRY(ensure_ws(p, scan_ws_elems<float>(p, nrhs) * sizeof(float), s));
    return run_levels_dispatch<float>(p, Vq, nrhs, Yq, (float *)p->ws.p, s, gate);
}

}  // namespace fgk
