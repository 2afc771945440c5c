// FP32 instantiation of the level scans (the path used inside mixed-precision
// CG); inputs may be FP32 or FP64, moments and outputs are FP32.
#include "fgk_scan.cuh"

namespace fgk {

int mvm_q_f32(Plan *p, const void *Vq, bool vin_f64, int nrhs, float *Yq, cudaStream_t s, const int *gate) {
    const int64_t n = p->N * nrhs;
    k_diag_init<float><<<grid_for(n, 256), 256, 0, s>>>(Vq, vin_f64 ? 1 : 0, n, (float)p->s2, Yq, gate);
    FGK_LAUNCH_CHECK();
    if (p->nlev == 0) return FGK_OK;
    FGK_TRY(ensure_ws(p, scan_ws_elems<float>(p, nrhs) * sizeof(float), s));
    return run_levels_dispatch<float>(p, Vq, vin_f64, nrhs, Yq, (float *)p->ws.p, s, gate);
}

}  // namespace fgk
