// FP32 instantiation of the level scans (the path used inside mixed-precision
// CG): FP32 vectors, moments and outputs.
#include "fgk_scan.cuh"

namespace fgk {

int mvm_q_f32(Plan *p, const float *Vq, int nrhs, float *Yq, cudaStream_t s, const int *gate, bool init_diag) {
    FGK_TRY(ensure_ws(p, scan_ws_elems<float>(p, nrhs) * sizeof(float), s));
    return run_levels_dispatch<float>(p, Vq, nrhs, Yq, (float *)p->ws.p, s, gate, init_diag);
}

// the same product with the caller's scratch (scan_ws_elems elements)
int mvm_q_f32_ws(Plan *p, const float *Vq, int nrhs, float *Yq, float *ws, cudaStream_t s) {
    return run_levels_dispatch<float>(p, Vq, nrhs, Yq, ws, s, nullptr, true);
}

// load the kernels of this plan's float product now (at build), so that no
// later product has the runtime load code
int scan_preload_f32(Plan *p) {
    return run_levels_dispatch<float>(p, nullptr, 1, nullptr, nullptr, nullptr, nullptr, true, true);
}

}  // namespace fgk
