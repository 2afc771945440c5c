// FP64 instantiation of the level scans (exact-path products and the
// true-residual recomputation of the solver).
#include "fgk_scan.cuh"

namespace fgk {

int mvm_q_f64(Plan *p, const double *Vq, int nrhs, double *Yq, cudaStream_t s, const int *gate, bool init_diag) {
    FGK_TRY(ensure_ws(p, scan_ws_elems<double>(p, nrhs) * sizeof(double), s));
    return run_levels_dispatch<double>(p, Vq, nrhs, Yq, (double *)p->ws.p, s, gate, init_diag);
}

// the same product with the caller's scratch (scan_ws_elems elements)
int mvm_q_f64_ws(Plan *p, const double *Vq, int nrhs, double *Yq, double *ws, cudaStream_t s) {
    return run_levels_dispatch<double>(p, Vq, nrhs, Yq, ws, s, nullptr, true);
}

size_t mvm_ws_bytes(const Plan *p, int nrhs, bool f64) {
    return f64 ? scan_ws_elems<double>(p, nrhs) * sizeof(double) : scan_ws_elems<float>(p, nrhs) * sizeof(float);
}

// load the kernels of this plan's double product now (at build), so that no
// later product has the runtime load code
int scan_preload_f64(Plan *p) {
    return run_levels_dispatch<double>(p, nullptr, 1, nullptr, nullptr, nullptr, nullptr, true, true);
}

}  // namespace fgk
