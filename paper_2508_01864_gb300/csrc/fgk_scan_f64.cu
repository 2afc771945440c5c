// FP64 instantiation of the level scans (exact-path products and the
// true-residual recomputation of the solver).
#include "fgk_scan.cuh"

namespace fgk {

int mvm_q_f64(Plan *p, const double *Vq, int nrhs, double *Yq, cudaStream_t s, const int *gate, bool init_diag) {
    const int64_t n = p->N * nrhs;
    if (init_diag) {
        k_diag_init<double><<<grid_for(n, 256), 256, 0, s>>>(Vq, n, p->s2, Yq, gate);
        FGK_LAUNCH_CHECK();
    }
    if (p->nlev == 0) return FGK_OK;
    FGK_TRY(ensure_ws(p, scan_ws_elems<double>(p, nrhs) * sizeof(double), s));
    return run_levels_dispatch<double>(p, Vq, nrhs, Yq, (double *)p->ws.p, s, gate);
}

size_t mvm_ws_bytes(const Plan *p, int nrhs, bool f64) {
    return f64 ? scan_ws_elems<double>(p, nrhs) * sizeof(double) : scan_ws_elems<float>(p, nrhs) * sizeof(float);
}

}  // namespace fgk
