// TV-penalised least squares (Eq. 3) by ISTA/FISTA with a Chambolle TV prox.
#include "common.cuh"

namespace pyhst {
size_t tv_workspace_bytes(const pyhst_geometry *g, const pyhst_tv_opts *o) { (void)g; (void)o; return 0; }
}  // namespace pyhst

extern "C" size_t pyhst_tv_workspace_size(const pyhst_geometry *g, const pyhst_tv_opts *opts) {
    return pyhst::tv_workspace_bytes(g, opts);
}

extern "C" int pyhst_tv_solve(const pyhst_geometry *g, const float *sino, const pyhst_tv_opts *opts, float *x,
                              double *energy, double *lipschitz_out, void *workspace, size_t ws_bytes,
                              pyhst_stream_t stream) {
    return pyhst::fail(PYHST_ERR_INVALID_ARG, "not built yet");
}
