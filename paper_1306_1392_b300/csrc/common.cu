// Error reporting, argument checks and the per-call angle table.
#include <cstdarg>
#include <cstdio>
#include <cmath>

#include <atomic>
#include <cstdint>

#include "common.cuh"

namespace pyhst {

static thread_local char g_err[1024] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_status(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PYHST_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return PYHST_OK;
}

int check_geometry(const pyhst_geometry *g) {
    if (!g) return fail(PYHST_ERR_INVALID_ARG, "geometry is NULL");
    if (g->n_angles < 1 || g->n_angles > 65535)
        return fail(PYHST_ERR_INVALID_ARG, "n_angles %d outside [1, 65535]", g->n_angles);
    if (g->n_bins < 1 || g->n_bins > 16384)
        return fail(PYHST_ERR_INVALID_ARG, "n_bins %d outside [1, 16384]", g->n_bins);
    if (g->nx < 1 || g->ny < 1 || g->nx > 16384 || g->ny > 16384)
        return fail(PYHST_ERR_INVALID_ARG, "image %d x %d outside [1, 16384]^2", g->nx, g->ny);
    if (g->n_slices < 1) return fail(PYHST_ERR_INVALID_ARG, "n_slices %d < 1", g->n_slices);
    if (!g->angles || !g->axis) return fail(PYHST_ERR_INVALID_ARG, "angles/axis pointer is NULL");
    if (!(g->pixel_size > 0.0f) || !std::isfinite(g->pixel_size))
        return fail(PYHST_ERR_INVALID_ARG, "pixel_size must be finite and > 0");
    if (!std::isfinite(g->cx) || !std::isfinite(g->cy))
        return fail(PYHST_ERR_INVALID_ARG, "cx/cy must be finite");
    // Tile-local coordinates use floor() through a float add: |t| must stay
    // well below 2^22 bins for every pixel.
    double reach = std::fabs((double)g->cx) + std::fabs((double)g->cy) + g->nx + g->ny + g->n_bins;
    if (reach > 1.0e6)
        return fail(PYHST_ERR_INVALID_ARG, "centre/size put detector coordinates beyond 1e6 bins");
    return PYHST_OK;
}

__global__ void angle_table_kernel(const float *__restrict__ angles, const float *__restrict__ axis,
                                   int n, AngleInfo *__restrict__ tab) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    double th = (double)angles[a];
    double s, c;
    sincos(th, &s, &c);
    AngleInfo e;
    e.c = c;
    e.s = s;
    e.axis = (double)axis[a];
    e.cf = (float)c;
    e.sf = (float)s;
    tab[a] = e;
}

int launch_angle_table(const float *angles, const float *axis, int n_angles, AngleInfo *tab,
                       cudaStream_t st) {
    angle_table_kernel<<<(n_angles + 127) / 128, 128, 0, st>>>(angles, axis, n_angles, tab);
    return cuda_status("angle table");
}

// Error bits recorded by kernels whose bounded waits gave up (one word per
// device; read and cleared by pyhst_device_status).
__device__ unsigned int g_dev_status;

unsigned *device_status_ptr() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dev_status) != cudaSuccess) return nullptr;
    return static_cast<unsigned *>(p);
}

std::atomic<int64_t> g_wait_limit{-1};

uint32_t pipeline_wait_limit() {
    const int64_t v = g_wait_limit.load(std::memory_order_relaxed);
    return v < 0 ? kDefaultWaitLimit : (uint32_t)v;
}

}  // namespace pyhst

extern "C" int pyhst_set_wait_limit(int64_t polls) {
    if (polls > (int64_t)UINT32_MAX) return pyhst::fail(PYHST_ERR_INVALID_ARG, "wait limit %lld beyond 2^32 - 1",
                                                        (long long)polls);
    pyhst::g_wait_limit.store(polls < 0 ? -1 : polls, std::memory_order_relaxed);
    return PYHST_OK;
}

extern "C" int pyhst_device_status(uint32_t *flags, int32_t clear) {
    if (!flags) return pyhst::fail(PYHST_ERR_INVALID_ARG, "flags pointer is NULL");
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, pyhst::g_dev_status, sizeof(v)) != cudaSuccess)
        return pyhst::cuda_status("reading the device status word");
    if (clear) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(pyhst::g_dev_status, &z, sizeof(z)) != cudaSuccess)
            return pyhst::cuda_status("clearing the device status word");
    }
    *flags = v;
    return PYHST_OK;
}

extern "C" const char *pyhst_last_error(void) { return pyhst::g_err; }

extern "C" const char *pyhst_version(void) { return "pyhst-b300 0.1 (sm_103a)"; }
