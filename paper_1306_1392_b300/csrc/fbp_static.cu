// pyhst_fbp_static: filtered back-projection that allocates nothing.
//
// Some callers cannot hand the library a workspace: code that runs where
// device allocation is forbidden or unavailable (inside a framework that owns
// every allocation and exposes none to plug-ins, a real-time acquisition loop
// that may not call cudaMalloc after start-up, or a host language binding that
// has no device allocator).  For them this entry point keeps its scratch in
// one file-scope device array of fixed size, kFbpStaticBytes, which every GPU
// that loads the library holds until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress; host code must not pass
// the array's name to a kernel, since on the host it is only a stand-in
// symbol.  Make that first call before any stream capture.  Later calls on
// the device reuse the address.
//
// The array is shared by every call: calls whose work overlaps on the GPU
// (on different streams, or from different host threads) race on it.  Each
// call writes every byte of scratch it reads (angle table, FFT tables,
// filtered rows) before reading it, so nothing needs clearing between calls.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace pyhst {

size_t filter_table_bytes(int P);
int launch_filter_tables(int P, int filter, void *tables, cudaStream_t st);
int launch_filter(int kind, const void *data, int64_t slice_stride, int64_t angle_stride, const float *flat,
                  const float *dark, int z0, int n_slices_chunk, int n_angles, int n_bins, int P,
                  const void *tables, float *q, cudaStream_t st);

namespace {

constexpr size_t kFbpStaticBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_fbp_static_scratch[kFbpStaticBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
int static_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PYHST_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PYHST_ERR_INVALID_ARG, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fbp_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(PYHST_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PYHST_OK;
}

}  // namespace
}  // namespace pyhst

extern "C" size_t pyhst_fbp_static_max_bytes(void) { return pyhst::kFbpStaticBytes; }

extern "C" int pyhst_fbp_static(const pyhst_geometry *g, int input_type, const void *data, int64_t slice_stride,
                                int64_t angle_stride, const float *flat, const float *dark, int filter,
                                int32_t pad_len, float *out, pyhst_stream_t stream) {
    using namespace pyhst;
    int P = pad_len;
    int rc = check_fbp_args(g, input_type, data, flat, dark, filter, &P, out);
    if (rc) return rc;
    // scratch: angle table | FFT tables | filtered rows of S slices
    const size_t tab_b = angle_table_bytes(g->n_angles), fft_b = filter_table_bytes(P);
    const size_t per = sizeof(float) * (size_t)g->n_angles * g->n_bins;
    if (tab_b + fft_b + per > kFbpStaticBytes)
        return fail(PYHST_ERR_INVALID_ARG,
                    "pyhst_fbp_static: %d angles x %d bins (pad %d) need %zu bytes of scratch, above its fixed %zu",
                    g->n_angles, g->n_bins, P, tab_b + fft_b + per, kFbpStaticBytes);
    const int S = (int)std::min<size_t>({(size_t)g->n_slices, (kFbpStaticBytes - tab_b - fft_b) / per,
                                         (size_t)max_slices_per_pass(g->n_angles)});
    void *base = nullptr;
    if ((rc = static_scratch(&base))) return rc;
    char *b = static_cast<char *>(base);
    AngleInfo *tab = reinterpret_cast<AngleInfo *>(b);
    void *tables = b + tab_b;
    float *q = reinterpret_cast<float *>(b + tab_b + fft_b);

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    if ((rc = launch_filter_tables(P, filter, tables, st))) return rc;
    const float weight = (float)(M_PI / ((double)g->n_angles * (double)g->pixel_size));
    for (int z0 = 0; z0 < g->n_slices; z0 += S) {
        const int n = std::min(S, g->n_slices - z0);
        rc = launch_filter(input_type, data, slice_stride, angle_stride, flat, dark, z0, n, g->n_angles, g->n_bins,
                           P, tables, q, st);
        if (rc) return rc;
        pyhst_geometry gc = *g;
        gc.n_slices = n;
        rc = launch_backproject(&gc, tab, BpSource{q, nullptr}, out + (size_t)z0 * g->nx * g->ny, weight, st);
        if (rc) return rc;
    }
    return PYHST_OK;
}
