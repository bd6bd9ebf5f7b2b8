// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstddef>
#include <cstdint>

#include "pyhst.h"

namespace pyhst {

// Per-angle geometry, computed on the device at the start of every call from
// the caller's float32 angle and axis arrays: cos/sin in float64 (used for the
// per-tile reference coordinate) and their float32 roundings (used for the
// small tile-local offsets).
struct __align__(16) AngleInfo {
    double c, s;      // cos(theta), sin(theta)
    double axis;      // rotation-axis position, bins
    float cf, sf;     // float32 roundings of c and s
};

// ----------------------------------------------------------------- errors
int fail(int code, const char *fmt, ...);   // records the message, returns code
int cuda_status(const char *what);          // PYHST_OK or PYHST_ERR_CUDA after a launch
int check_geometry(const pyhst_geometry *g);
// Argument checks of the FBP entry points (fbp.cu): geometry, input kind,
// filter, pointers, flat/dark for raw kinds, and the pad length (*P = 0 is
// replaced by the default power of two >= max(64, 2 n_bins)).
int check_fbp_args(const pyhst_geometry *g, int kind, const void *data, const float *flat, const float *dark,
                   int filter, int *P, const void *out);
bool valid_pad(int P, int n_bins);
// Slices per filter/back-projection pass: the back-projector's grid has one
// row per slice (at most 65535) and the filter's grid one CTA per two of the
// pass's rows (at most 2^30 rows).
inline int max_slices_per_pass(int n_angles) {
    const int by_rows = (1 << 30) / (n_angles > 0 ? n_angles : 1);
    return by_rows < 1 ? 1 : (by_rows < 65535 ? by_rows : 65535);
}
// Residual CNN prox (cnn.cu): out = network(z) for n images of H x W.
int cnn_forward(const float *params, const float *z, float *out, int n, int H, int W, void *ws, cudaStream_t st);
size_t cnn_workspace_size(int n, int H, int W);

// Device address of this device's status word (kernels OR error bits into it).
unsigned *device_status_ptr();
// Polls after which the pipeline waits of the tensor-core kernels give up
// (pyhst_set_wait_limit; kDefaultWaitLimit unless lowered for a test).  The
// waits that drain in-flight tensor-core work before TMEM is freed always use
// kDefaultWaitLimit.
constexpr uint32_t kDefaultWaitLimit = 1u << 22;
uint32_t pipeline_wait_limit();

// ----------------------------------------------------------------- workspace
constexpr size_t kAlign = 256;
inline size_t align_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

struct Carver {
    char *base;
    size_t cap, off;
    Carver(void *b, size_t c) : base(static_cast<char *>(b)), cap(c), off(0) {}
    template <class T> T *take(size_t n) {
        off = align_up(off);
        T *p = reinterpret_cast<T *>(base + off);
        off += n * sizeof(T);
        return p;
    }
    bool ok() const { return off <= cap; }
};
inline size_t angle_table_bytes(int n_angles) { return align_up(sizeof(AngleInfo) * n_angles); }

// ----------------------------------------------------------------- launchers
// Fill `tab` [n_angles] from the caller's arrays.
int launch_angle_table(const float *angles, const float *axis, int n_angles, AngleInfo *tab,
                       cudaStream_t st);

// Source of back-projected rows: plain sinogram, or the residual a - b of two
// sinograms (used by the iterative solver's gradient step).
struct BpSource {
    const float *a;          // [n_slices][n_angles][n_bins]
    const float *b;          // NULL, or subtracted from a
    // gradient step in the epilogue: with y given, img receives
    // z = y - invL[slice] * (weight * back-projection) instead
    const float *y = nullptr;
    const float *invL = nullptr;
};
// angle_block: angles staged per block (8, 16, 24); <= 0 takes the tuned or
// default choice for the geometry (bp_block_for).
int launch_backproject(const pyhst_geometry *g, const AngleInfo *tab, BpSource src, float *img,
                       float weight, cudaStream_t st, int angle_block = 0);
bool bp_block_supported(int na);
// Angles per block for images of ny x nx and n_angles angles: the autotuned
// choice (pyhst_autotune_backproject / pyhst_set_backproject_block), else 16.
int bp_block_for(int nx, int ny, int n_angles);

// Projector: img [n_slices][ny][nx] -> sino [n_slices][n_angles][n_bins],
// scaled by `scale`; `xt` is scratch for the transposed slice stack
// ([n_slices][nx][ny] floats).
// staging: 256, 384 or 512 columns; <= 0 takes the tuned or rule-based choice (project_width)
int launch_project(const pyhst_geometry *g, const AngleInfo *tab, const float *img, float *sino,
                   float scale, float *xt, cudaStream_t st, int staging = 0);
size_t project_scratch_bytes(const pyhst_geometry *g);

// ----------------------------------------------------------------- mixed batches
// Per-slice descriptor of a mixed-size batch (device memory).  The
// back-projector reads bp_a (- bp_b) into bp_out with weight pixel_size; the
// projector reads proj_in (and proj_inT, its transpose) into proj_out scaled
// by pixel_size.  The solver fills the remaining fields.
struct BatchSlice {
    const AngleInfo *tab;
    int n_angles, n_bins, nx, ny;
    double cx, cy;
    float pixel_size;
    const float *bp_a, *bp_b;
    float *bp_out;
    const float *proj_in;
    float *proj_inT, *proj_out;
    int proj_nseg;          // row segments of the projector (proj_segments of this geometry)
    const float *bp_y;      // NULL, or the gradient step: bp_out = bp_y - *bp_invL * back-projection
    const float *bp_invL;
};
int bp_tiles(int nx, int ny, int *tx, int *ty);
int launch_backproject_batch(const BatchSlice *slices, const int4 *items, int n_items, bool residual,
                             cudaStream_t st, int angle_block = 16);
int proj_blocks(int n_angles, int n_bins, int *nb, int *na);
// Staging width of the projector for a geometry: 256, 384 or 512 columns (the
// autotuned choice, else 512 for sparse angle sets and 256 otherwise); every
// width gives the same bits
int project_width(int nx, int ny, int n_angles);
// row segments of the projector's walks for a slice geometry (fixes the float32 summation order)
int proj_segments(const pyhst_geometry *g);
// Sets the projector kernels' shared-memory attributes (call before a
// stream capture that launches them).
int set_proj_attr();
int launch_project_batch(const BatchSlice *slices, const int4 *proj_items, int n_proj_items,
                         const int4 *tr_items, int n_tr_items, int width, cudaStream_t st, int ns = 1);

// ----------------------------------------------------------------- profiling
// Opt-in per-launch timing (pyhst_profile_enable): events recorded on the
// launch stream around each kernel of a kind; off by default.  On a stream
// that is being captured the events become event-record nodes of the graph
// (recorded when the graph runs).
enum ProfKind { kProfBackproject = 0, kProfFilter = 1, kProfProject = 2, kProfChambolle = 3, kProfKinds = 4 };
struct ProfScope {
    int kind;
    cudaStream_t st;
    void *end;
    unsigned flags;
    ProfScope(int kind, cudaStream_t st);
    ~ProfScope();
};

// ----------------------------------------------------------------- device helpers
// floor(u) for 0 <= u < 2^22 in one add rounded toward -inf: the sum with
// 1.5 * 2^23 has unit spacing, so its low mantissa bits hold floor(u).
constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;

__device__ __forceinline__ float add_rd(float a, float b) {
    float r;
    asm("add.rm.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// A float64 sum fed in float32 runs of 8 terms (relative error ~5e-7 per
// run): one float64 add per 8 terms, FP64 throughput being scarce here.
struct RunSum {
    double acc = 0.0;
    float run = 0.0f;
    int n = 0;
    __device__ __forceinline__ void add(float v) {
        run += v;
        if (++n == 8) {
            acc += (double)run;
            run = 0.0f;
            n = 0;
        }
    }
    __device__ __forceinline__ double total() const { return acc + (double)run; }
};

// Paired float32 arithmetic (sm_100+ f32x2): two lanes of work per instruction.
__device__ __forceinline__ float2 add2_rd(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rm.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 lds64(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

}  // namespace pyhst
