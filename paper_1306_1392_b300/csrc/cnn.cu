// Residual CNN prox: forward pass.
//
// Activation layout (bfloat16, 32 channels): per image and row, four
// "chunk planes" of 8 channels each, [row][chunk][x][8] -> 16 bytes per pixel
// and chunk.  Eight consecutive pixels of one chunk plane are one tensor-core
// core matrix (8 rows x 16 bytes), so the shifted windows of a 3x3
// convolution are plain descriptor offsets into the staged rows.
//
//   layer 1   (1 -> 32):  conv_first_kernel, CUDA cores (9 MACs per output)
//   layers 2-7 (32 -> 32): conv_mid_kernel, tcgen05 implicit GEMM:
//                          M = 128 pixels of one row, N = 32 output channels,
//                          K = 9 taps x 32 input channels in 18 steps of 16
//   layer 8   (32 -> 1) + residual: conv_last_kernel, CUDA cores
#include <cmath>

#include "common.cuh"
#include "tc.cuh"

namespace pyhst {
namespace {

constexpr int kC = 32;                         // hidden channels
constexpr int kMid = 6;                        // 32 -> 32 layers
constexpr int64_t kW1 = 0;                     // offsets in the flat parameter vector
constexpr int64_t kB1 = 9 * kC;
constexpr int64_t kMid0 = kB1 + kC;
constexpr int64_t kMidStride = 9 * kC * kC + kC;
constexpr int64_t kW8 = kMid0 + kMid * kMidStride;
constexpr int64_t kB8 = kW8 + 9 * kC;
constexpr int64_t kNParams = kB8 + 1;          // 56097

// ----------------------------------------------------------------- packing
// One 32 -> 32 layer as the B operand: 18 K-slices (tap t = 3u + v, half h:
// input channels 16h .. 16h+15), each [4 groups of 8 output channels][2 core
// matrices along K][8 rows][8 bf16] = 1 KB.
constexpr int kSliceBytes = 1024;
constexpr int kLayerBytes = 18 * kSliceBytes;

__global__ void pack_mid_kernel(const float *__restrict__ params, __nv_bfloat16 *__restrict__ packed) {
    const int l = blockIdx.y;                                    // 0 .. kMid-1
    const int i = blockIdx.x * blockDim.x + threadIdx.x;         // element within the layer
    if (i >= 18 * 512) return;
    const int slice = i >> 9, r = i & 511;
    const int t = slice >> 1, h = slice & 1;
    const int e = r & 7, row = (r >> 3) & 7, kc = (r >> 6) & 1, ng = r >> 7;
    const int cout = ng * 8 + row, cin = 16 * h + 8 * kc + e;
    const float w = params[kMid0 + l * kMidStride + ((int64_t)cout * kC + cin) * 9 + t];
    packed[(size_t)l * (kLayerBytes / 2) + i] = __float2bfloat16_rn(w);
}

__device__ __forceinline__ uint4 pack8(const float *v) {
    uint4 o;
    __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]), b1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 b2 = __floats2bfloat162_rn(v[4], v[5]), b3 = __floats2bfloat162_rn(v[6], v[7]);
    o.x = *reinterpret_cast<uint32_t *>(&b0);
    o.y = *reinterpret_cast<uint32_t *>(&b1);
    o.z = *reinterpret_cast<uint32_t *>(&b2);
    o.w = *reinterpret_cast<uint32_t *>(&b3);
    return o;
}

__device__ __forceinline__ void unpack8(uint4 u, float *v) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = __uint_as_float(w[j] << 16);
        v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
    }
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ----------------------------------------------------------------- layer 1
// One thread per pixel: 32 outputs from the 3x3 neighbourhood of z.
__global__ void __launch_bounds__(128) conv_first_kernel(const float *__restrict__ z, const float *__restrict__ params,
                                                         uint4 *__restrict__ act, int H, int W) {
    __shared__ float sw[9 * kC], sb[kC];
    for (int i = threadIdx.x; i < 9 * kC; i += 128) sw[i] = bf16r(params[kW1 + i]);
    if (threadIdx.x < kC) sb[threadIdx.x] = params[kB1 + threadIdx.x];
    __syncthreads();
    const int x = blockIdx.x * 128 + threadIdx.x, y = blockIdx.y, img = blockIdx.z;
    if (x >= W) return;
    const float *zi = z + (size_t)img * H * W;
    float nb[9];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const int yy = y + u - 1, xx = x + v - 1;
            nb[3 * u + v] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? zi[(size_t)yy * W + xx] : 0.0f;
        }
    uint4 *row = act + ((size_t)img * H + y) * 4 * W;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int ch = 8 * c + k;
            float a = 0.0f;
#pragma unroll
            for (int t = 0; t < 9; ++t) a = fmaf(sw[ch * 9 + t], nb[t], a);
            o[k] = fmaxf(a + sb[ch], 0.0f);
        }
        row[(size_t)c * W + x] = pack8(o);
    }
}

// ----------------------------------------------------------------- layers 2-7
constexpr int kR = 4;                              // output rows per CTA
constexpr int kXS = 130;                           // staged pixels per row: 128 + halo
constexpr int kInBytes = (kR + 2) * 4 * kXS * 16;  // 49,920
// Every address a descriptor of this kernel can reach (with either reading
// of LBO and SBO) lies below 80 KB; the allocation covers it.
constexpr int kMidSmem = 80 * 1024;
constexpr uint32_t kWaitLimit = 1u << 22;

__global__ void __launch_bounds__(256) conv_mid_kernel(const uint4 *__restrict__ in, uint4 *__restrict__ out,
                                                       const uint4 *__restrict__ wpack,
                                                       const float *__restrict__ bias, int H, int W,
                                                       unsigned *__restrict__ status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *s_in = sm;
    uint8_t *s_w = sm + kInBytes;
    __shared__ float s_bias[kC];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * kR, img = blockIdx.z;
    const uint4 *inb = in + (size_t)img * H * 4 * W;

    // stage rows y0-1 .. y0+kR, pixels x0-1 .. x0+128, zero outside the image
    for (int i = tid; i < (kR + 2) * 4 * kXS; i += 256) {
        const int px = i % kXS, rc = i / kXS, c = rc & 3, rr = rc >> 2;
        const int y = y0 - 1 + rr, x = x0 - 1 + px;
        const bool ok = y >= 0 && y < H && x >= 0 && x < W;
        tc::cp16(s_in + (size_t)i * 16, ok ? inb + ((size_t)(y * 4 + c) * W + x) : inb, ok ? 16u : 0u);
    }
    for (int i = tid; i < kLayerBytes / 16; i += 256) tc::cp16(s_w + (size_t)i * 16, wpack + i, 16u);
    if (tid < kC) s_bias[tid] = bias[tid];
    __syncwarp();
    if (warp == 0) tc::tmem_alloc(&s_tmem, kR * kC);
    if (tid == 0) tc::bar_init(&s_bar, 1);
    tc::cp_wait_all();
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tm = s_tmem;

    if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(s_in), b0 = tc::smem_u32(s_w);
        constexpr uint32_t idesc = tc::idesc_bf16(128, kC);
#pragma unroll 1
        for (int r = 0; r < kR; ++r)
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int u = t / 3, v = t % 3;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t a = a0 + (uint32_t)((((r + u) * 4 + 2 * h) * kXS + v) * 16);
                    const uint32_t b = b0 + (uint32_t)((2 * t + h) * kSliceBytes);
                    tc::mma_bf16(tm + (uint32_t)(r * kC), tc::sdesc(a, kXS * 16, 128), tc::sdesc(b, 128, 256), idesc,
                                 (t | h) != 0);
                }
            }
        tc::mma_commit(&s_bar);
    }
    __syncwarp();
    bool ok = __all_sync(0xffffffffu, tc::bar_wait(&s_bar, 0, kWaitLimit));
    if (!ok) {
        if (lane == 0) atomicOr(status, tc::kErrMmaTimeout);
        // let the MMAs drain before freeing TMEM; skip the epilogue
        tc::bar_wait(&s_bar, 0, kWaitLimit);
        ok = false;
    }
    tc::fence_after();
    if (ok) {
        // warp w reads TMEM lanes 32 (w % 4) .. +31 (pixels), rows 2 (w / 4), +1
        const int q = warp & 3, m = 32 * q + lane, x = x0 + m;
#pragma unroll 1
        for (int rr = 0; rr < 2; ++rr) {
            const int r = 2 * (warp >> 2) + rr, y = y0 + r;
            float v[32];
            tc::tmem_ld32(tm + ((uint32_t)(32 * q) << 16) + (uint32_t)(r * kC), v);
            if (x < W && y < H) {
#pragma unroll
                for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + s_bias[k], 0.0f);
                uint4 *row = out + ((size_t)img * H + y) * 4 * W;
#pragma unroll
                for (int c = 0; c < 4; ++c) row[(size_t)c * W + x] = pack8(v + 8 * c);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tm, kR * kC);
    }
}

// ----------------------------------------------------------------- layer 8
// One thread per pixel: r = sum over 3x3 x 32 of bf16(W_8) a_7, out = z + r + b_8.
__global__ void __launch_bounds__(128) conv_last_kernel(const uint4 *__restrict__ act, const float *__restrict__ z,
                                                        const float *__restrict__ params, float *__restrict__ out,
                                                        int H, int W) {
    __shared__ float sw[9 * kC];
    for (int i = threadIdx.x; i < 9 * kC; i += 128) {
        const int c = i / 9, t = i % 9;                    // params hold W_8[0][c][t]
        sw[t * kC + c] = bf16r(params[kW8 + i]);
    }
    __syncthreads();
    const int x = blockIdx.x * 128 + threadIdx.x, y = blockIdx.y, img = blockIdx.z;
    if (x >= W) return;
    const uint4 *a = act + (size_t)img * H * 4 * W;
    float acc = 0.0f;
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
        const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[8];
            unpack8(a[((size_t)yy * 4 + c) * W + xx], v);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = fmaf(sw[t * kC + 8 * c + k], v[k], acc);
        }
    }
    const size_t o = ((size_t)img * H + y) * W + x;
    out[o] = z[o] + (acc + params[kB8]);
}

struct CnnLayout {
    size_t packed, act0, act1, bytes;
};

CnnLayout cnn_layout(int n, int H, int W) {
    CnnLayout l{};
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    const size_t act = (size_t)n * H * W * 64;
    l.packed = take((size_t)kMid * kLayerBytes);
    l.act0 = take(act);
    l.act1 = take(act);
    l.bytes = off;
    return l;
}

bool cnn_sizes_ok(int n, int H, int W) { return n >= 1 && n <= 65535 && H >= 1 && W >= 1 && H <= 16384 && W <= 16384; }

}  // namespace

int cnn_forward(const float *params, const float *z, float *out, int n, int H, int W, void *ws, cudaStream_t st) {
    const CnnLayout L = cnn_layout(n, H, W);
    char *base = static_cast<char *>(ws);
    __nv_bfloat16 *packed = reinterpret_cast<__nv_bfloat16 *>(base + L.packed);
    uint4 *a0 = reinterpret_cast<uint4 *>(base + L.act0), *a1 = reinterpret_cast<uint4 *>(base + L.act1);
    unsigned *status = device_status_ptr();
    if (!status) return fail(PYHST_ERR_CUDA, "device status word unavailable");
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(conv_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMidSmem) != cudaSuccess)
            return cuda_status("conv_mid_kernel shared-memory attribute");
        attr_set[dev] = true;
    }
    pack_mid_kernel<<<dim3((18 * 512 + 255) / 256, kMid), 256, 0, st>>>(params, packed);
    int rc = cuda_status("pack_mid_kernel");
    if (rc) return rc;
    conv_first_kernel<<<dim3((W + 127) / 128, H, n), 128, 0, st>>>(z, params, a0, H, W);
    if ((rc = cuda_status("conv_first_kernel"))) return rc;
    uint4 *src = a0, *dst = a1;
    for (int l = 0; l < kMid; ++l) {
        conv_mid_kernel<<<dim3((W + 127) / 128, (H + kR - 1) / kR, n), 256, kMidSmem, st>>>(
            src, dst, reinterpret_cast<const uint4 *>(packed + (size_t)l * (kLayerBytes / 2)),
            params + kMid0 + l * kMidStride + 9 * kC * kC, H, W, status);
        if ((rc = cuda_status("conv_mid_kernel"))) return rc;
        uint4 *t = src;
        src = dst;
        dst = t;
    }
    conv_last_kernel<<<dim3((W + 127) / 128, H, n), 128, 0, st>>>(src, z, params, out, H, W);
    return cuda_status("conv_last_kernel");
}

size_t cnn_workspace_size(int n, int H, int W) { return cnn_sizes_ok(n, H, W) ? cnn_layout(n, H, W).bytes : 0; }

}  // namespace pyhst

using namespace pyhst;

extern "C" int64_t pyhst_cnn_param_count(void) { return kNParams; }

extern "C" size_t pyhst_cnn_workspace_size(int32_t n_images, int32_t ny, int32_t nx) {
    return cnn_workspace_size(n_images, ny, nx);
}

extern "C" int pyhst_cnn_forward(const float *params, const float *z, float *out, int32_t n_images, int32_t ny,
                                 int32_t nx, void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    if (!params || !z || !out) return fail(PYHST_ERR_INVALID_ARG, "params/z/out pointer is NULL");
    if (!cnn_sizes_ok(n_images, ny, nx))
        return fail(PYHST_ERR_INVALID_ARG, "sizes %d x %d x %d outside [1, 65535] x [1, 16384]^2", n_images, ny, nx);
    const size_t need = cnn_workspace_size(n_images, ny, nx);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    return cnn_forward(params, z, out, n_images, ny, nx, workspace, reinterpret_cast<cudaStream_t>(stream));
}
