// Residual CNN prox: forward pass.
//
// Activation layout (bfloat16, 32 channels): NHWC, 64 bytes per pixel, read
// and written as four 16-byte chunks of 8 channels.  Staged in shared memory
// as 64-byte rows (one per pixel) in the tensor core's 64-byte swizzle, so the
// shifted windows of a 3x3 convolution are plain descriptor offsets into the
// staged image rows.
//
//   layer 1   (1 -> 32):  conv_first_kernel, CUDA cores (9 MACs per output)
//   layers 2-7 (32 -> 32): conv_mid_kernel, tcgen05 implicit GEMM:
//                          M = 128 pixels of one row, N = 32 output channels,
//                          K = 9 taps x 32 input channels in 18 steps of 16
//   layer 8   (32 -> 1) + residual: conv_last_rows_kernel, CUDA cores
#include <cmath>
#include <algorithm>
#include <utility>

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
// One 32 -> 32 layer as the B operand, arranged for row reuse: an input row
// feeds output rows rho - 1, rho, rho + 1 through the kernel rows u = 2, 1, 0,
// so the weights of the three kernel rows are stacked along N:
// n = 32 j + c_out with u = 2 - j (N = 96).  Layout [v][n][32 input
// channels]: one 64-byte row per (v, n), its 16-byte chunk c stored at chunk
// c ^ ((row >> 1) & 3) (the tensor core's 64-byte swizzle, for a copy placed
// at a 1024-byte aligned address).
constexpr int kBRows = 3 * 96;
constexpr int kLayerBytes = kBRows * 64;        // 18,432

// kBwd packs the weights of the input-gradient convolution instead:
// W'[o = cin][i = cout][u][v] = W[cout][cin][2 - u][2 - v] (transposed, 180-degree flip).
template <bool kBwd>
__global__ void pack_mid_kernel(const float *__restrict__ params, __nv_bfloat16 *__restrict__ packed) {
    const int l = blockIdx.y;                                    // 0 .. kMid-1
    const int i = blockIdx.x * blockDim.x + threadIdx.x;         // logical element (v, n, c)
    if (i >= kBRows * kC) return;
    const int c = i & 31, row = i >> 5, v = row / 96, n = row % 96;
    const int j = n >> 5, o = n & 31, u = 2 - j;                 // output channel o of this conv
    const int64_t base = kMid0 + l * kMidStride;
    const float w = kBwd ? params[base + ((int64_t)c * kC + o) * 9 + (2 - u) * 3 + (2 - v)]
                         : params[base + ((int64_t)o * kC + c) * 9 + u * 3 + v];
    const int phys = row * kC + (((c >> 3) ^ ((row >> 1) & 3)) << 3) + (c & 7);
    packed[(size_t)l * (kLayerBytes / 2) + phys] = __float2bfloat16_rn(w);
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

// 16-byte chunk c (channels 8c .. 8c+7) of pixel (img, y, x)
__device__ __forceinline__ size_t act_idx(int img, int y, int x, int c, int H, int W) {
    return (((size_t)img * H + y) * W + x) * 4 + c;
}

// ----------------------------------------------------------------- layer 1
// One thread per pixel: 32 outputs from the 3x3 neighbourhood of z.  The
// CTA's 128 output pixels (64 B each, contiguous in NHWC) pass through shared
// memory so that the global stores are consecutive 16-byte words.
__global__ void __launch_bounds__(128) conv_first_kernel(const float *__restrict__ z, const float *__restrict__ params,
                                                         uint4 *__restrict__ act, int H, int W) {
    __shared__ __align__(16) float sw[9 * kC];         // [tap][channel]: four weights per 16-byte read
    __shared__ float sb[kC];
    __shared__ __align__(16) uint4 so[4][129];          // [chunk][pixel], one pad word per chunk row
    for (int i = threadIdx.x; i < 9 * kC; i += 128) {
        const int ch = i / 9, t = i - 9 * ch;           // params hold W_1[ch][0][t]
        sw[t * kC + ch] = bf16r(params[kW1 + i]);
    }
    if (threadIdx.x < kC) sb[threadIdx.x] = params[kB1 + threadIdx.x];
    __syncthreads();
    const int x0 = blockIdx.x * 128, x = x0 + threadIdx.x, y = blockIdx.y, img = blockIdx.z;
    if (x < W) {
        const float *zi = z + (size_t)img * H * W;
        float nb[9];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const int yy = y + u - 1, xx = x + v - 1;
                nb[3 * u + v] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? zi[(size_t)yy * W + xx] : 0.0f;
            }
        // per channel, taps summed in order 0 .. 8; channel pairs share paired
        // fmas (each half rounds as its scalar fma would)
        float2 a[kC / 2];
#pragma unroll
        for (int ch = 0; ch < kC / 2; ++ch) a[ch] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float2 zt = make_float2(nb[t], nb[t]);
#pragma unroll
            for (int q = 0; q < kC / 4; ++q) {
                const float4 w = *reinterpret_cast<const float4 *>(&sw[t * kC + 4 * q]);
                a[2 * q] = fma2(make_float2(w.x, w.y), zt, a[2 * q]);
                a[2 * q + 1] = fma2(make_float2(w.z, w.w), zt, a[2 * q + 1]);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float o[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                o[2 * k] = fmaxf(a[4 * c + k].x + sb[8 * c + 2 * k], 0.0f);
                o[2 * k + 1] = fmaxf(a[4 * c + k].y + sb[8 * c + 2 * k + 1], 0.0f);
            }
            so[c][threadIdx.x] = pack8(o);
        }
    }
    __syncthreads();
    const int npx = min(128, W - x0);
    uint4 *dst = act + act_idx(img, y, x0, 0, H, W);
    for (int e = threadIdx.x; e < 4 * npx; e += 128) dst[e] = so[e & 3][e >> 2];
}

// ----------------------------------------------------------------- layers 2-7
// Persistent and pipelined: one CTA per SM walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; a tile is kR output rows x 128 pixels.  Two
// input buffers and two TMEM accumulator halves: while the tensor core runs
// tile i, the CTA drains tile i-1 from TMEM (epilogue) and loads tile i+1.
constexpr int kR = 8;                              // output rows per tile
constexpr int kXS = 130;                           // staged pixels per row: 128 + halo
constexpr int kInBytes = ((kR + 2) * kXS * 64 + 1023) / 1024 * 1024;   // 84,992 per buffer
constexpr int kMidSmem = 1024 + 2 * kInBytes + kLayerBytes;         // + alignment slack
constexpr uint32_t kTmemCols = 2 * kR * kC;        // 512: two accumulator halves

struct MidTiles {
    int tx, ty, H, W;
    long total;
    __device__ void decode(long t, int &img, int &y0, int &x0) const {
        const long per = (long)tx * ty;
        img = (int)(t / per);
        const int rem = (int)(t % per);
        y0 = (rem / tx) * kR;
        x0 = (rem % tx) * 128;
    }
};

// MMA schedule of one tile (the same for every tile).  Input row rho
// (staged row rho + 1) and kernel rows j_lo .. j_hi of a K-slice (kernel
// column v, half h) update output rows rho - 1 + j_lo .. rho - 1 + j_hi in one
// MMA of N = 32 (j_hi - j_lo + 1).  A first pass (kernel row u = 0 of slice
// (v, h) = (0, 0)) initialises every output row; all later MMAs accumulate.
// The tile's output rows are split between kMmaWarps issuing warps, which
// issue in parallel into disjoint accumulator columns; an MMA whose rows
// straddle two warps is split.  The schedule is unrolled at compile time for
// each issuing warp: every offset is a constant, so the issuing thread sends a
// tile's MMAs back to back (a table of MMAs in shared memory cost it a load and
// the address arithmetic per MMA: measured 16 % slower over a forward pass,
// same bits).
constexpr int kMmaWarps = 2;
constexpr int kRowsPerMmaWarp = kR / kMmaWarps;

template <int G>
__device__ __forceinline__ void issue_tile(uint64_t a_desc, uint64_t b_desc, uint32_t d0) {
    auto one = [&](int rho, int slice, int jlo, int jhi, bool acc) {
        const int lo = max(jlo, G * kRowsPerMmaWarp - rho + 1);
        const int hi = min(jhi, (G + 1) * kRowsPerMmaWarp - rho);
        if (lo > hi) return;
        const int v = slice >> 1, h = slice & 1;
        const uint32_t a_off = (uint32_t)(((rho + 1) * kXS + v) * 64 + h * 32);
        const uint32_t b_off = (uint32_t)((v * 96 + lo * 32) * 64 + h * 32);
        tc::mma_bf16(d0 + (uint32_t)((rho - 1 + lo) * kC), a_desc + (a_off >> 4), b_desc + (b_off >> 4),
                     tc::idesc_bf16(128, 32 * (hi - lo + 1)), acc);
    };
#pragma unroll
    for (int rho = -1; rho <= kR - 2; ++rho) one(rho, 0, 2, 2, false);
#pragma unroll
    for (int slice = 0; slice < 6; ++slice) {
#pragma unroll
        for (int rho = -1; rho <= kR; ++rho) {
            const int jlo = rho < 1 ? 1 - rho : 0;
            const int jhi = min(slice == 0 ? 1 : 2, kR - rho);
            if (jlo <= jhi) one(rho, slice, jlo, jhi, true);
        }
    }
}

constexpr int kWorkers = 256;                     // worker threads after the issuing warps (512: no gain)
constexpr int kWRows = kR / (kWorkers / 128);     // output rows a worker warp drains per tile
static_assert(kWorkers % 128 == 0 && kR % (kWorkers / 128) == 0, "worker warps: whole lane quarters");
constexpr int kMidThreads = 32 * kMmaWarps + kWorkers;

// Forward: out = bf16(ReLU(conv(in) + bias)).  kBwd (input gradient of a
// layer): out = bf16(conv'(in) masked by aux > 0), where in is the gradient
// of the layer's pre-activation, conv' uses the transposed, flipped weights
// and aux holds the previous layer's activations (the ReLU derivative).
//
// Warps 0 .. kMmaWarps-1 issue the tensor-core work; the next 8 warps stage
// tiles and drain the accumulators.  Per tile i (buffer and accumulator half
// b = i & 1):
//   loaded[b]  workers -> MMA warps: tile i staged and visible to the tensor core
//   mma[b]     tcgen05.commit of every MMA warp -> workers: accumulators complete
//   tfree[b]   workers -> MMA warps: accumulator half b read out
template <bool kBwd>
__global__ void __launch_bounds__(kMidThreads, 1) conv_mid_kernel(const uint4 *__restrict__ in,
                                                                  uint4 *__restrict__ out,
                                                                  const uint4 *__restrict__ wpack,
                                                                  const float *__restrict__ bias,
                                                                  const uint4 *__restrict__ aux, MidTiles T,
                                                                  unsigned *__restrict__ status,
                                                                  uint32_t wait_limit) {
    extern __shared__ __align__(1024) uint8_t sm_raw[];
    // swizzled operands need 1024-byte aligned shared addresses
    uint8_t *sm = sm_raw + ((1024 - (tc::smem_u32(sm_raw) & 1023)) & 1023);
    uint8_t *s_in[2] = {sm, sm + kInBytes};
    uint8_t *s_w = sm + 2 * kInBytes;
    __shared__ float s_bias[kC];
    __shared__ __align__(8) uint64_t bar_loaded[2], bar_mma[2], bar_tfree[2], bar_drain[kMmaWarps];
    // a worker warp's 32 output pixels, chunk-major, on their way to coalesced
    // stores (rows of 34 words: both the chunk-row writes and the
    // pixel-major reads are free of bank conflicts)
    __shared__ __align__(16) uint4 s_out[kWorkers / 32][4][34];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long first = blockIdx.x, stride = gridDim.x;
    const int n_my = first < T.total ? (int)((T.total - 1 - first) / stride + 1) : 0;

    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, kTmemCols);
        if (lane == 0) {
            for (int b = 0; b < 2; ++b) {
                tc::bar_init(&bar_loaded[b], kWorkers);
                tc::bar_init(&bar_mma[b], kMmaWarps);
                tc::bar_init(&bar_tfree[b], kWorkers);
            }
            for (int g = 0; g < kMmaWarps; ++g) tc::bar_init(&bar_drain[g], 1);
        }
    } else if (warp >= kMmaWarps) {
        const int w = tid - 32 * kMmaWarps;
        for (int i = w; i < kLayerBytes / 16; i += kWorkers) tc::cp16(s_w + (size_t)i * 16, wpack + i, 16u);
        if (w < kC) s_bias[w] = kBwd ? 0.0f : bias[w];
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tm = s_tmem;
    bool ok = true;

    if (warp < kMmaWarps) {
        // ---------------------------------------------------------- MMA warps
        const uint32_t b0 = tc::smem_u32(s_w);
        const uint64_t hi = tc::sdesc_sw64(0, 512);          // descriptor without its start address
        for (int i = 0; i < n_my && ok; ++i) {
            const int b = i & 1;
            bool good = tc::bar_wait(&bar_loaded[b], (uint32_t)((i >> 1) & 1), wait_limit);
            if (good && i >= 2) good = tc::bar_wait(&bar_tfree[b], (uint32_t)(((i >> 1) - 1) & 1), wait_limit);
            ok = __all_sync(0xffffffffu, good);
            if (!ok) break;
            tc::fence_after();
            const uint32_t d0 = tm + (uint32_t)(b * kR * kC);
            // start addresses below 2^18 bytes: the 14-bit field takes the offsets without a carry
            const uint64_t a_desc = hi | (uint64_t)(tc::smem_u32(s_in[b]) >> 4), b_desc = hi | (uint64_t)(b0 >> 4);
            if (lane == 0) {
                static_assert(kMmaWarps == 2, "one issue_tile instantiation per issuing warp");
                if (warp == 0)
                    issue_tile<0>(a_desc, b_desc, d0);
                else
                    issue_tile<1>(a_desc, b_desc, d0);
            }
            __syncwarp();
            if (lane == 0) tc::mma_commit(&bar_mma[b]);
            __syncwarp();
        }
        if (!ok && lane == 0) atomicOr(status, tc::kErrMmaTimeout);
        // every MMA this warp issued has finished before the tensor memory is
        // freed: a commit tracks all of the issuing thread's earlier MMAs (the
        // wait keeps the default limit even when the pipeline waits are lowered)
        if (lane == 0) {
            tc::mma_commit(&bar_drain[warp]);
            if (!tc::bar_wait(&bar_drain[warp], 0, kDefaultWaitLimit)) atomicOr(status, tc::kErrMmaTimeout);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- workers
        const int w = tid - 32 * kMmaWarps, ww = warp - kMmaWarps;   // worker warp 0 .. kWorkers / 32 - 1
        const int q = warp & 3;                            // TMEM lanes 32 q .. 32 q + 31 (pixels)
        const int r0 = kWRows * (ww >> 2);                 // output rows r0 .. r0 + kWRows - 1
        auto stage = [&](int i) {                          // tile i into buffer i & 1
            int img, y0, x0;
            T.decode(first + (long)i * stride, img, y0, x0);
            uint8_t *buf = s_in[i & 1];
            for (int e = w; e < (kR + 2) * kXS * 4; e += kWorkers) {
                const int c = e & 3, qq = e >> 2, px = qq % kXS, rr = qq / kXS;
                const int y = y0 - 1 + rr, x = x0 - 1 + px;
                const bool in_img = y >= 0 && y < T.H && x >= 0 && x < T.W;
                tc::cp16(buf + (size_t)qq * 64 + ((c ^ ((qq >> 1) & 3)) << 4),
                         in_img ? in + act_idx(img, y, x, c, T.H, T.W) : in, in_img ? 16u : 0u);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        auto publish = [&](int i) {                        // staged tile i -> MMA warp
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            tc::fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&bar_loaded[i & 1]))
                         : "memory");
        };
        if (n_my > 0) {
            stage(0);
            publish(0);
        }
        for (int i = 0; i <= n_my; ++i) {
            if (i >= 1) {
                const int j = i - 1;
                ok = __all_sync(0xffffffffu, tc::bar_wait(&bar_mma[j & 1], (uint32_t)((j >> 1) & 1), wait_limit));
                if (!ok) {
                    if (lane == 0) atomicOr(status, tc::kErrMmaTimeout);
                    break;
                }
                tc::fence_after();
            }
            if (i + 1 < n_my) stage(i + 1);                 // buffer of tile i-1: its MMAs are done
            if (i >= 1) {
                const int j = i - 1, bj = j & 1;
                int img, y0, x0;
                T.decode(first + (long)j * stride, img, y0, x0);
                const int x = x0 + 32 * q + lane;
#pragma unroll 1
                for (int rr = 0; rr < kWRows; ++rr) {
                    const int r = r0 + rr, y = y0 + r;
                    float v[32];
                    tc::tmem_ld32(tm + ((uint32_t)(32 * q) << 16) + (uint32_t)((bj * kR + r) * kC), v);
                    const bool row_in = y < T.H;
                    if (row_in && x < T.W) {
                        const size_t px = act_idx(img, y, x, 0, T.H, T.W);
                        if (kBwd) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                float a[8];
                                unpack8(aux[px + c], a);
#pragma unroll
                                for (int k = 0; k < 8; ++k) v[8 * c + k] = a[k] > 0.0f ? v[8 * c + k] : 0.0f;
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k] + s_bias[k], 0.0f);
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) s_out[ww][c][lane] = pack8(v + 8 * c);
                    }
                    __syncwarp();
                    // the warp's pixels x0 + 32 q .. + 31 are consecutive in NHWC: 16-byte word
                    // e = 4 pixel + chunk of them, stored by lane e mod 32 (512 contiguous bytes per store)
                    if (row_in) {
                        const int xw = x0 + 32 * q, npx = min(32, T.W - xw);
                        if (npx > 0) {
                            uint4 *dst = out + act_idx(img, y, xw, 0, T.H, T.W);
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int e = lane + 32 * k;
                                if ((e >> 2) < npx) dst[e] = s_out[ww][e & 3][e >> 2];
                            }
                        }
                    }
                    __syncwarp();
                }
                tc::fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&bar_tfree[bj])) : "memory");
            }
            if (i + 1 < n_my) publish(i + 1);
        }
    }
    // every thread gets here (all waits are bounded; the MMA warps have drained
    // their tensor-core work, and the workers' copies were waited for before
    // each publish, so none is in flight)
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tm, kTmemCols);
    }
}

// ----------------------------------------------------------------- layer 8
// r = sum over 3x3 x 32 of bf16(W_8) a_7, out = z + r + b_8.
// A CTA of 128 threads reconstructs kLR rows x 128 pixels; its kLR + 2 input
// rows (130 pixels each, 64 B per pixel) are staged once in shared memory,
// channel-chunk-major, by asynchronous 16-byte copies, so that a warp's reads
// of one (tap, chunk) are 32 consecutive 16-byte words (staging three rows
// per output row cost 4 % more over a forward pass).  A thread owns one
// column: each staged 8-channel chunk it unpacks feeds up to three of its
// output rows (kernel rows u = 0, 1, 2), the 24 weights of a (kernel column,
// chunk) pair stay in registers while it walks the rows, and channel pairs
// accumulate in paired float32 (two partial sums per row, added at the end).
template <int kLR>
__global__ void __launch_bounds__(128) conv_last_rows_kernel(const uint4 *__restrict__ act,
                                                             const float *__restrict__ z,
                                                             const float *__restrict__ params,
                                                             float *__restrict__ out, int H, int W) {
    extern __shared__ __align__(16) uint4 srows[];                 // [kLR + 2][4][130]
    __shared__ __align__(16) float sw[9 * kC];                      // [tap][channel]
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * kLR, img = blockIdx.z, tid = threadIdx.x;
    for (int i = tid; i < 9 * kC; i += 128) {
        const int c = i / 9, t = i % 9;                              // params hold W_8[0][c][t]
        sw[t * kC + c] = bf16r(params[kW8 + i]);
    }
    for (int rr = 0; rr < kLR + 2; ++rr) {                           // asynchronous copies, all in flight at once
        const int yy = y0 - 1 + rr;
        const bool row_in = yy >= 0 && yy < H;
        const uint4 *src_row = act + act_idx(img, row_in ? yy : 0, 0, 0, H, W);
        for (int e = tid; e < 130 * 4; e += 128) {                  // e = 4 px + c: consecutive 16-byte words
            const int px = e >> 2, c = e & 3, xx = x0 - 1 + px;
            const bool in = row_in && xx >= 0 && xx < W;
            tc::cp16(&srows[(rr * 4 + c) * 130 + px], in ? src_row + 4 * xx + c : act, in ? 16u : 0u);
        }
    }
    tc::cp_wait_all();
    __syncthreads();
    const int x = x0 + tid;
    if (x >= W) return;
    float2 acc[kLR];
#pragma unroll
    for (int r = 0; r < kLR; ++r) acc[r] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const int xx = x + v - 1;
        if (xx < 0 || xx >= W) continue;                            // taps outside the image add nothing
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 wt[3][4];                                         // kernel rows u = 0, 1, 2
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const float4 w0 = *reinterpret_cast<const float4 *>(&sw[(3 * u + v) * kC + 8 * c]);
                const float4 w1 = *reinterpret_cast<const float4 *>(&sw[(3 * u + v) * kC + 8 * c + 4]);
                wt[u][0] = make_float2(w0.x, w0.y);
                wt[u][1] = make_float2(w0.z, w0.w);
                wt[u][2] = make_float2(w1.x, w1.y);
                wt[u][3] = make_float2(w1.z, w1.w);
            }
#pragma unroll
            for (int rr = 0; rr < kLR + 2; ++rr) {
                const int yy = y0 - 1 + rr;
                if (yy < 0 || yy >= H) continue;
                float p[8];
                unpack8(srows[(rr * 4 + c) * 130 + tid + v], p);
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int r = rr - u;                            // output row y0 + r reads row yy at kernel row u
                    if (r < 0 || r >= kLR) continue;
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[r] = fma2(wt[u][k], make_float2(p[2 * k], p[2 * k + 1]), acc[r]);
                }
            }
        }
    }
    const float b8 = params[kB8];
#pragma unroll
    for (int r = 0; r < kLR; ++r) {
        const int y = y0 + r;
        if (y >= H) break;
        const size_t o = ((size_t)img * H + y) * W + x;
        out[o] = z[o] + ((acc[r].x + acc[r].y) + b8);
    }
}
template <int kLR> constexpr int last_rows_smem() { return (kLR + 2) * 4 * 130 * 16; }
// rows per CTA: 4 (49.9 KB of staged rows, four CTAs per SM; 2 was slower, the
// one-row kernel it replaced 4 % slower over a forward pass)
constexpr int kLastRows = 4;

bool cnn_sizes_ok(int n, int H, int W) { return n >= 1 && n <= 65535 && H >= 1 && W >= 1 && H <= 16384 && W <= 16384; }

int set_smem_attrs() {
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status("cudaGetDevice");
    if (dev >= 0 && dev < 64 && done[dev]) return PYHST_OK;
    if (cudaFuncSetAttribute(conv_mid_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMidSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(conv_mid_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMidSmem) !=
            cudaSuccess)
        return cuda_status("conv_mid_kernel shared-memory attribute");
    if (cudaFuncSetAttribute(conv_last_rows_kernel<kLastRows>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             last_rows_smem<kLastRows>()) != cudaSuccess)
        return cuda_status("conv_last_rows_kernel shared-memory attribute");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return PYHST_OK;
}

int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

int launch_conv_mid(bool bwd, const uint4 *in, uint4 *out, const __nv_bfloat16 *packed_layer, const float *bias,
                    const uint4 *aux, int n, int H, int W, unsigned *status, cudaStream_t st) {
    MidTiles T;
    T.tx = (W + 127) / 128;
    T.ty = (H + kR - 1) / kR;
    T.H = H;
    T.W = W;
    T.total = (long)n * T.tx * T.ty;
    const int grid = (int)std::min<long>(T.total, sm_count());
    const uint4 *wp = reinterpret_cast<const uint4 *>(packed_layer);
    if (bwd)
        conv_mid_kernel<true><<<grid, kMidThreads, kMidSmem, st>>>(in, out, wp, bias, aux, T, status,
                                                                   pipeline_wait_limit());
    else
        conv_mid_kernel<false><<<grid, kMidThreads, kMidSmem, st>>>(in, out, wp, bias, aux, T, status,
                                                                    pipeline_wait_limit());
    return cuda_status("conv_mid_kernel");
}

// Forward pass.  acts: NULL (activations ping-pong between act_a and act_b)
// or 7 buffers that keep a_1 .. a_7 for the backward pass.
int forward_pass(const float *params, const float *z, float *out, int n, int H, int W, __nv_bfloat16 *packed,
                 uint4 *act_a, uint4 *act_b, uint4 *const *acts, cudaStream_t st) {
    unsigned *status = device_status_ptr();
    if (!status) return fail(PYHST_ERR_CUDA, "device status word unavailable");
    int rc = set_smem_attrs();
    if (rc) return rc;
    pack_mid_kernel<false><<<dim3((kBRows * kC + 255) / 256, kMid), 256, 0, st>>>(params, packed);
    if ((rc = cuda_status("pack_mid_kernel"))) return rc;
    uint4 *src = acts ? acts[0] : act_a;
    conv_first_kernel<<<dim3((W + 127) / 128, H, n), 128, 0, st>>>(z, params, src, H, W);
    if ((rc = cuda_status("conv_first_kernel"))) return rc;
    for (int l = 0; l < kMid; ++l) {
        uint4 *dst = acts ? acts[l + 1] : (src == act_a ? act_b : act_a);
        if ((rc = launch_conv_mid(false, src, dst, packed + (size_t)l * (kLayerBytes / 2),
                                  params + kMid0 + l * kMidStride + 9 * kC * kC, nullptr, n, H, W, status, st)))
            return rc;
        src = dst;
    }
    conv_last_rows_kernel<kLastRows><<<dim3((W + 127) / 128, (H + kLastRows - 1) / kLastRows, n), 128,
                                        last_rows_smem<kLastRows>(), st>>>(src, z, params, out, H, W);
    return cuda_status("conv_last_rows_kernel");
}


// ----------------------------------------------------------------- training
// Mean squared error over all pixels of the batch: d = out - target,
// dout = (2/N) d, and FP64 partial sums of d^2 per block (fixed grid).
constexpr int kLossBlocks = 592;

__device__ __forceinline__ double block_sum256(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = l < 8 ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(256) loss_kernel(const float *__restrict__ out, const float *__restrict__ target,
                                                   size_t N, float scale, float *__restrict__ dout,
                                                   double *__restrict__ part) {
    __shared__ double red[8];
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (size_t)gridDim.x * 256) {
        const float d = out[i] - target[i];
        dout[i] = scale * d;
        acc += (double)d * (double)d;
    }
    acc = block_sum256(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) loss_final_kernel(const double *__restrict__ part, int nb, double invN,
                                                         double *__restrict__ loss) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) acc += part[i];
    acc = block_sum256(acc, red);
    if (threadIdx.x == 0) *loss = acc * invN;
}

// Gradient of the last layer's input: dA_7[p][c] = sum_{u,v} W_8[c][u][v]
// dout[p - (u-1, v-1)], masked by a_7 > 0 (the ReLU), stored as bf16 planes.
__global__ void __launch_bounds__(128) conv_last_bwd_kernel(const float *__restrict__ dout,
                                                            const uint4 *__restrict__ a7,
                                                            const float *__restrict__ params,
                                                            uint4 *__restrict__ dz, int H, int W) {
    __shared__ float sw[9 * kC];
    for (int i = threadIdx.x; i < 9 * kC; i += 128) {
        const int c = i / 9, t = i % 9;
        sw[t * kC + c] = bf16r(params[kW8 + i]);
    }
    __syncthreads();
    const int x = blockIdx.x * 128 + threadIdx.x, y = blockIdx.y, img = blockIdx.z;
    if (x >= W) return;
    float d[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
        d[t] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? dout[((size_t)img * H + yy) * W + xx] : 0.0f;
    }
    const size_t px = act_idx(img, y, x, 0, H, W);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float a[8], o[8];
        unpack8(a7[px + c], a);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float acc = 0.0f;
#pragma unroll
            for (int t = 0; t < 9; ++t) acc = fmaf(sw[t * kC + 8 * c + k], d[t], acc);
            o[k] = a[k] > 0.0f ? acc : 0.0f;
        }
        dz[px + c] = pack8(o);
    }
}

// Weight gradients are sums over every pixel of the batch.  kGradCtas CTAs
// each accumulate the tiles blockIdx.x, blockIdx.x + kGradCtas, ... in
// registers and write one partial row; reduce_partials adds the rows in a
// fixed order (deterministic).  Tiles: 8 rows x 32 pixels.
constexpr int kGradCtas = 296;
constexpr int kTR = 8, kTC = 32;
constexpr int kPartRow = 9 * kC * kC + kC;        // 9248: the widest layer (W then b)
constexpr int kGradSmem = ((kTR + 2) * (kTC + 2) * kC + kTR * kTC * kC) * 4;   // 76,288 B

// stage bf16 planes of rows y0-1 .. y0+kTR, pixels x0-1 .. x0+kTC (halo 1,
// zero outside) as float32 [kTR+2][kTC+2][32]
__device__ __forceinline__ void stage_halo(const uint4 *__restrict__ src, float *dst, int img, int y0, int x0, int H,
                                           int W) {
    for (int i = threadIdx.x; i < (kTR + 2) * (kTC + 2) * 4; i += blockDim.x) {
        const int c = i & 3, px = i >> 2, rr = px / (kTC + 2), cc = px % (kTC + 2);
        const int y = y0 - 1 + rr, x = x0 - 1 + cc;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (y >= 0 && y < H && x >= 0 && x < W) unpack8(src[act_idx(img, y, x, c, H, W)], v);
        float4 *d = reinterpret_cast<float4 *>(dst + px * kC + 8 * c);
        d[0] = make_float4(v[0], v[1], v[2], v[3]);
        d[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

// the tile itself (no halo) as float32 [kTR][kTC][32]
__device__ __forceinline__ void stage_tile(const uint4 *__restrict__ src, float *dst, int img, int y0, int x0, int H,
                                           int W) {
    for (int i = threadIdx.x; i < kTR * kTC * 4; i += blockDim.x) {
        const int c = i & 3, px = i >> 2, rr = px / kTC, cc = px % kTC;
        const int y = y0 + rr, x = x0 + cc;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (y < H && x < W) unpack8(src[act_idx(img, y, x, c, H, W)], v);
        float4 *d = reinterpret_cast<float4 *>(dst + px * kC + 8 * c);
        d[0] = make_float4(v[0], v[1], v[2], v[3]);
        d[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

// 32 -> 32 layer: gW[o][c][t] = sum_p dz[p][o] a[p + tap t][c], gb[o] = sum_p dz[p][o].
// Thread: input channel c = lane, output channels 4 warp .. 4 warp + 3, all 9 taps.
__global__ void __launch_bounds__(256) wgrad_mid_kernel(const uint4 *__restrict__ dz, const uint4 *__restrict__ act,
                                                        int n, int H, int W, float *__restrict__ part) {
    extern __shared__ float4 smg4[];
    float *s_a = reinterpret_cast<float *>(smg4);
    float *s_d = s_a + (kTR + 2) * (kTC + 2) * kC;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    float acc[4][9], accb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        accb[j] = 0.0f;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[j][t] = 0.0f;
    }
    const int tx = (W + kTC - 1) / kTC, ty = (H + kTR - 1) / kTR;
    const long total = (long)n * tx * ty;
    for (long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int img = (int)(tile / ((long)tx * ty)), rem = (int)(tile % ((long)tx * ty));
        const int y0 = (rem / tx) * kTR, x0 = (rem % tx) * kTC;
        __syncthreads();
        stage_halo(act, s_a, img, y0, x0, H, W);
        stage_tile(dz, s_d, img, y0, x0, H, W);
        __syncthreads();
#pragma unroll 2
        for (int p = 0; p < kTR * kTC; ++p) {
            const int r = p / kTC, cc = p % kTC;
            const float4 d = *reinterpret_cast<const float4 *>(s_d + p * kC + 4 * g);
            accb[0] += d.x;
            accb[1] += d.y;
            accb[2] += d.z;
            accb[3] += d.w;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float a = s_a[((r + t / 3) * (kTC + 2) + cc + t % 3) * kC + lane];
                acc[0][t] = fmaf(d.x, a, acc[0][t]);
                acc[1][t] = fmaf(d.y, a, acc[1][t]);
                acc[2][t] = fmaf(d.z, a, acc[2][t]);
                acc[3][t] = fmaf(d.w, a, acc[3][t]);
            }
        }
    }
    float *row = part + (size_t)blockIdx.x * kPartRow;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int o = 4 * g + j;
#pragma unroll
        for (int t = 0; t < 9; ++t) row[(o * kC + lane) * 9 + t] = acc[j][t];
        if (lane == 0) row[9 * kC * kC + o] = accb[j];
    }
}

// First layer: gW_1[c][t] = sum_p dz_1[p][c] z[p + tap t], gb_1[c] = sum_p dz_1[p][c].
// Last layer: gW_8[c][t] = sum_p dout[p] a_7[p + tap t][c], gb_8 = sum_p dout[p].
// Thread: channel c = lane, tap t = warp (9 warps).
template <bool kLast>
__global__ void __launch_bounds__(288) wgrad_edge_kernel(const uint4 *__restrict__ planes, const float *__restrict__ img1,
                                                         int n, int H, int W, float *__restrict__ part) {
    extern __shared__ float4 smg4[];
    float *s_p = reinterpret_cast<float *>(smg4);                  // planes: halo (last) or tile (first)
    float *s_1 = s_p + (kTR + 2) * (kTC + 2) * kC;                 // one-channel image: tile (last) or halo (first)
    const int c = threadIdx.x & 31, t = threadIdx.x >> 5, u = t / 3, v = t % 3;
    float acc = 0.0f, accb = 0.0f;
    const int tx = (W + kTC - 1) / kTC, ty = (H + kTR - 1) / kTR;
    const long total = (long)n * tx * ty;
    for (long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int im = (int)(tile / ((long)tx * ty)), rem = (int)(tile % ((long)tx * ty));
        const int y0 = (rem / tx) * kTR, x0 = (rem % tx) * kTC;
        __syncthreads();
        if (kLast) {
            stage_halo(planes, s_p, im, y0, x0, H, W);
            for (int i = threadIdx.x; i < kTR * kTC; i += blockDim.x) {
                const int y = y0 + i / kTC, x = x0 + i % kTC;
                s_1[i] = (y < H && x < W) ? img1[((size_t)im * H + y) * W + x] : 0.0f;
            }
        } else {
            stage_tile(planes, s_p, im, y0, x0, H, W);
            for (int i = threadIdx.x; i < (kTR + 2) * (kTC + 2); i += blockDim.x) {
                const int y = y0 - 1 + i / (kTC + 2), x = x0 - 1 + i % (kTC + 2);
                s_1[i] = (y >= 0 && y < H && x >= 0 && x < W) ? img1[((size_t)im * H + y) * W + x] : 0.0f;
            }
        }
        __syncthreads();
        for (int p = 0; p < kTR * kTC; ++p) {
            const int r = p / kTC, cc = p % kTC;
            const int h = (r + u) * (kTC + 2) + cc + v;               // halo index of p + tap
            if (kLast) {
                const float d = s_1[p];
                acc = fmaf(d, s_p[h * kC + c], acc);
                accb += d;
            } else {
                const float d = s_p[p * kC + c];
                acc = fmaf(d, s_1[h], acc);
                accb += d;
            }
        }
    }
    float *row = part + (size_t)blockIdx.x * kPartRow;
    row[c * 9 + t] = acc;
    if (t == 0) {
        if (kLast) {
            if (c == 0) row[9 * kC] = accb;
        } else {
            row[9 * kC + c] = accb;
        }
    }
}

// grad[j] = sum over the partial rows b = 0 .. nb-1 of part[b][j], in order.
__global__ void reduce_partials_kernel(const float *__restrict__ part, int nb, int len, float *__restrict__ grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(size_t)b * kPartRow + j];
    grad[j] = (float)acc;
}

// Adam (Kingma & Ba 2015): c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

struct TrainLayout {
    size_t packed_f, packed_b, acts[7], dz[2], out, dout, part, loss_part, bytes;
};

TrainLayout train_layout(int n, int H, int W) {
    TrainLayout l{};
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    const size_t act = (size_t)n * H * W * 64, img = (size_t)n * H * W * 4;
    l.packed_f = take((size_t)kMid * kLayerBytes);
    l.packed_b = take((size_t)kMid * kLayerBytes);
    for (auto &a : l.acts) a = take(act);
    for (auto &d : l.dz) d = take(act);
    l.out = take(img);
    l.dout = take(img);
    l.part = take((size_t)kGradCtas * kPartRow * sizeof(float));
    l.loss_part = take(kLossBlocks * sizeof(double));
    l.bytes = off;
    return l;
}

int set_grad_attrs() {
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status("cudaGetDevice");
    if (dev >= 0 && dev < 64 && done[dev]) return PYHST_OK;
    if (cudaFuncSetAttribute(wgrad_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGradSmem) != cudaSuccess ||
        cudaFuncSetAttribute(wgrad_edge_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGradSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(wgrad_edge_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGradSmem) !=
            cudaSuccess)
        return cuda_status("weight-gradient shared-memory attribute");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return PYHST_OK;
}

int reduce_into(const float *part, int len, float *grad, cudaStream_t st) {
    reduce_partials_kernel<<<(len + 255) / 256, 256, 0, st>>>(part, kGradCtas, len, grad);
    return cuda_status("reduce_partials_kernel");
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

}  // namespace

int cnn_forward(const float *params, const float *z, float *out, int n, int H, int W, void *ws, cudaStream_t st) {
    const CnnLayout L = cnn_layout(n, H, W);
    char *base = static_cast<char *>(ws);
    return forward_pass(params, z, out, n, H, W, reinterpret_cast<__nv_bfloat16 *>(base + L.packed),
                        reinterpret_cast<uint4 *>(base + L.act0), reinterpret_cast<uint4 *>(base + L.act1), nullptr,
                        st);
}

int cnn_grad(const float *params, const float *z, const float *target, int n, int H, int W, float *grad,
             double *loss, void *ws, cudaStream_t st) {
    const TrainLayout L = train_layout(n, H, W);
    char *base = static_cast<char *>(ws);
    auto P = [&](size_t o) { return reinterpret_cast<uint4 *>(base + o); };
    __nv_bfloat16 *packed_f = reinterpret_cast<__nv_bfloat16 *>(base + L.packed_f);
    __nv_bfloat16 *packed_b = reinterpret_cast<__nv_bfloat16 *>(base + L.packed_b);
    uint4 *acts[7];
    for (int i = 0; i < 7; ++i) acts[i] = P(L.acts[i]);
    float *out = reinterpret_cast<float *>(base + L.out), *dout = reinterpret_cast<float *>(base + L.dout);
    float *part = reinterpret_cast<float *>(base + L.part);
    double *lpart = reinterpret_cast<double *>(base + L.loss_part);
    unsigned *status = device_status_ptr();
    if (!status) return fail(PYHST_ERR_CUDA, "device status word unavailable");
    int rc = set_grad_attrs();
    if (rc) return rc;

    if ((rc = forward_pass(params, z, out, n, H, W, packed_f, nullptr, nullptr, acts, st))) return rc;
    const size_t N = (size_t)n * H * W;
    loss_kernel<<<kLossBlocks, 256, 0, st>>>(out, target, N, (float)(2.0 / (double)N), dout, lpart);
    if (loss) loss_final_kernel<<<1, 256, 0, st>>>(lpart, kLossBlocks, 1.0 / (double)N, loss);
    pack_mid_kernel<true><<<dim3((kBRows * kC + 255) / 256, kMid), 256, 0, st>>>(params, packed_b);
    if ((rc = cuda_status("loss / packing kernels"))) return rc;

    // layer 8
    wgrad_edge_kernel<true><<<kGradCtas, 288, kGradSmem, st>>>(acts[6], dout, n, H, W, part);
    if ((rc = cuda_status("wgrad_edge_kernel (last)"))) return rc;
    if ((rc = reduce_into(part, 9 * kC + 1, grad + kW8, st))) return rc;
    uint4 *dzc = P(L.dz[0]), *dzn = P(L.dz[1]);
    conv_last_bwd_kernel<<<dim3((W + 127) / 128, H, n), 128, 0, st>>>(dout, acts[6], params, dzc, H, W);
    if ((rc = cuda_status("conv_last_bwd_kernel"))) return rc;
    // layers 7 .. 2 (mid index l: input a_{l+1} = acts[l])
    for (int l = kMid - 1; l >= 0; --l) {
        wgrad_mid_kernel<<<kGradCtas, 256, kGradSmem, st>>>(dzc, acts[l], n, H, W, part);
        if ((rc = cuda_status("wgrad_mid_kernel"))) return rc;
        if ((rc = reduce_into(part, kPartRow, grad + kMid0 + l * kMidStride, st))) return rc;
        if ((rc = launch_conv_mid(true, dzc, dzn, packed_b + (size_t)l * (kLayerBytes / 2), nullptr, acts[l], n, H, W,
                                  status, st)))
            return rc;
        std::swap(dzc, dzn);
    }
    // layer 1
    wgrad_edge_kernel<false><<<kGradCtas, 288, kGradSmem, st>>>(dzc, z, n, H, W, part);
    if ((rc = cuda_status("wgrad_edge_kernel (first)"))) return rc;
    return reduce_into(part, 9 * kC + kC, grad + kW1, st);
}

size_t cnn_train_workspace_size(int n, int H, int W) { return cnn_sizes_ok(n, H, W) ? train_layout(n, H, W).bytes : 0; }

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

extern "C" size_t pyhst_cnn_train_workspace_size(int32_t n_images, int32_t ny, int32_t nx) {
    return cnn_train_workspace_size(n_images, ny, nx);
}

extern "C" int pyhst_cnn_grad(const float *params, const float *z, const float *target, int32_t n_images, int32_t ny,
                              int32_t nx, float *grad, double *loss, void *workspace, size_t ws_bytes,
                              pyhst_stream_t stream) {
    if (!params || !z || !target || !grad) return fail(PYHST_ERR_INVALID_ARG, "params/z/target/grad pointer is NULL");
    if (!cnn_sizes_ok(n_images, ny, nx))
        return fail(PYHST_ERR_INVALID_ARG, "sizes %d x %d x %d outside [1, 65535] x [1, 16384]^2", n_images, ny, nx);
    const size_t need = cnn_train_workspace_size(n_images, ny, nx);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    return cnn_grad(params, z, target, n_images, ny, nx, grad, loss, workspace, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int pyhst_cnn_adam(float *params, const float *grad, float *m, float *v, int64_t count, int32_t step,
                              float lr, float beta1, float beta2, float eps, pyhst_stream_t stream) {
    if (!params || !grad || !m || !v) return fail(PYHST_ERR_INVALID_ARG, "params/grad/m/v pointer is NULL");
    if (count < 1 || step < 1) return fail(PYHST_ERR_INVALID_ARG, "count and step must be >= 1");
    if (!(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(PYHST_ERR_INVALID_ARG, "need lr > 0, 0 <= beta1, beta2 < 1, eps > 0");
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, step)), c2 = 1.0 / (1.0 - std::pow((double)beta2, step));
    adam_kernel<<<(unsigned)((count + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        params, grad, m, v, count, lr, beta1, beta2, eps, (float)c1, (float)c2);
    return cuda_status("adam_kernel");
}
