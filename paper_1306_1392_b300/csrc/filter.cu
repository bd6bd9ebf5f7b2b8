// Flat/dark normalisation fused into the ramp filter (Sec. 2.3).
//
// For each detector row (slice z, angle a) the kernel loads the raw values,
// forms p = -ln((I - D) / (F - D)) (p = 0 where F - D <= 0; ratio clamped
// below at 1e-6), zero-pads to P, convolves circularly with the filter's
// spatial kernel h truncated to (-P/2, P/2) and keeps the first n_bins
// outputs.  For P >= 2 n_bins this is exactly the linear convolution
//   q[m] = sum_k h(m - k) p[k]
// (Ram-Lak by default: h(0) = 1/4, h(odd n) = -1/(pi n)^2, h(even n) = 0;
// Shepp-Logan and Hann below).
//
// Two real rows ride in one complex FFT (row A real, row B imaginary); since
// the filter spectrum H is real and even, the inverse transform returns
// (A * h) + i (B * h) with no unpacking.  The forward transform is radix-2
// decimation in frequency (natural order in, bit-reversed order out), the
// spectrum is multiplied in bit-reversed order, and the inverse is decimation
// in time (bit-reversed in, natural out), so no permutation pass is needed.
// Consecutive radix-2 stages run fused three at a time in registers (the
// same butterflies in the same order), so a 4096-point transform makes 4
// shared-memory passes each way instead of 12.  The whole padded row pair
// lives in shared memory (P * 8 bytes plus one pad slot per 16 elements).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pyhst {
namespace {

// tw[k] = exp(-2 pi i k / P) for k < P/2, rounded to float from float64; the
// second quarter is formed as -i times the first (exact), so that
// tw[k + P/4] = -i tw[k] holds bit for bit (the transform derives half of its
// twiddles that way).
__global__ void twiddle_kernel(int P, float2 *__restrict__ tw, double *__restrict__ costab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        double s, c;
        sincospi(2.0 * (double)k / (double)P, &s, &c);
        costab[k] = c;
        if (k < P / 2) {
            const int j = k % (P / 4);
            sincospi(2.0 * (double)j / (double)P, &s, &c);
            const float2 w = make_float2((float)c, (float)-s);
            tw[k] = k < P / 4 ? w : make_float2(w.y, -w.x);
        }
    }
}

// H[k] = sum_{n=-P/2}^{P/2-1} h(n) cos(2 pi k n / P) = 1/4 + 2 sum_{odd n < P/2} h(n) cos(...)
// stored at bit-reversed positions with the inverse-FFT factor 1/P folded in.
// Spatial kernels of the filters (tau = 1 bin), even in n:
//   Ram-Lak      h(0) = 1/4, h(odd n) = -1/(pi n)^2, h(even n != 0) = 0   (DTFT |w| / 2 pi)
//   Shepp-Logan  h(n) = -2 / (pi^2 (4 n^2 - 1))                           (DTFT |sin(w/2)| / pi)
//   Hann         h(n) = h_RL(n) / 2 + (h_RL(n - 1) + h_RL(n + 1)) / 4       (DTFT |w| / 2 pi x (1 + cos w) / 2)
__device__ __forceinline__ double ramlak_h(long long n) {
    if (n < 0) n = -n;
    if (n == 0) return 0.25;
    return (n & 1) ? -1.0 / (M_PI * M_PI * (double)n * (double)n) : 0.0;
}

__device__ __forceinline__ double filter_h(int filter, long long n) {
    switch (filter) {
        case PYHST_SHEPP_LOGAN: return -2.0 / (M_PI * M_PI * (4.0 * (double)n * (double)n - 1.0));
        case PYHST_HANN: return 0.5 * ramlak_h(n) + 0.25 * (ramlak_h(n - 1) + ramlak_h(n + 1));
        default: return ramlak_h(n);
    }
}

// H[k] = (h(0) + 2 sum_{n=1}^{P/2-1} h(n) cos(2 pi k n / P)) / P in float64:
// the DFT of the kernel truncated to |n| < P/2 (which is all the linear
// convolution of n_bins <= P/2 samples uses), with the 1/P of the inverse
// transform folded in; stored in bit-reversed order.
__global__ void spectrum_kernel(int P, int logP, int filter, const double *__restrict__ costab,
                                float *__restrict__ hrev) {
    const int k = blockIdx.x;   // frequency 0..P/2
    double acc = 0.0;
    const int step = filter == PYHST_RAMLAK ? 2 : 1;   // Ram-Lak: odd n only
    for (int n = 1 + step * threadIdx.x; n < P / 2; n += step * blockDim.x) {
        const long long m = ((long long)k * n) % P;
        acc += filter_h(filter, n) * costab[m];
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float H = (float)((filter_h(filter, 0) + 2.0 * red[0]) / (double)P);
        hrev[__brev(k) >> (32 - logP)] = H;
        if (k > 0 && k < P / 2) hrev[__brev(P - k) >> (32 - logP)] = H;
    }
}

// Raw value of sample idx as float (counts, or the pre-normalised sinogram).
template <int kKind>
__device__ __forceinline__ float load_raw(const void *data, int64_t idx) {
    if (kKind == PYHST_U16_RAW) return (float)static_cast<const uint16_t *>(data)[idx];
    if (kKind == PYHST_F32_RAW || kKind == PYHST_F32_SINO) return static_cast<const float *>(data)[idx];
    if (kKind == PYHST_F16_SINO) return __half2float(static_cast<const __half *>(data)[idx]);
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(data)[idx]);
}
// p = -ln((I - D) / (F - D)) for counts (0 where F - D <= 0, ratio clamped
// below at 1e-6); the value itself for sinogram kinds.
template <int kKind>
__device__ __forceinline__ float to_p(float v, float F, float D) {
    if (kKind == PYHST_U16_RAW || kKind == PYHST_F32_RAW) {
        const float den = F - D;
        if (!(den > 0.0f)) return 0.0f;
        const float r = fmaxf((v - D) / den, 1e-6f);
        return -logf(r);
    }
    return v;
}

// The transform's arithmetic is written with the rounding intrinsics
// (__fadd_rn, __fmul_rn, fmaf), which the compiler never contracts into
// other operations: the register-fused passes therefore give the bits of the
// pass-by-pass transform, where every stage's results went through shared
// memory.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -__fmul_rn(a.y, b.y)), fmaf(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// Shared-memory slot of element i: one pad slot per 16 elements, so the
// stride-16 accesses of the last pass spread over all banks.
__device__ __forceinline__ int slot(int i) { return i + (i >> 4); }

// NST consecutive radix-2 stages (top, top-1, ..., top-NST+1 for the
// decimation in frequency; lo, lo+1, ... for the decimation in time) fused in
// registers: the 2^NST elements base + k 2^lo (k < 2^NST) are closed under
// them.  Every butterfly and twiddle is the one the stage-by-stage radix-2
// transform uses, in the same order, so the result is the same bits with a
// quarter of the shared-memory passes.
// The NST stages on the registers of one group: v[k] holds element
// base + k 2^lo.
template <int NST, bool kDIF>
__device__ __forceinline__ void group_stages(float2 (&v)[1 << NST], const float2 *__restrict__ tw, int logP, int lo,
                                             int base) {
    constexpr int G = 1 << NST;
    const int stride = 1 << lo, b0 = base & (stride - 1);
#pragma unroll
    for (int t = 0; t < NST; ++t) {
        const int sl = kDIF ? NST - 1 - t : t;      // stage within the group
        const int s = lo + sl, hk = 1 << sl;
        // the butterfly of element base + k 2^lo at stage s takes twiddle
        // ((base + k 2^lo) mod 2^s) 2^(logP-1-s) = (b0 + (k mod 2^sl) 2^lo) 2^(logP-1-s):
        // 2^sl distinct entries.  The upper half of them lie P/4 further in
        // the table, and tw[k + P/4] = -i tw[k] exactly (both rounded from
        // float64 values of opposite signs), so those are formed, not loaded.
        float2 wt[G / 2];
#pragma unroll
        for (int m = 0; m < (hk + 1) / 2; ++m) wt[m] = tw[(b0 + m * stride) << (logP - 1 - s)];
#pragma unroll
        for (int m = (hk + 1) / 2; m < hk; ++m) wt[m] = make_float2(wt[m - hk / 2].y, -wt[m - hk / 2].x);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k & hk) continue;
            const float2 w = wt[k & (hk - 1)];
            const float2 u = v[k];
            if (kDIF) {
                const float2 b = v[k + hk];
                v[k] = make_float2(__fadd_rn(u.x, b.x), __fadd_rn(u.y, b.y));
                v[k + hk] = cmul(make_float2(__fsub_rn(u.x, b.x), __fsub_rn(u.y, b.y)), w);
            } else {
                const float2 t2 = cmul(v[k + hk], make_float2(w.x, -w.y));
                v[k] = make_float2(__fadd_rn(u.x, t2.x), __fadd_rn(u.y, t2.y));
                v[k + hk] = make_float2(__fsub_rn(u.x, t2.x), __fsub_rn(u.y, t2.y));
            }
        }
    }
}

template <int NST, bool kDIF>
__device__ __forceinline__ void fused_stages(float2 *z, const float2 *__restrict__ tw, int P, int logP, int lo) {
    constexpr int G = 1 << NST;
    const int top = lo + NST - 1, stride = 1 << lo, ngroups = P >> NST;
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const int base = (g & (stride - 1)) | ((g >> lo) << (top + 1));
        float2 v[G];
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = z[slot(base + k * stride)];
        group_stages<NST, kDIF>(v, tw, logP, lo, base);
#pragma unroll
        for (int k = 0; k < G; ++k) z[slot(base + k * stride)] = v[k];
    }
}

constexpr int kFuse = 3;   // radix-2 stages fused per shared-memory pass (8 elements per thread)

template <bool kDIF>
__device__ __forceinline__ void fused_pass(int nst, float2 *z, const float2 *__restrict__ tw, int P, int logP, int lo) {
    switch (nst) {
        case 3: fused_stages<3, kDIF>(z, tw, P, logP, lo); break;
        case 2: fused_stages<2, kDIF>(z, tw, P, logP, lo); break;
        default: fused_stages<1, kDIF>(z, tw, P, logP, lo); break;
    }
}

// One CTA filters rows 2*blockIdx.x and 2*blockIdx.x+1 of the chunk; row r is
// (slice z0 + r / n_angles, angle r % n_angles).
template <int kKind, bool kFused>
__global__ void __launch_bounds__(1024) filter_kernel(const void *__restrict__ data, int64_t slice_stride, int64_t angle_stride,
                              const float *__restrict__ flat, const float *__restrict__ dark, int z0,
                              int n_rows, int n_angles, int n_bins, int P, int logP,
                              const float2 *__restrict__ tw, const float *__restrict__ hrev,
                              float *__restrict__ q) {
    extern __shared__ float2 z[];
    const int rA = 2 * blockIdx.x, rB = rA + 1;
    const bool hasB = rB < n_rows;
    const int zA = z0 + rA / n_angles, aA = rA % n_angles;
    const int zB = z0 + rB / n_angles, aB = rB % n_angles;
    const int64_t baseA = (int64_t)zA * slice_stride + (int64_t)aA * angle_stride;
    const int64_t baseB = (int64_t)zB * slice_stride + (int64_t)aB * angle_stride;
    constexpr bool raw = (kKind == PYHST_U16_RAW || kKind == PYHST_F32_RAW);
    if (kFused) {
        // One 8-element group per thread (blockDim = P / 8).  The first
        // forward pass (stages logP-1 .. logP-3) works on the elements
        // tid + j P/8, which are the samples the thread loads; the last
        // inverse pass (logP-3 .. logP-1) on the same elements, which it
        // stores; and the last forward pass (2, 1, 0), the spectrum and the
        // first inverse pass (0, 1, 2) on eight consecutive elements.  So these
        // run in registers: six shared-memory passes in all, with the
        // butterflies of the pass-by-pass transform in the same order.
        const int S = P / 8, tid = threadIdx.x;
        float2 v[8];
        {
            // all samples of the thread (and their flat / dark values) are
            // loaded before any is used; P >= 2 n_bins, so j >= 4 is padding
            constexpr int kJ = 4;
            float IA[kJ], IB[kJ], FA[kJ], DA[kJ], FB[kJ], DB[kJ];
#pragma unroll
            for (int j = 0; j < kJ; ++j) {
                const int k = tid + j * S;
                IA[j] = IB[j] = FA[j] = DA[j] = FB[j] = DB[j] = 0.0f;
                if (k < n_bins) {
                    IA[j] = load_raw<kKind>(data, baseA + k);
                    if (raw) {
                        FA[j] = flat[(size_t)zA * n_bins + k];
                        DA[j] = dark[(size_t)zA * n_bins + k];
                    }
                    if (hasB) {
                        IB[j] = load_raw<kKind>(data, baseB + k);
                        if (raw) {
                            FB[j] = flat[(size_t)zB * n_bins + k];
                            DB[j] = dark[(size_t)zB * n_bins + k];
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = tid + j * S;
                float va = 0.0f, vb = 0.0f;
                if (j < kJ && k < n_bins) {
                    va = to_p<kKind>(IA[j], FA[j], DA[j]);
                    if (hasB) vb = to_p<kKind>(IB[j], FB[j], DB[j]);
                }
                v[j] = make_float2(va, vb);
            }
        }
        // forward: decimation in frequency
        group_stages<3, true>(v, tw, logP, logP - 3, tid);
#pragma unroll
        for (int j = 0; j < 8; ++j) z[slot(tid + j * S)] = v[j];
        __syncthreads();
        for (int top = logP - 4; top >= 3; top -= kFuse) {
            const int nst = min(kFuse, top - 2);
            fused_pass<true>(nst, z, tw, P, logP, top - nst + 1);
            __syncthreads();
        }
        {
            const int base = 8 * tid;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = z[slot(base + k)];
            group_stages<3, true>(v, tw, logP, 0, base);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float H = hrev[base + k];
                v[k] = make_float2(__fmul_rn(v[k].x, H), __fmul_rn(v[k].y, H));
            }
            // inverse: decimation in time with conjugate twiddles
            group_stages<3, false>(v, tw, logP, 0, base);
#pragma unroll
            for (int k = 0; k < 8; ++k) z[slot(base + k)] = v[k];
        }
        __syncthreads();
        for (int lo = 3; lo <= logP - 4; lo += kFuse) {
            fused_pass<false>(min(kFuse, logP - 3 - lo), z, tw, P, logP, lo);
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = z[slot(tid + j * S)];
        group_stages<3, false>(v, tw, logP, logP - 3, tid);
        float *qA = q + (size_t)rA * n_bins;
        float *qB = q + (size_t)rB * n_bins;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = tid + j * S;
            if (k < n_bins) {
                qA[k] = v[j].x;
                if (hasB) qB[k] = v[j].y;
            }
        }
        return;
    }
    // Other lengths: the pass-by-pass transform through shared memory.
    // The thread's first four samples (and their flat / dark values) are all
    // loaded before any is used; this covers [0, n_bins) whenever n_bins <=
    // 4 blockDim; the tail loop takes any remaining samples and the zero padding.
    constexpr int kJ = 4;
    float IA[kJ], IB[kJ], FA[kJ], DA[kJ], FB[kJ], DB[kJ];
#pragma unroll
    for (int j = 0; j < kJ; ++j) {
        const int k = threadIdx.x + j * blockDim.x;
        IA[j] = IB[j] = FA[j] = DA[j] = FB[j] = DB[j] = 0.0f;
        if (k < n_bins) {
            IA[j] = load_raw<kKind>(data, baseA + k);
            if (raw) {
                FA[j] = flat[(size_t)zA * n_bins + k];
                DA[j] = dark[(size_t)zA * n_bins + k];
            }
            if (hasB) {
                IB[j] = load_raw<kKind>(data, baseB + k);
                if (raw) {
                    FB[j] = flat[(size_t)zB * n_bins + k];
                    DB[j] = dark[(size_t)zB * n_bins + k];
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kJ; ++j) {
        const int k = threadIdx.x + j * blockDim.x;
        float va = 0.0f, vb = 0.0f;
        if (k < n_bins) {
            va = to_p<kKind>(IA[j], FA[j], DA[j]);
            if (hasB) vb = to_p<kKind>(IB[j], FB[j], DB[j]);
        }
        if (k < P) z[slot(k)] = make_float2(va, vb);
    }
    for (int k = threadIdx.x + kJ * blockDim.x; k < P; k += blockDim.x) {
        float va = 0.0f, vb = 0.0f;
        if (k < n_bins) {
            va = to_p<kKind>(load_raw<kKind>(data, baseA + k), raw ? flat[(size_t)zA * n_bins + k] : 0.0f,
                             raw ? dark[(size_t)zA * n_bins + k] : 0.0f);
            if (hasB)
                vb = to_p<kKind>(load_raw<kKind>(data, baseB + k), raw ? flat[(size_t)zB * n_bins + k] : 0.0f,
                                 raw ? dark[(size_t)zB * n_bins + k] : 0.0f);
        }
        z[slot(k)] = make_float2(va, vb);
    }
    __syncthreads();
    // forward: decimation in frequency, stages logP-1 .. 0 in passes of up to kFuse
    for (int top = logP - 1; top >= 0; top -= kFuse) {
        const int nst = min(kFuse, top + 1);
        fused_pass<true>(nst, z, tw, P, logP, top - nst + 1);
        __syncthreads();
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const float H = hrev[k];
        const float2 v = z[slot(k)];
        z[slot(k)] = make_float2(__fmul_rn(v.x, H), __fmul_rn(v.y, H));
    }
    __syncthreads();
    // inverse: decimation in time with conjugate twiddles, stages 0 .. logP-1
    for (int lo = 0; lo < logP; lo += kFuse) {
        fused_pass<false>(min(kFuse, logP - lo), z, tw, P, logP, lo);
        __syncthreads();
    }
    float *qA = q + (size_t)rA * n_bins;
    float *qB = q + (size_t)rB * n_bins;
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
        const float2 v = z[slot(k)];
        qA[k] = v.x;
        if (hasB) qB[k] = v.y;
    }
}

}  // namespace

size_t filter_table_bytes(int P) {
    return align_up(sizeof(float2) * (P / 2)) + align_up(sizeof(double) * P) + align_up(sizeof(float) * P);
}

int launch_filter_tables(int P, int filter, void *tables, cudaStream_t st) {
    Carver cv(tables, filter_table_bytes(P));
    float2 *tw = cv.take<float2>(P / 2);
    double *costab = cv.take<double>(P);
    float *hrev = cv.take<float>(P);
    int logP = 0;
    while ((1 << logP) < P) ++logP;
    twiddle_kernel<<<(P + 255) / 256, 256, 0, st>>>(P, tw, costab);
    int rc = cuda_status("twiddle kernel");
    if (rc) return rc;
    spectrum_kernel<<<P / 2 + 1, 256, 0, st>>>(P, logP, filter, costab, hrev);
    return cuda_status("filter spectrum kernel");
}

int launch_filter(int kind, const void *data, int64_t slice_stride, int64_t angle_stride, const float *flat,
                  const float *dark, int z0, int n_slices_chunk, int n_angles, int n_bins, int P,
                  const void *tables, float *q, cudaStream_t st) {
    Carver cv(const_cast<void *>(tables), filter_table_bytes(P));
    const float2 *tw = cv.take<float2>(P / 2);
    cv.take<double>(P);
    const float *hrev = cv.take<float>(P);
    int logP = 0;
    while ((1 << logP) < P) ++logP;
    const int n_rows = n_slices_chunk * n_angles;
    const int threads = std::min(1024, std::max(64, P / 8));   // one 8-element group per thread and pass
    const size_t smem = sizeof(float2) * (P + P / 16);   // one pad slot per 16 elements
    const int grid = (n_rows + 1) / 2;
    // register-fused passes when a thread holds exactly one 8-element group
    const bool fused = threads * 8 == P;
#define PYHST_FILTER_CASE(K)                                                                             \
    case K: {                                                                                            \
        auto kern = fused ? filter_kernel<K, true> : filter_kernel<K, false>;                            \
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        kern<<<grid, threads, smem, st>>>(data, slice_stride, angle_stride, flat, dark, z0, n_rows, n_angles, \
                                          n_bins, P, logP, tw, hrev, q);                                 \
        break;                                                                                           \
    }
    ProfScope prof(kProfFilter, st);
    switch (kind) {
        PYHST_FILTER_CASE(PYHST_U16_RAW)
        PYHST_FILTER_CASE(PYHST_F32_RAW)
        PYHST_FILTER_CASE(PYHST_F32_SINO)
        PYHST_FILTER_CASE(PYHST_F16_SINO)
        PYHST_FILTER_CASE(PYHST_BF16_SINO)
        default: return fail(PYHST_ERR_INVALID_ARG, "unknown input kind %d", kind);
    }
#undef PYHST_FILTER_CASE
    return cuda_status("filter kernel");
}

}  // namespace pyhst
