// Microbenchmarks of the on-chip rates that bound the hot-path kernels, the
// denominators of their rooflines: the shared-memory data pipe (the
// back-projector and the projector read their staged windows and bands
// through it; 128 bytes per clock and SM), the FP32 fma rate (128 lanes per
// clock and SM) and the MUFU rate of the XU pipe (16 per clock and SM; the
// Chambolle steps take a square root and a reciprocal per cell).
// Each kernel runs 4 CTAs of 256 threads on every SM; the caller times a
// launch on its stream and divides the bytes or operations it reports.
#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kMbThreads = 256;
constexpr int kMbCtasPerSm = 4;
constexpr int kMbEntries = 4096;                       // float2 entries: 32 KB of shared memory
constexpr int kMbLoads = kMbEntries / kMbThreads;      // loads per thread and iteration
constexpr int kMbChains = 8;                           // independent fma chains per thread
constexpr int kMbFmaUnroll = 8;                        // fmas per chain and iteration
constexpr int kMbMufuUnroll = 4;                       // steps per chain and iteration

// Each warp instruction reads 32 consecutive float2 (256 bytes: two
// wavefronts, no bank conflicts) at a constant offset from the thread's base.
// The loads are volatile in the PTX itself, so that the assembler neither
// hoists them out of the loop nor merges them (the buffer never changes), and
// four paired accumulators keep the adds off the critical path.
__global__ void __launch_bounds__(kMbThreads) smem_read_kernel(float *__restrict__ sink, int iters) {
    __shared__ __align__(16) float2 buf[kMbEntries];
    for (int e = threadIdx.x; e < kMbEntries; e += kMbThreads) buf[e] = make_float2((float)e, 1.0f);
    __syncthreads();
    const uint32_t base = smem_addr(&buf[threadIdx.x]);
    float2 acc[4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kMbLoads; ++k) {
            float2 v;
            asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];"
                         : "=f"(v.x), "=f"(v.y) : "r"(base + k * kMbThreads * 8));
            acc[k & 3] = add2(acc[k & 3], v);
        }
    }
    const float2 s = add2(add2(acc[0], acc[1]), add2(acc[2], acc[3]));
    sink[blockIdx.x * kMbThreads + threadIdx.x] = s.x + s.y;
}

// kMbChains independent chains x <- x * a + b per thread: scalar fmas
// (kPaired false) or paired f32x2 fmas over chain pairs (kPaired true).
template <bool kPaired>
__global__ void __launch_bounds__(kMbThreads) fma_kernel(float *__restrict__ sink, int iters, float a, float b) {
    float x[kMbChains];
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kMbFmaUnroll; ++r) {
            if constexpr (kPaired) {
#pragma unroll
                for (int k = 0; k < kMbChains; k += 2) {
                    const float2 y = fma2(make_float2(x[k], x[k + 1]), a2, b2);
                    x[k] = y.x;
                    x[k + 1] = y.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kMbChains; ++k) x[k] = fmaf(x[k], a, b);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) s += x[k];
    sink[blockIdx.x * kMbThreads + threadIdx.x] = s;
}

// kMbChains independent chains x <- sqrt(1 / x + 1) per thread (approximate
// reciprocal and square root: two MUFU operations and one add per step; the
// chains stay near the golden ratio).
__global__ void __launch_bounds__(kMbThreads) mufu_kernel(float *__restrict__ sink, int iters) {
    float x[kMbChains];
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) x[k] = 1.0f + 1e-3f * (float)threadIdx.x + (float)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kMbMufuUnroll; ++r)
#pragma unroll
            for (int k = 0; k < kMbChains; ++k) {
                float y;
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
                y += 1.0f;
                asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(y));
            }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) s += x[k];
    sink[blockIdx.x * kMbThreads + threadIdx.x] = s;
}

int mb_ctas(int *ctas) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cuda_status("device query");
    *ctas = sms * kMbCtasPerSm;
    return PYHST_OK;
}

}  // namespace
}  // namespace pyhst

extern "C" size_t pyhst_microbench_sink_floats(void) {
    int ctas = 0;
    if (pyhst::mb_ctas(&ctas)) return 0;
    return (size_t)ctas * pyhst::kMbThreads;
}

extern "C" int pyhst_microbench(int32_t kind, int32_t iters, float *sink, double *units, pyhst_stream_t stream) {
    using namespace pyhst;
    if (kind < 0 || kind > 3) return fail(PYHST_ERR_INVALID_ARG, "microbenchmark kind %d: need 0 to 3", kind);
    if (iters < 1) return fail(PYHST_ERR_INVALID_ARG, "iters must be >= 1");
    if (!sink || !units) return fail(PYHST_ERR_INVALID_ARG, "sink/units pointer is NULL");
    int ctas = 0;
    int rc = mb_ctas(&ctas);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double threads = (double)ctas * kMbThreads;
    if (kind == 0) {
        smem_read_kernel<<<ctas, kMbThreads, 0, st>>>(sink, iters);
        *units = threads * iters * kMbLoads * sizeof(float2);                 // bytes read from shared memory
    } else if (kind == 3) {
        mufu_kernel<<<ctas, kMbThreads, 0, st>>>(sink, iters);
        *units = threads * iters * kMbMufuUnroll * kMbChains * 2.0;          // MUFU operations
    } else {
        if (kind == 1)
            fma_kernel<false><<<ctas, kMbThreads, 0, st>>>(sink, iters, 0.999999f, 1e-6f);
        else
            fma_kernel<true><<<ctas, kMbThreads, 0, st>>>(sink, iters, 0.999999f, 1e-6f);
        *units = threads * iters * kMbFmaUnroll * kMbChains * 2.0;           // flops (an fma is two)
    }
    return cuda_status("microbenchmark kernel");
}
