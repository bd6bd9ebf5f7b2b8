// Overlapping-patch prior (Sec. 3.2.1): the image of the coefficients
// (Eq. 7), the gradient of Eq. 8 by the steps of Algorithm 1, and ISTA/FISTA
// with L1 shrinkage on the coefficients.
//
// Per gradient evaluation at coefficients W [N][n_atoms]:
//   gemm_tc_kernel   P = W D                          (N x m^2; tensor cores, split bf16)
//   image_kernel     x_j = P[core(j)][j - r], S_j = sum of covering patches,
//                    Nv_j = their number
//   (projector)      R = Pi^T (Pi x - y)  (or x - y for denoising)
//   paux_kernel      P'_{p,i} = rho (P_{p,i} - x_{r_p+i})
//                               + [core(r_p+i) = p] (R + rho (Nv x - S))_{r_p+i},
//                    and the penalty sum_p sum_i (x_{r_p+i} - P_{p,i})^2
//   gemm_tc_kernel   G = 2 P' D^T
// Energies and norms are float64 block partials summed in a fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace pyhst {
namespace {

constexpr int kPT = 256;            // threads of the element kernels
constexpr int kPBlocks = 296;       // fixed grid of the reductions (partials are summed in order)
constexpr int kPauxBlocks = 1184;   // fixed grid of the auxiliary-patch kernel (gathers: more warps in flight)
// partial sums: data term, penalty, L1 norm, dot products
constexpr int kOffData = 0, kOffPen = kPBlocks, kOffL1 = kOffPen + kPauxBlocks, kOffDot = kOffL1 + kPBlocks;
constexpr int kPartTotal = kOffDot + kPBlocks;

struct PDims {
    int ny, nx, m, stride, kr, kc, N, nc, mm;
};

int axis_count(int n, int m, int stride) { return (n - m + stride - 1) / stride + 1; }

__host__ __device__ __forceinline__ int axis_start(int k, int n, int m, int stride) {
    const int r = k * stride;
    return r > n - m ? n - m : r;
}

// Core patch of every coordinate along one axis: the nearest centre
// start + (m-1)/2, ties to the lower index (Eq. 6 on a product grid).  The
// starts increase strictly with k, so along the axis the nearest centre only
// moves forward: one pass, advancing while the next centre is strictly nearer.
void core_table(int n, int m, int stride, int K, std::vector<int> &core) {
    core.assign(n, 0);
    auto dist = [&](int i, int k) { return std::fabs((double)i - ((double)axis_start(k, n, m, stride) + 0.5 * (m - 1))); };
    int k = 0;
    for (int i = 0; i < n; ++i) {
        while (k + 1 < K && dist(i, k + 1) < dist(i, k)) ++k;
        core[i] = k;
    }
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kPT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = l < kPT / 32 ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// C [M][N] = alpha A [M][K] B [K][N] (row-major, float32 sums in k order).
// Both patch products use it: P = W D (M = patches, K = atoms, N = m^2) and
// G = 2 P' D^T (K = m^2, N = atoms).  The products are tall and skinny (N and
// K of tens to hundreds), so a CTA of 16 x 16 threads takes 128 rows and all
// of N at once when N <= 192 (16 * kTN columns), and A is read from HBM once.
// Thread (tr, tc) owns rows {4 tr .. 4 tr + 3} and {64 + 4 tr .. 64 + 4 tr + 3}
// and columns tc + 16 j (j < kTN), so its global stores are coalesced.  K runs
// in chunks of 16, double-buffered in shared memory by asynchronous 4-byte
// copies (any K, any alignment; out-of-range elements are zero-filled), the
// next chunk in flight while the current one is multiplied.  The A chunk is
// staged transposed (As[k][row]) with the row index XORed by 2k: the 16
// threads of a half-warp that copy one row (16 consecutive k) then hit 16
// different banks, and the float4 read of four rows becomes a read of a
// permuted group of four (the permutation depends on the parity of k only).
constexpr int kGM = 128, kGK = 16, kGThreads = 256, kGMaxTN = 12;

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// One k of the product: four rows from each half of the swizzled A chunk
// (kP: the in-group permutation of this k), kTN columns of B.
template <int kTN, int kP>
__device__ __forceinline__ void gemm_step(const float *__restrict__ a_row, const float *__restrict__ b_row, int tr,
                                          int tc, int sw, float (&acc)[8][kTN]) {
    const float4 a0 = *reinterpret_cast<const float4 *>(a_row + ((4 * tr) ^ sw));
    const float4 a1 = *reinterpret_cast<const float4 *>(a_row + ((64 + 4 * tr) ^ sw));
    const float x0[4] = {a0.x, a0.y, a0.z, a0.w}, x1[4] = {a1.x, a1.y, a1.z, a1.w};
    float av[8], bv[kTN];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        av[i] = x0[i ^ kP];
        av[4 + i] = x1[i ^ kP];
    }
#pragma unroll
    for (int j = 0; j < kTN; ++j) bv[j] = b_row[tc + 16 * j];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < kTN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
}

template <int kTN>
__global__ void __launch_bounds__(kGThreads, 2) gemm_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                            float *__restrict__ C, int M, int N, int K, float alpha) {
    constexpr int kBN = 16 * kTN;
    constexpr int kAV = kGM * kGK / kGThreads;             // A elements per thread per chunk (8)
    __shared__ __align__(16) float As[2][kGK][kGM];
    __shared__ __align__(16) float Bs[2][kGK][kBN];
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kBN;
    auto fetch = [&](int buf, int k0) {
#pragma unroll
        for (int v = 0; v < kAV; ++v) {
            const int e = tid + v * kGThreads, r = e >> 4, k = e & 15;   // a half-warp copies one row's 16 k
            const int gm = m0 + r, gk = k0 + k;
            const bool ok = gm < M && gk < K;
            cp_async4(&As[buf][k][r ^ (2 * k)], ok ? A + (size_t)gm * K + gk : A, ok);
        }
#pragma unroll
        for (int v = 0; v < kTN; ++v) {
            const int e = tid + v * kGThreads, kb = e / kBN, c = e - kb * kBN;
            const int gk = k0 + kb, gn = n0 + c;
            const bool ok = gk < K && gn < N;
            cp_async4(&Bs[buf][kb][c], ok ? B + (size_t)gk * N + gn : B, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float acc[8][kTN] = {};
    fetch(0, 0);
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += kGK, buf ^= 1) {
        if (k0 + kGK < K) {
            fetch(buf ^ 1, k0 + kGK);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < kGK; k += 2) {
            gemm_step<kTN, 0>(As[buf][k], Bs[buf][k], tr, tc, (2 * k) & ~3, acc);        // even k: rows in order
            gemm_step<kTN, 2>(As[buf][k + 1], Bs[buf][k + 1], tr, tc, (2 * k + 2) & ~3, acc);  // odd k: pairs swapped
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + (i < 4 ? 4 * tr + i : 64 + 4 * tr + i - 4);
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < kTN; ++j) {
            const int gn = n0 + tc + 16 * j;
            if (gn < N) C[(size_t)gm * N + gn] = alpha * acc[i][j];
        }
    }
}

template <int kTN>
void gemm_launch(const float *A, const float *B, float *C, int M, int N, int K, float alpha, cudaStream_t st) {
    gemm_kernel<kTN><<<dim3((M + kGM - 1) / kGM, (N + 16 * kTN - 1) / (16 * kTN)), kGThreads, 0, st>>>(A, B, C, M, N,
                                                                                                       K, alpha);
}

// Column tile: all of N in one tile up to 16 * kGMaxTN columns, else tiles of 128.
int gemm_tn(int N) { return N <= 16 * kGMaxTN ? (N + 15) / 16 : 8; }

void gemm_simt(const float *A, const float *B, float *C, int M, int N, int K, float alpha, cudaStream_t st) {
    switch (gemm_tn(N)) {
    case 1: gemm_launch<1>(A, B, C, M, N, K, alpha, st); break;
    case 2: gemm_launch<2>(A, B, C, M, N, K, alpha, st); break;
    case 3: gemm_launch<3>(A, B, C, M, N, K, alpha, st); break;
    case 4: gemm_launch<4>(A, B, C, M, N, K, alpha, st); break;
    case 5: gemm_launch<5>(A, B, C, M, N, K, alpha, st); break;
    case 6: gemm_launch<6>(A, B, C, M, N, K, alpha, st); break;
    case 7: gemm_launch<7>(A, B, C, M, N, K, alpha, st); break;
    case 8: gemm_launch<8>(A, B, C, M, N, K, alpha, st); break;
    case 9: gemm_launch<9>(A, B, C, M, N, K, alpha, st); break;
    case 10: gemm_launch<10>(A, B, C, M, N, K, alpha, st); break;
    case 11: gemm_launch<11>(A, B, C, M, N, K, alpha, st); break;
    default: gemm_launch<12>(A, B, C, M, N, K, alpha, st); break;
    }
}

// ---------------------------------------------------------------- tensor cores
// The same product on the tensor cores (tcgen05, bf16 operands, float32
// accumulation in tensor memory), accurate to float32 rounding: each operand
// is split exactly into three bf16 terms x = x1 + x2 + x3 (x1: the leading 8
// significant bits of x, x2 the next 8 of the remainder, x3 the rest, which
// has at most 8), and the six products x_i y_j with i + j <= 4 are
// accumulated (the dropped ones are below 2^-22 of a term, about 1e-7 of the
// result in practice).  For a padded N of 32 or 64 the B terms, stacked along
// N, go in as one
// operand: x1 [y1 y2 y3], x2 [y1 y2], x3 y1 are three MMAs of N = 3, 2 and 1
// times the padded N into three column blocks of the accumulator, added in the
// read-back (half the MMAs of one per product).  Persistent CTAs walk 128-row
// tiles of C: warp 0
// issues the MMAs; warps 1-8 read the accumulators back (two warps per
// tensor-memory lane quarter, alternate 32-column chunks), transpose each
// 32 x 32 block through shared memory and store C rows coalesced; warps 9-16
// stage A in chunks of 32 k (float32 loads issued three chunks ahead into
// registers, split, K-major 8 x 16-byte core matrices in a 4-stage ring).  B,
// with N and K padded to multiples of 16, is split and staged once per CTA.
// Two accumulators let the read-back of one tile overlap the MMAs of the
// next.  Every wait is bounded; a wait that gives up sets the device status.
constexpr int kTcKC = 32;                          // k per ring stage
constexpr int kTcStages = 4;
constexpr int kTcProd = 256;                       // staging threads (warps 9-16)
constexpr int kTcEpi = 256;                        // read-back threads (warps 1-8)
constexpr int kTcThreads = 32 + kTcEpi + kTcProd;
constexpr int kTcProd0 = 32 + kTcEpi;              // first staging thread
constexpr int kTcSplit = 128 * kTcKC * 2;          // bytes of one bf16 term of a stage
constexpr int kTcStage = 3 * kTcSplit;
constexpr int kTcEpiBytes = 8 * 32 * 33 * 4;       // a 32 x 33 transpose block per read-back warp
constexpr size_t kTcBMax = 64 * 1024;              // bytes of the staged B terms at most
constexpr size_t kTcMinSmem = 120 * 1024;          // one CTA per SM (its tensor memory is 512 columns)

// x = x1 + x2 + x3 exactly; each term's bf16 value is the high half of the word.
__device__ __forceinline__ void split3(float x, uint32_t &a, uint32_t &b, uint32_t &c) {
    a = __float_as_uint(x) & 0xFFFF0000u;
    const float r = x - __uint_as_float(a);
    b = __float_as_uint(r) & 0xFFFF0000u;
    c = __float_as_uint(r - __uint_as_float(b));
}

// high halves of two words -> one word of two bf16 (lo in the low half)
__device__ __forceinline__ uint32_t pack_hi(uint32_t lo, uint32_t hi) { return __byte_perm(lo, hi, 0x7632); }

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
gemm_tc_kernel(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int M, int N, int K,
               int NT, int Kp, float alpha, unsigned *__restrict__ status, uint32_t kTcWait) {
    extern __shared__ __align__(128) uint8_t tc_smem[];
    uint8_t *ring = tc_smem;                                   // kTcStages x 3 terms x [128 rows][32 k]
    float *epi = reinterpret_cast<float *>(tc_smem + kTcStages * kTcStage);   // 8 x [32][33]
    uint8_t *bs = tc_smem + kTcStages * kTcStage + kTcEpiBytes;              // 3 terms x [NT rows][Kp k]
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], acc_full[2], acc_empty[2], drain;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = (M + 127) / 128, nC = (Kp + kTcKC - 1) / kTcKC;
    const int n_my = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const bool stacked = NT == 32 || NT == 64;                  // B terms stacked along N (3 NT <= 256)
    const uint32_t acc_stride = (NT <= 128 && !stacked) ? 128u : 256u;
    const uint32_t b_term = (uint32_t)NT * Kp * 2;

    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 2 * acc_stride);
        if (lane == 0) {
            for (int s = 0; s < kTcStages; ++s) {
                tc::bar_init(&full[s], kTcProd);
                tc::bar_init(&empty[s], 1);
            }
            for (int b = 0; b < 2; ++b) {
                tc::bar_init(&acc_full[b], 1);
                tc::bar_init(&acc_empty[b], kTcEpi);
            }
            tc::bar_init(&drain, 1);
        }
    } else if (tid >= kTcProd0) {
        // B [K][N] -> three bf16 terms, N-major rows of Kp k: element (n, k) at
        // (n / 8) (16 Kp) + (k / 8) 128 + (n % 8) 16 + (k % 8) 2.  Consecutive
        // threads read consecutive n (coalesced), eight loads in flight each.
        constexpr int kU = 8;
        for (int e0 = tid - kTcProd0; e0 < NT * Kp; e0 += kU * kTcProd) {
            float x[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int e = e0 + u * kTcProd, k = e / NT, n = e - k * NT;
                x[u] = (e < NT * Kp && n < N && k < K) ? __ldg(B + (size_t)k * N + n) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int e = e0 + u * kTcProd, k = e / NT, n = e - k * NT;
                if (e >= NT * Kp) break;
                uint32_t t[3];
                split3(x[u], t[0], t[1], t[2]);
                const uint32_t off =
                    (uint32_t)(n >> 3) * (16u * Kp) + (uint32_t)(k >> 3) * 128u + (n & 7) * 16u + (k & 7) * 2u;
#pragma unroll
                for (int j = 0; j < 3; ++j) *reinterpret_cast<uint16_t *>(bs + j * b_term + off) = (uint16_t)(t[j] >> 16);
            }
        }
        tc::fence_async_smem();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tm = s_tmem;
    bool ok = true;

    if (warp == 0) {
        // ------------------------------------------------------------ MMA issue
        const uint32_t idesc = tc::idesc_bf16(128, NT);
        const uint32_t idesc_s[3] = {tc::idesc_bf16(128, 3 * NT), tc::idesc_bf16(128, 2 * NT), idesc};
        const uint32_t ring0 = tc::smem_u32(ring), b0 = tc::smem_u32(bs);
        constexpr int kA[6] = {0, 0, 1, 0, 1, 2}, kB[6] = {0, 1, 0, 2, 1, 0};
        int q = 0;
        for (int t = 0; t < n_my && ok; ++t) {
            const int b = t & 1;
            if (t >= 2) ok = __all_sync(0xffffffffu, tc::bar_wait(&acc_empty[b], (uint32_t)(((t >> 1) - 1) & 1), kTcWait));
            if (!ok) break;
            tc::fence_after();
            const uint32_t d = tm + (uint32_t)b * acc_stride;
            for (int c = 0; c < nC; ++c, ++q) {
                const int s = q % kTcStages;
                ok = __all_sync(0xffffffffu, tc::bar_wait(&full[s], (uint32_t)((q / kTcStages) & 1), kTcWait));
                if (!ok) break;
                tc::fence_after();
                if (lane == 0) {
                    for (int j = 0; j < kTcKC / 16; ++j) {
                        const int kk = c * (kTcKC / 16) + j;        // k step (16 k) within Kp
                        if (kk * 16 >= Kp) break;
                        if (stacked) {
                            // x_i against the stacked terms y_1 .. y_(3-i): columns [0, (3 - i) NT)
                            const uint64_t db = tc::sdesc(b0 + kk * 256, 128, 16 * Kp);
#pragma unroll
                            for (int i = 0; i < 3; ++i) {
                                const uint64_t da = tc::sdesc(ring0 + s * kTcStage + i * kTcSplit + j * 256, 128, 16 * kTcKC);
                                tc::mma_bf16(d, da, db, idesc_s[i], c > 0 || j > 0 || i > 0);
                            }
                        } else {
#pragma unroll
                            for (int p = 0; p < 6; ++p) {
                                const uint64_t da = tc::sdesc(ring0 + s * kTcStage + kA[p] * kTcSplit + j * 256, 128, 16 * kTcKC);
                                const uint64_t db = tc::sdesc(b0 + kB[p] * b_term + kk * 256, 128, 16 * Kp);
                                tc::mma_bf16(d, da, db, idesc, c > 0 || j > 0 || p > 0);
                            }
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) tc::mma_commit(&acc_full[b]);
            __syncwarp();
        }
        if (!ok && lane == 0) atomicOr(status, tc::kErrMmaTimeout);
        // every MMA issued has finished before the tensor memory is freed
        if (lane == 0) {
            tc::mma_commit(&drain);
            if (!tc::bar_wait(&drain, 0, kDefaultWaitLimit)) atomicOr(status, tc::kErrMmaTimeout);
        }
        __syncwarp();
    } else if (tid < kTcProd0) {
        // ------------------------------------------------------------ read-back
        const int qd = warp & 3, half = (warp - 1) >> 2;      // lane quarter; even or odd column chunks
        float(*tb)[33] = reinterpret_cast<float(*)[33]>(epi + (warp - 1) * 32 * 33);
        for (int t = 0; t < n_my; ++t) {
            const int b = t & 1;
            ok = __all_sync(0xffffffffu, tc::bar_wait(&acc_full[b], (uint32_t)((t >> 1) & 1), kTcWait));
            if (!ok) {
                if (lane == 0) atomicOr(status, tc::kErrMmaTimeout);
                break;
            }
            tc::fence_after();
            const int row0 = (blockIdx.x + t * gridDim.x) * 128 + 32 * qd;   // this warp's 32 rows
            for (int j = half; j * 32 < NT; j += 2) {
                float v[32];
                const uint32_t ta = tm + ((uint32_t)(32 * qd) << 16) + (uint32_t)b * acc_stride + 32u * j;
                tc::tmem_ld32(ta, v);
                if (stacked) {                                    // + x_i y_2 block + x_1 y_3 block
                    float w[32];
                    tc::tmem_ld32(ta + (uint32_t)NT, w);
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] += w[k];
                    tc::tmem_ld32(ta + 2u * NT, w);
#pragma unroll
                    for (int k = 0; k < 32; ++k) v[k] += w[k];
                }
#pragma unroll
                for (int k = 0; k < 32; ++k) tb[lane][k] = v[k];       // lane = row
                __syncwarp();
                const int col = 32 * j + lane;
#pragma unroll 4
                for (int r = 0; r < 32; ++r)                            // lane = column
                    if (row0 + r < M && col < N) C[(size_t)(row0 + r) * N + col] = alpha * tb[r][lane];
                __syncwarp();
            }
            tc::fence_before();
            bar_arrive(&acc_empty[b]);
        }
    } else {
        // ------------------------------------------------------------ staging
        const int pw = (tid - kTcProd0) >> 5, r8 = lane & 7, kq = lane >> 3;
        const bool vec = (K & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
        const int total = n_my * nC;
        // chunk q: tile q / nC of this CTA, k chunk q % nC.  Unit u of a chunk:
        // 8 rows x 16 k; lane (r8, kq) holds row r8, k 4 kq .. 4 kq + 3.
        auto fetch = [&](int q, float4 (&x)[4]) {
            const int t = q / nC, c = q - t * nC;
            const int m0 = (blockIdx.x + t * gridDim.x) * 128;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int unit = 4 * pw + u, rg = unit >> 1, kg = unit & 1;
                const int row = m0 + 8 * rg + r8, k = c * kTcKC + 16 * kg + 4 * kq;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < M) {
                    const float *src = A + (size_t)row * K + k;
                    if (vec) {
                        if (k < K) v = __ldg(reinterpret_cast<const float4 *>(src));   // K % 4 == 0
                    } else {
                        if (k < K) v.x = __ldg(src);
                        if (k + 1 < K) v.y = __ldg(src + 1);
                        if (k + 2 < K) v.z = __ldg(src + 2);
                        if (k + 3 < K) v.w = __ldg(src + 3);
                    }
                }
                x[u] = v;
            }
        };
        float4 xa[4], xb[4], xc[4], xd[4];
        if (total > 0) fetch(0, xa);
        if (total > 1) fetch(1, xb);
        if (total > 2) fetch(2, xc);
        for (int q = 0; q < total; ++q) {
            if (q + 3 < total) fetch(q + 3, xd);           // three chunks ahead
            const int s = q % kTcStages;
            if (q >= kTcStages) {
                ok = __all_sync(0xffffffffu, tc::bar_wait(&empty[s], (uint32_t)(((q / kTcStages) - 1) & 1), kTcWait));
                if (!ok) {
                    if (lane == 0) atomicOr(status, tc::kErrMmaTimeout);
                    break;
                }
                tc::fence_after();
            }
            uint8_t *st = ring + s * kTcStage;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int unit = 4 * pw + u, rg = unit >> 1, kg = unit & 1;
                uint32_t h[3][4];
                split3(xa[u].x, h[0][0], h[1][0], h[2][0]);
                split3(xa[u].y, h[0][1], h[1][1], h[2][1]);
                split3(xa[u].z, h[0][2], h[1][2], h[2][2]);
                split3(xa[u].w, h[0][3], h[1][3], h[2][3]);
                const uint32_t off = rg * 512u + (uint32_t)(2 * kg + (kq >> 1)) * 128u + r8 * 16u + (kq & 1) * 8u;
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    *reinterpret_cast<uint2 *>(st + j * kTcSplit + off) =
                        make_uint2(pack_hi(h[j][0], h[j][1]), pack_hi(h[j][2], h[j][3]));
            }
            tc::fence_async_smem();
            bar_arrive(&full[s]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xa[u] = xb[u];
                xb[u] = xc[u];
                xc[u] = xd[u];
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tm, 2 * acc_stride);
    }
}

int g_sm_count = 0;

bool gemm_tc_fits(int N, int K) {
    const int NT = (N + 15) & ~15, Kp = (K + 15) & ~15;
    return N >= 1 && K >= 1 && NT <= 256 && (size_t)3 * NT * Kp * 2 <= kTcBMax;
}

void gemm_tc(const float *A, const float *B, float *C, int M, int N, int K, float alpha, cudaStream_t st) {
    const int NT = (N + 15) & ~15, Kp = (K + 15) & ~15;
    const size_t smem =
        std::max(kTcMinSmem, (size_t)kTcStages * kTcStage + (size_t)kTcEpiBytes + (size_t)3 * NT * Kp * 2);
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
        cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kTcStages * kTcStage + kTcEpiBytes + kTcBMax));
    }
    const int tiles = (M + 127) / 128;
    gemm_tc_kernel<<<std::min(tiles, g_sm_count), kTcThreads, smem, st>>>(A, B, C, M, N, K, NT, Kp, alpha,
                                                                         device_status_ptr(),
                                                                         pipeline_wait_limit());
}

// Shapes whose padded B fits the tensor-core kernel take it; the rest (more
// than 256 columns, very long k) take the SIMT kernel.
void gemm(const float *A, const float *B, float *C, int M, int N, int K, float alpha, cudaStream_t st) {
    if (M <= 0) return;
    if (gemm_tc_fits(N, K))
        gemm_tc(A, B, C, M, N, K, alpha, st);
    else
        gemm_simt(A, B, C, M, N, K, alpha, st);
}

// Eq. 7 and the patch sums: one thread per pixel.
__global__ void image_kernel(const float *__restrict__ P, const int *__restrict__ core_r,
                             const int *__restrict__ core_c, PDims d, float *__restrict__ X, float *__restrict__ S,
                             float *__restrict__ Nv) {
    const int j = blockIdx.x * kPT + threadIdx.x;
    if (j >= d.ny * d.nx) return;
    const int i = j / d.nx, c = j % d.nx;
    {
        const int a = core_r[i], b = core_c[c];
        const int ri = axis_start(a, d.ny, d.m, d.stride), rc = axis_start(b, d.nx, d.m, d.stride);
        X[j] = P[((size_t)a * d.kc + b) * d.mm + (i - ri) * d.m + (c - rc)];
    }
    float s = 0.0f;
    int nv = 0;
    const int a0 = max(0, (i - d.m + 1 + d.stride - 1) / d.stride - 1);
    const int b0 = max(0, (c - d.m + 1 + d.stride - 1) / d.stride - 1);
    for (int a = a0; a < d.kr; ++a) {
        const int ri = axis_start(a, d.ny, d.m, d.stride);
        if (ri > i) break;
        if (i >= ri + d.m) continue;
        for (int b = b0; b < d.kc; ++b) {
            const int rc = axis_start(b, d.nx, d.m, d.stride);
            if (rc > c) break;
            if (c >= rc + d.m) continue;
            s += P[((size_t)a * d.kc + b) * d.mm + (i - ri) * d.m + (c - rc)];
            ++nv;
        }
    }
    S[j] = s;
    Nv[j] = (float)nv;
}

// r = a - b (float32) and the float64 partial of sum r^2.
__global__ void diff_kernel(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ r, size_t n,
                            double *__restrict__ part) {
    RunSum rs;
    for (size_t k = (size_t)blockIdx.x * kPT + threadIdx.x; k < n; k += (size_t)gridDim.x * kPT) {
        const float v = a[k] - (b ? b[k] : 0.0f);
        if (r) r[k] = v;
        rs.add(v * v);
    }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// The auxiliary patches P' of Algorithm 1 and the penalty partials.  A
// block takes 256 / m^2 patches at a time (thread: one pixel of one patch).
__global__ void paux_kernel(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ R,
                            const float *__restrict__ S, const float *__restrict__ Nv, const int *__restrict__ core_r,
                            const int *__restrict__ core_c, PDims d, float rho, float *__restrict__ Pp,
                            double *__restrict__ part) {
    // penalty: each thread's squared differences in float32 over runs of 8
    // (relative error ~5e-7 per run), the runs and the block in float64 (FP64
    // throughput is scarce: one float64 add per 8 elements)
    double acc = 0.0;
    float run = 0.0f;
    int n_run = 0;
    const int ppb = kPT / d.mm;                       // patches per pass of a block (m <= 16)
    const int i = threadIdx.x % d.mm, sub = threadIdx.x / d.mm;
    const int di = i / d.m, dj = i % d.m;
    const float inv_kc = 1.0f / (float)d.kc;
    for (int p = blockIdx.x * ppb + sub; sub < ppb && p < d.N; p += gridDim.x * ppb) {
        const size_t o = (size_t)p * d.mm + i;
        // a = p / kc, b = p % kc; for p < 2^24 the float quotient is off by at
        // most one and is corrected, larger grids divide exactly
        int a;
        if (d.N < (1 << 24)) {
            a = (int)((float)p * inv_kc);
            if (a * d.kc > p) --a;
            else if ((a + 1) * d.kc <= p) ++a;
        } else {
            a = p / d.kc;
        }
        const int b = p - a * d.kc;
        const int rr = axis_start(a, d.ny, d.m, d.stride) + di;
        const int cc = axis_start(b, d.nx, d.m, d.stride) + dj;
        const size_t j = (size_t)rr * d.nx + cc;
        const float x = X[j], pv = P[o];
        float v = rho * (pv - x);
        if (Pp) {
            if (core_r[rr] == a && core_c[cc] == b) v += R[j] + rho * (Nv[j] * x - S[j]);
            Pp[o] = v;
        }
        const float e = x - pv;
        run = fmaf(e, e, run);
        if (++n_run == 8) {
            acc += (double)run;
            run = 0.0f;
            n_run = 0;
        }
    }
    acc += (double)run;
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void transpose_kernel(const float *__restrict__ D, float *__restrict__ Dt, int nc, int mm) {
    const int o = blockIdx.x * kPT + threadIdx.x;
    if (o >= nc * mm) return;
    const int t = o / mm, i = o % mm;
    Dt[(size_t)i * nc + t] = D[o];
}

// Scalars of a solve (device): L, and its float32 step and threshold.
struct PScal {
    double *L;       // [1]
    float *invL;     // [1]
    float *thr;      // [1] beta / L
    double *acc;     // [4] scratch sums
};

// sum of part[0..n) (fixed order) into *out (scaled)
__global__ void finalize_kernel(const double *__restrict__ part, int n, double scale, double *__restrict__ out) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += kPT) acc += part[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc * scale;
}

// f = data + rho pen (+ beta l1 when with_l1) into *out; part holds the
// partials at kOffData, kOffPen, kOffL1
__global__ void energy_kernel(const double *__restrict__ part, bool with_l1, double rho, double beta,
                              double *__restrict__ out) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < kPBlocks; k += kPT) {
        a += part[kOffData + k];
        if (with_l1) c += part[kOffL1 + k];
    }
    for (int k = threadIdx.x; k < kPauxBlocks; k += kPT) b += part[kOffPen + k];
    a = block_sum(a);
    b = block_sum(b);
    c = block_sum(c);
    if (threadIdx.x == 0) *out = a + rho * b + beta * c;
}

// W = soft(Y - G / L, beta / L); Y = W + w (W - Wold); Wold = W; L1 partials of W.
__global__ void fista_update_kernel(float *__restrict__ W, float *__restrict__ Y, float *__restrict__ Wold,
                                    const float *__restrict__ G, size_t n, PScal sc, float w,
                                    double *__restrict__ part) {
    const float invL = *sc.invL, thr = *sc.thr;
    RunSum rs;
    for (size_t k = (size_t)blockIdx.x * kPT + threadIdx.x; k < n; k += (size_t)gridDim.x * kPT) {
        const float v = Y[k] - G[k] * invL;
        const float a = fabsf(v) - thr;
        const float wn = a > 0.0f ? copysignf(a, v) : 0.0f;
        W[k] = wn;
        Y[k] = wn + w * (wn - Wold[k]);
        Wold[k] = wn;
        rs.add(fabsf(wn));
    }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// power iteration: v = h / ||h||, with ||h||^2 in *nrm (float64)
__global__ void pnorm_kernel(const float *__restrict__ h, float *__restrict__ v, size_t n, const double *__restrict__ nrm2) {
    const double s = 1.0 / sqrt(*nrm2);
    for (size_t k = (size_t)blockIdx.x * kPT + threadIdx.x; k < n; k += (size_t)gridDim.x * kPT)
        v[k] = (float)((double)h[k] * s);
}

__global__ void dot_kernel(const float *__restrict__ a, const float *__restrict__ b, size_t n, double *__restrict__ part) {
    RunSum rs;
    for (size_t k = (size_t)blockIdx.x * kPT + threadIdx.x; k < n; k += (size_t)gridDim.x * kPT) rs.add(a[k] * b[k]);
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void set_step_kernel(const double *__restrict__ rq, double given, float beta, PScal sc) {
    const double L = given > 0.0 ? given : 1.01 * *rq;
    *sc.L = L;
    *sc.invL = (float)(1.0 / L);
    *sc.thr = (float)((double)beta / L);
}

__global__ void fill_f(float *__restrict__ v, float val, size_t n) {
    for (size_t k = (size_t)blockIdx.x * kPT + threadIdx.x; k < n; k += (size_t)gridDim.x * kPT) v[k] = val;
}

struct PLayout {
    size_t core_r, core_c, P, Pp, X, R, S, Nv, Dt, sdata, tab, xt, zero, Y, Wold, G, V, part, scal, bytes;
};

struct PCtx {
    PDims d;
    const pyhst_patch_problem *pp;
    const pyhst_geometry *g;
    int *core_r, *core_c;
    float *P, *Pp, *X, *R, *S, *Nv, *Dt, *sdata, *xt, *zero, *Y, *Wold, *G, *V;
    AngleInfo *tab;
    double *part;      // [kPartTotal]
    PScal sc;
    size_t M;          // data size
};

bool make_dims(const pyhst_patch_problem *pp, PDims &d) {
    if (!pp || pp->ny < 1 || pp->nx < 1 || pp->m < 1 || pp->m > 16 || pp->stride < 1 || pp->stride > pp->m ||
        pp->m > pp->ny || pp->m > pp->nx || pp->n_atoms < 1 || (int64_t)pp->n_atoms * pp->m * pp->m > 65536)
        return false;
    d.ny = pp->ny;
    d.nx = pp->nx;
    d.m = pp->m;
    d.stride = pp->stride;
    d.kr = axis_count(pp->ny, pp->m, pp->stride);
    d.kc = axis_count(pp->nx, pp->m, pp->stride);
    d.N = d.kr * d.kc;
    d.nc = pp->n_atoms;
    d.mm = pp->m * pp->m;
    return true;
}

PLayout playout(const PDims &d, const pyhst_geometry *g) {
    PLayout l{};
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    const size_t img = sizeof(float) * (size_t)d.ny * d.nx;
    const size_t M = g ? (size_t)g->n_angles * g->n_bins : (size_t)d.ny * d.nx;
    l.core_r = take(sizeof(int) * d.ny);
    l.core_c = take(sizeof(int) * d.nx);
    l.P = take(sizeof(float) * (size_t)d.N * d.mm);
    l.Pp = take(sizeof(float) * (size_t)d.N * d.mm);
    l.X = take(img);
    l.R = take(img);
    l.S = take(img);
    l.Nv = take(img);
    l.Dt = take(sizeof(float) * (size_t)d.nc * d.mm);
    l.sdata = take(sizeof(float) * M);
    l.zero = take(sizeof(float) * M);
    if (g) {
        pyhst_geometry g1 = *g;
        g1.n_slices = 1;
        l.tab = take(angle_table_bytes(g->n_angles));
        l.xt = take(project_scratch_bytes(&g1));
    }
    const size_t coef = sizeof(float) * (size_t)d.N * d.nc;
    l.Y = take(coef);
    l.Wold = take(coef);
    l.G = take(coef);
    l.V = take(coef);
    l.part = take(sizeof(double) * kPartTotal);
    l.scal = take(64);
    l.bytes = off;
    return l;
}

int prepare(const pyhst_patch_problem *pp, const pyhst_geometry *g, void *ws, cudaStream_t st, PCtx &c) {
    if (!make_dims(pp, c.d)) return fail(PYHST_ERR_INVALID_ARG, "patch problem sizes out of range");
    const PLayout l = playout(c.d, g);
    char *b = static_cast<char *>(ws);
    c.pp = pp;
    c.g = g;
    c.core_r = reinterpret_cast<int *>(b + l.core_r);
    c.core_c = reinterpret_cast<int *>(b + l.core_c);
    c.P = reinterpret_cast<float *>(b + l.P);
    c.Pp = reinterpret_cast<float *>(b + l.Pp);
    c.X = reinterpret_cast<float *>(b + l.X);
    c.R = reinterpret_cast<float *>(b + l.R);
    c.S = reinterpret_cast<float *>(b + l.S);
    c.Nv = reinterpret_cast<float *>(b + l.Nv);
    c.Dt = reinterpret_cast<float *>(b + l.Dt);
    c.sdata = reinterpret_cast<float *>(b + l.sdata);
    c.zero = reinterpret_cast<float *>(b + l.zero);
    c.tab = g ? reinterpret_cast<AngleInfo *>(b + l.tab) : nullptr;
    c.xt = g ? reinterpret_cast<float *>(b + l.xt) : nullptr;
    c.Y = reinterpret_cast<float *>(b + l.Y);
    c.Wold = reinterpret_cast<float *>(b + l.Wold);
    c.G = reinterpret_cast<float *>(b + l.G);
    c.V = reinterpret_cast<float *>(b + l.V);
    c.part = reinterpret_cast<double *>(b + l.part);
    double *sc = reinterpret_cast<double *>(b + l.scal);
    c.sc.L = sc;
    c.sc.acc = sc + 1;
    c.sc.invL = reinterpret_cast<float *>(sc + 5);
    c.sc.thr = c.sc.invL + 1;
    c.M = g ? (size_t)g->n_angles * g->n_bins : (size_t)c.d.ny * c.d.nx;
    std::vector<int> cr, cc;
    core_table(c.d.ny, c.d.m, c.d.stride, c.d.kr, cr);
    core_table(c.d.nx, c.d.m, c.d.stride, c.d.kc, cc);
    cudaMemcpyAsync(c.core_r, cr.data(), sizeof(int) * cr.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c.core_c, cc.data(), sizeof(int) * cc.size(), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);   // the host tables are local
    cudaMemsetAsync(c.zero, 0, sizeof(float) * c.M, st);
    transpose_kernel<<<(c.d.nc * c.d.mm + kPT - 1) / kPT, kPT, 0, st>>>(pp->dict, c.Dt, c.d.nc, c.d.mm);
    int rc = cuda_status("patch set-up");
    if (rc) return rc;
    if (g && (rc = launch_angle_table(g->angles, g->axis, g->n_angles, c.tab, st))) return rc;
    return PYHST_OK;
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + kPT - 1) / kPT, 1u << 30); }

// P = W D and the image (Eq. 7), patch sums and cover counts.
int synth_image(PCtx &c, const float *W, cudaStream_t st) {
    gemm(W, c.pp->dict, c.P, c.d.N, c.d.mm, c.d.nc, 1.0f, st);
    image_kernel<<<blocks_for((size_t)c.d.ny * c.d.nx), kPT, 0, st>>>(c.P, c.core_r, c.core_c, c.d, c.X, c.S, c.Nv);
    return cuda_status("patch synthesis");
}

// Evaluate at W: image, residual R, penalty; with G != NULL also the
// gradient.  Partials: part[0] data, part[1] penalty.
int evaluate(PCtx &c, const float *W, const float *y, float *G, cudaStream_t st) {
    int rc = synth_image(c, W, st);
    if (rc) return rc;
    if (c.g) {
        pyhst_geometry g1 = *c.g;
        g1.n_slices = 1;
        if ((rc = launch_project(&g1, c.tab, c.X, c.sdata, c.g->pixel_size, c.xt, st))) return rc;
        diff_kernel<<<kPBlocks, kPT, 0, st>>>(c.sdata, y, nullptr, c.M, c.part);
        if (G && (rc = launch_backproject(&g1, c.tab, BpSource{c.sdata, y}, c.R, c.g->pixel_size, st))) return rc;
    } else {
        diff_kernel<<<kPBlocks, kPT, 0, st>>>(c.X, y, c.R, c.M, c.part);
    }
    paux_kernel<<<kPauxBlocks, kPT, 0, st>>>(c.P, c.X, c.R, c.S, c.Nv, c.core_r, c.core_c, c.d, c.pp->rho,
                                            G ? c.Pp : nullptr, c.part + kOffPen);
    if (G) gemm(c.Pp, c.Dt, G, c.d.N, c.d.nc, c.d.mm, 2.0f, st);
    return cuda_status("patch gradient");
}

int check_common(const pyhst_patch_problem *pp, const pyhst_geometry *g, void *ws, size_t ws_bytes) {
    PDims d;
    if (!pp || !make_dims(pp, d))
        return fail(PYHST_ERR_INVALID_ARG, "patch problem: need 1 <= stride <= m <= min(16, ny, nx), "
                                           "n_atoms >= 1, n_atoms m^2 <= 65536");
    if (!pp->dict) return fail(PYHST_ERR_INVALID_ARG, "dictionary pointer is NULL");
    if (!(pp->rho >= 0.0f) || !std::isfinite(pp->rho)) return fail(PYHST_ERR_INVALID_ARG, "rho must be >= 0");
    if (g) {
        pyhst_geometry g1 = *g;
        g1.n_slices = 1;
        int rc = check_geometry(&g1);
        if (rc) return rc;
        if (g->nx != pp->nx || g->ny != pp->ny) return fail(PYHST_ERR_INVALID_ARG, "geometry image size differs");
    }
    const size_t need = playout(d, g).bytes;
    if (!ws || ws_bytes < need || ((uintptr_t)ws % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    return PYHST_OK;
}

}  // namespace
}  // namespace pyhst

using namespace pyhst;

extern "C" int pyhst_patch_grid(int32_t ny, int32_t nx, int32_t m, int32_t stride, int32_t *k_rows, int32_t *k_cols) {
    if (!k_rows || !k_cols) return fail(PYHST_ERR_INVALID_ARG, "output pointers are NULL");
    if (m < 1 || stride < 1 || stride > m || m > ny || m > nx)
        return fail(PYHST_ERR_INVALID_ARG, "need 1 <= stride <= m <= min(ny, nx)");
    *k_rows = axis_count(ny, m, stride);
    *k_cols = axis_count(nx, m, stride);
    return PYHST_OK;
}

extern "C" size_t pyhst_patch_workspace_size(const pyhst_patch_problem *pp, const pyhst_geometry *g) {
    PDims d;
    if (!pp || !make_dims(pp, d)) return 0;
    return playout(d, g).bytes;
}

extern "C" int pyhst_patch_image(const pyhst_patch_problem *pp, const float *W, float *x, void *workspace,
                                 size_t ws_bytes, pyhst_stream_t stream) {
    int rc = check_common(pp, nullptr, workspace, ws_bytes);
    if (rc) return rc;
    if (!W || !x) return fail(PYHST_ERR_INVALID_ARG, "W/x pointer is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PCtx c;
    if ((rc = prepare(pp, nullptr, workspace, st, c))) return rc;
    if ((rc = synth_image(c, W, st))) return rc;
    cudaMemcpyAsync(x, c.X, sizeof(float) * (size_t)c.d.ny * c.d.nx, cudaMemcpyDeviceToDevice, st);
    return cuda_status("patch image copy");
}

extern "C" int pyhst_patch_gradient(const pyhst_patch_problem *pp, const pyhst_geometry *g, const float *W,
                                    const float *y, float *G, double *f_out, void *workspace, size_t ws_bytes,
                                    pyhst_stream_t stream) {
    int rc = check_common(pp, g, workspace, ws_bytes);
    if (rc) return rc;
    if (!W || !y || !G) return fail(PYHST_ERR_INVALID_ARG, "W/y/G pointer is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PCtx c;
    if ((rc = prepare(pp, g, workspace, st, c))) return rc;
    if ((rc = evaluate(c, W, y, G, st))) return rc;
    if (f_out) energy_kernel<<<1, kPT, 0, st>>>(c.part, false, pp->rho, 0.0, f_out);
    return cuda_status("patch energy");
}

extern "C" int pyhst_patch_solve(const pyhst_patch_problem *pp, const pyhst_geometry *g, const float *y, float beta,
                                 double lipschitz, int32_t n_power_iter, int32_t n_iter, int32_t use_fista, float *W,
                                 float *x, double *energy, double *lipschitz_out, void *workspace, size_t ws_bytes,
                                 pyhst_stream_t stream) {
    int rc = check_common(pp, g, workspace, ws_bytes);
    if (rc) return rc;
    if (!W || !y) return fail(PYHST_ERR_INVALID_ARG, "W/y pointer is NULL");
    if (!(beta >= 0.0f) || !std::isfinite(beta)) return fail(PYHST_ERR_INVALID_ARG, "beta must be >= 0");
    if (n_iter < 1) return fail(PYHST_ERR_INVALID_ARG, "n_iter must be >= 1");
    if (!(lipschitz >= 0.0) || !std::isfinite(lipschitz))
        return fail(PYHST_ERR_INVALID_ARG, "lipschitz must be >= 0 (0: estimate)");
    if (lipschitz == 0.0 && n_power_iter < 1)
        return fail(PYHST_ERR_INVALID_ARG, "n_power_iter must be >= 1 when lipschitz is estimated");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PCtx c;
    if ((rc = prepare(pp, g, workspace, st, c))) return rc;
    const size_t nw = (size_t)c.d.N * c.d.nc;

    // ---- step size: the Hessian of f is constant; H v = grad f(v) at y = 0
    if (lipschitz == 0.0) {
        fill_f<<<kPBlocks, kPT, 0, st>>>(c.V, 1.0f, nw);
        for (int it = 0; it < n_power_iter; ++it) {
            if ((rc = evaluate(c, c.V, c.zero, c.G, st))) return rc;
            dot_kernel<<<kPBlocks, kPT, 0, st>>>(c.G, c.G, nw, c.part + kOffDot);
            finalize_kernel<<<1, kPT, 0, st>>>(c.part + kOffDot, kPBlocks, 1.0, c.sc.acc);
            pnorm_kernel<<<kPBlocks, kPT, 0, st>>>(c.G, c.V, nw, c.sc.acc);
        }
        // Rayleigh quotient <v, H v> with ||v|| = 1
        if ((rc = evaluate(c, c.V, c.zero, c.G, st))) return rc;
        dot_kernel<<<kPBlocks, kPT, 0, st>>>(c.V, c.G, nw, c.part + kOffDot);
        finalize_kernel<<<1, kPT, 0, st>>>(c.part + kOffDot, kPBlocks, 1.0, c.sc.acc + 1);
    }
    set_step_kernel<<<1, 1, 0, st>>>(c.sc.acc + 1, lipschitz, beta, c.sc);
    if (lipschitz_out) cudaMemcpyAsync(lipschitz_out, c.sc.L, sizeof(double), cudaMemcpyDeviceToDevice, st);
    if ((rc = cuda_status("patch step size"))) return rc;

    // ---- ISTA / FISTA: Y = Wold = W
    cudaMemcpyAsync(c.Y, W, sizeof(float) * nw, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c.Wold, W, sizeof(float) * nw, cudaMemcpyDeviceToDevice, st);
    double t = 1.0;
    for (int k = 0; k < n_iter; ++k) {
        if ((rc = evaluate(c, c.Y, y, c.G, st))) return rc;
        double w = 0.0;
        if (use_fista) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            w = (t - 1.0) / tn;
            t = tn;
        }
        fista_update_kernel<<<kPBlocks, kPT, 0, st>>>(W, c.Y, c.Wold, c.G, nw, c.sc, (float)w, c.part + kOffL1);
        if ((rc = cuda_status("patch update"))) return rc;
        if (energy) {
            if ((rc = evaluate(c, W, y, nullptr, st))) return rc;
            energy_kernel<<<1, kPT, 0, st>>>(c.part, true, pp->rho, (double)beta, energy + k);
        }
    }
    if (x) {
        if ((rc = synth_image(c, W, st))) return rc;
        cudaMemcpyAsync(x, c.X, sizeof(float) * (size_t)c.d.ny * c.d.nx, cudaMemcpyDeviceToDevice, st);
    }
    return cuda_status("patch solve");
}
