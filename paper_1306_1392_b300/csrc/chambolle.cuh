// Fused Chambolle steps for the TV prox (Eq. 2; Chambolle's dual fixed point):
//   G = div p - z / lam,   p <- (p + tau grad G) / (1 + tau |grad G|)
// with forward differences and Neumann boundary (grad is zero across the last
// row/column, div = -grad^T).
//
// K steps on one tile run in shared memory: the tile is loaded with a halo of
// K pixels (a step reads its neighbours at distance one), every step is
// computed over the whole loaded region, and after K steps the central tile,
// whose dependence cone stayed inside the region, is written out.  The loaded
// region is 64 wide (output 64 - 2K + halo K each side) so that warps of 32
// columns fill it.  K (2 .. 8) trades halo recomputation against launches;
// every K gives bit-identical results, so it is a free tuning parameter
// (chosen per image size by the autotuner, default 5).  z/lam is formed once per launch; |grad G| and the
// reciprocal of 1 + tau |grad G| use the hardware approximations (within two
// ulp), and the rounding of every operation is spelled out (fmaf, __fmul_rn,
// ...) so that all kernels built on this function give bit-identical results.
#pragma once

#include "common.cuh"

namespace pyhst {

constexpr int kChR = 64;                    // loaded region (two full warp rows)
constexpr int kChW = kChR + 2;              // region + zero guard ring
constexpr int kChKDefault = 5;              // steps fused per launch unless tuned
__host__ __device__ constexpr int chambolle_tile_size(int K) { return kChR - 2 * K; }
inline bool chambolle_k_supported(int K) { return K == 2 || K == 3 || K == 4 || K == 5 || K == 6 || K == 8; }
constexpr int kChThreads = 256;
constexpr size_t kChSmem = sizeof(float) * 4 * kChW * kChW;   // dynamic shared memory per CTA

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int kChK>
__device__ __forceinline__ void chambolle_tile(const float *__restrict__ z, const float *__restrict__ p1,
                                               const float *__restrict__ p2, float *__restrict__ q1,
                                               float *__restrict__ q2, float lam, float tau, int nx, int ny, int i0,
                                               int j0, int steps, bool first) {
    // sz holds z / lam; threads as 32 columns x 8 rows
    extern __shared__ __align__(16) float ch_smem[];
    float(*sz)[kChW] = reinterpret_cast<float(*)[kChW]>(ch_smem);
    float(*s1)[kChW] = sz + kChW;
    float(*s2)[kChW] = s1 + kChW;
    float(*sg)[kChW] = s2 + kChW;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int ri0 = i0 - kChK - 1, rj0 = j0 - kChK - 1;   // global coordinates of array cell (0, 0)
    for (int r = ty; r < kChW; r += 8)
        for (int c = tx; c < kChW; c += 32) {
            const int gi = ri0 + r, gj = rj0 + c;
            float vz = 0.0f, v1 = 0.0f, v2 = 0.0f;
            if (r >= 1 && r <= kChR && c >= 1 && c <= kChR && gi >= 0 && gi < ny && gj >= 0 && gj < nx) {
                const size_t k = (size_t)gi * nx + gj;
                vz = __fdiv_rn(z[k], lam);
                if (!first) {
                    v1 = p1[k];
                    v2 = p2[k];
                }
            }
            sz[r][c] = vz;
            s1[r][c] = v1;
            s2[r][c] = v2;
            sg[r][c] = 0.0f;
        }
    __syncthreads();
    // cells of the loaded region that lie inside the image
    const int r_lo = max(1, -ri0), r_hi = min(kChR, ny - 1 - ri0);
    const int c_lo = max(1, -rj0), c_hi = min(kChR, nx - 1 - rj0);
    // Boundary handling without branches in the cell loops: p1 stays exactly 0
    // on the last image row and p2 on the last column (their forward
    // differences are 0 there, and p starts at 0), and cells outside the image
    // hold 0, so div p adds its four terms unconditionally (adding or
    // subtracting 0 changes no bits); the forward differences of the last row
    // and column are masked by multiplying with 0.
    float m2c[(kChR + 31) / 32];                       // per column of this thread: gj + 1 < nx
#pragma unroll
    for (int q = 0; q < (kChR + 31) / 32; ++q) {
        const int c = c_lo + tx + 32 * q;
        m2c[q] = (rj0 + c + 1 < nx) ? 1.0f : 0.0f;
    }
    for (int st = 0; st < steps; ++st) {
        for (int r = r_lo + ty; r <= r_hi; r += 8) {
            for (int c = c_lo + tx; c <= c_hi; c += 32) {
                float d = 0.0f;
                d = __fadd_rn(d, s1[r][c]);
                d = __fsub_rn(d, s1[r - 1][c]);
                d = __fadd_rn(d, s2[r][c]);
                d = __fsub_rn(d, s2[r][c - 1]);
                sg[r][c] = __fsub_rn(d, sz[r][c]);
            }
        }
        __syncthreads();
        for (int r = r_lo + ty; r <= r_hi; r += 8) {
            const float m1 = (ri0 + r + 1 < ny) ? 1.0f : 0.0f;
#pragma unroll
            for (int q = 0; q < (kChR + 31) / 32; ++q) {
                const int c = c_lo + tx + 32 * q;
                if (c > c_hi) break;
                const float g0 = sg[r][c];
                const float g1 = __fmul_rn(m1, __fsub_rn(sg[r + 1][c], g0));
                const float g2 = __fmul_rn(m2c[q], __fsub_rn(sg[r][c + 1], g0));
                const float inv = rcp_approx(fmaf(tau, sqrt_approx(fmaf(g1, g1, __fmul_rn(g2, g2))), 1.0f));
                s1[r][c] = __fmul_rn(fmaf(tau, g1, s1[r][c]), inv);
                s2[r][c] = __fmul_rn(fmaf(tau, g2, s2[r][c]), inv);
            }
        }
        __syncthreads();
    }
    constexpr int kChT = chambolle_tile_size(kChK);
    for (int r = ty; r < kChT; r += 8)
        for (int c = tx; c < kChT; c += 32) {
            const int gi = i0 + r, gj = j0 + c;
            if (gi < ny && gj < nx) {
                const size_t k = (size_t)gi * nx + gj;
                q1[k] = s1[r + kChK + 1][c + kChK + 1];
                q2[k] = s2[r + kChK + 1][c + kChK + 1];
            }
        }
}

// Launch plan of n_inner steps: launch m runs steps(m) steps, the first
// from a zero dual field; the result is in the "a" buffers if the number of
// launches is odd, else in "b".
__host__ __device__ inline int chambolle_launches(int n_inner, int K) { return (n_inner + K - 1) / K; }
__host__ __device__ inline int chambolle_steps(int n_inner, int m, int K) {
    return m + 1 < chambolle_launches(n_inner, K) ? K : n_inner - K * m;
}

// Steps fused per launch for an image size: the autotuned choice if there is
// one (pyhst_autotune_tv_prox / pyhst_set_tv_prox_steps), else kChKDefault.
int chambolle_k_for(int nx, int ny);

// Instantiate F<K> for the supported K and call it (returns its status).
#define PYHST_CHAMBOLLE_DISPATCH(K, F, ...)         \
    switch (K) {                                    \
        case 2: return F<2>(__VA_ARGS__);           \
        case 3: return F<3>(__VA_ARGS__);           \
        case 4: return F<4>(__VA_ARGS__);           \
        case 6: return F<6>(__VA_ARGS__);           \
        case 8: return F<8>(__VA_ARGS__);           \
        default: return F<5>(__VA_ARGS__);          \
    }

}  // namespace pyhst
