// Fused Chambolle steps for the TV prox (Eq. 2; Chambolle's dual fixed point):
//   G = div p - z / lam,   p <- (p + tau grad G) / (1 + tau |grad G|)
// with forward differences and Neumann boundary (grad is zero across the last
// row/column, div = -grad^T).
//
// K steps on one tile run on chip: the tile is loaded with a halo of K
// pixels (a step reads its neighbours at distance one), every step is
// computed over the whole loaded region, and after K steps the central tile,
// whose dependence cone stayed inside the region, is written out.  The loaded
// region is 64 x 64 (output 64 - 2K, halo K each side); outside it every field
// reads as zero.  K (2 .. 8) trades halo recomputation against launches;
// every K gives bit-identical results, so it is a free tuning parameter
// (chosen per image size by the autotuner, default 5).
//
// The fields live in registers: warp w holds region rows 8w+1 .. 8w+8 and
// lane l the two columns 2l+1, 2l+2 of them (p1, p2 and G for 16 cells per
// thread; z / lam, read once per cell and step, in shared memory or in
// registers, a per-kernel choice).  Horizontal neighbours come from the adjacent lane by a
// shuffle, vertical ones from the thread's own rows, and only the first G row
// and the last p1 row of each strip cross to the neighbouring warp, through
// two small shared-memory arrays (two barriers per step).  z/lam is formed
// once per launch; |grad G| and the reciprocal of 1 + tau |grad G| use the
// hardware approximations (within two ulp).  A thread's two cells of a row
// are computed together by paired float32 instructions (f32x2; each half
// rounds as the scalar operation would), and the rounding of every operation
// is spelled out (fma2, mul2, ...) so that all kernels built on this function
// give bit-identical results.
#pragma once

#include "common.cuh"

namespace pyhst {

constexpr int kChRows = 8;                  // region rows per warp
constexpr int kChWarps = 8;                 // warps per CTA (16, a 128 x 64 region, measured slower)
constexpr int kChRH = kChRows * kChWarps;   // loaded region: rows
constexpr int kChRW = 64;                   // loaded region: columns (two per lane)
constexpr int kChKDefault = 5;              // steps fused per launch unless tuned
// output tile of K fused steps: the region less a halo of K on each side
__host__ __device__ constexpr int chambolle_tile_h(int K) { return kChRH - 2 * K; }
__host__ __device__ constexpr int chambolle_tile_w(int K) { return kChRW - 2 * K; }
inline bool chambolle_k_supported(int K) { return K == 2 || K == 3 || K == 4 || K == 5 || K == 6 || K == 8; }
constexpr int kChThreads = 32 * kChWarps;
constexpr int kChMinBlocks = 1024 / kChThreads;   // register budget: 64 registers a thread (1024 threads per SM)
// dynamic shared memory per CTA: the strips' last p1 rows and first G rows,
// each with a zero guard row, then (kChSmem) z / lam of the region as float2
// pairs of a thread's two columns; kChSmemRegs when z / lam stays in
// registers (see chambolle_tile)
constexpr size_t kChExchange = sizeof(float) * 2 * (kChWarps + 1) * kChRW;
constexpr size_t kChSmem = kChExchange + sizeof(float) * kChRH * kChRW;
constexpr size_t kChSmemRegs = kChExchange;

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

// The K steps on the registers of one thread.  kEdge: the region touches the
// image border.  Then the forward differences of the last image row / column
// and of the rows / columns outside the image are multiplied by 0 (m1, m2;
// inside the image every such factor is 1 and is left out, which changes no
// bits).  That keeps p1 on the row above the image and p2 on the column left
// of it at their initial +0 (a zero gradient leaves +0 at +0), the only
// outside values a cell inside reads (its divergence reads p1 above and p2
// to the left; its gradient reads G below and to the right, masked at the
// last row and column), so the cells outside evolve freely without
// changing a bit inside and need no masks of their own.
//
// Rows stream through a step: G of row i is formed from the dual field as it
// was at the start of the step (row i - 1 is updated only after G of row i
// exists), then row i - 1 is updated from G of rows i - 1 and i, so only two
// rows of G are live.  Each cell's operations and their order are those of
// the step as written above.
template <bool kEdge, bool kZsSmem>
__device__ __forceinline__ void chambolle_steps_regs(const float2 (*zs)[kChRW / 2], const float2 (&zl)[kChRows],
                                                     float2 (&a1)[kChRows], float2 (&a2)[kChRows],
                                                     float (*xp)[kChRW], float (*xg)[kChRW], float tau, int steps,
                                                     const float (&m1)[kChRows],
                                                     const float2 m2) {
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float2 tau2 = make_float2(tau, tau), one2 = make_float2(1.0f, 1.0f);
    // G of row i (old dual field); u: p1 of the row above
    auto form_g = [&](int i, float2 u) {
        float left = __shfl_up_sync(0xffffffffu, a2[i].y, 1);
        if (tx == 0) left = 0.0f;
        const float2 zz = kZsSmem ? zs[kChRows * w + i][tx] : zl[i];   // z / lam of the thread's two cells
        float2 d = sub2(a1[i], u);
        d = add2(d, a2[i]);
        d = sub2(d, make_float2(left, a2[i].x));
        return sub2(d, zz);
    };
    // update row i from G of rows i and i + 1
    auto update = [&](int i, float2 G, float2 dn) {
        float right = __shfl_down_sync(0xffffffffu, G.x, 1);
        if (tx == 31) right = 0.0f;
        float2 g1 = sub2(dn, G), g2 = sub2(make_float2(G.y, right), G);
        if (kEdge) {
            g1 = mul2(make_float2(m1[i], m1[i]), g1);
            g2 = mul2(m2, g2);
        }
        const float2 s = fma2(g1, g1, mul2(g2, g2));
        const float2 den = fma2(tau2, make_float2(sqrt_approx(s.x), sqrt_approx(s.y)), one2);
        const float2 inv = make_float2(rcp_approx(den.x), rcp_approx(den.y));
        const float2 n1 = mul2(fma2(tau2, g1, a1[i]), inv);
        const float2 n2 = mul2(fma2(tau2, g2, a2[i]), inv);
        a1[i] = n1;
        a2[i] = n2;
    };
    for (int st = 0; st < steps; ++st) {
        const float2 up = *reinterpret_cast<const float2 *>(&xp[w][2 * tx]);   // p1 row above the strip
        float2 Gp = form_g(0, up);
        *reinterpret_cast<float2 *>(&xg[w][2 * tx]) = Gp;
#pragma unroll
        for (int i = 1; i < kChRows; ++i) {
            const float2 Gc = form_g(i, a1[i - 1]);
            update(i - 1, Gp, Gc);
            Gp = Gc;
        }
        __syncthreads();
        const float2 down = *reinterpret_cast<const float2 *>(&xg[w + 1][2 * tx]);   // G row below the strip
        update(kChRows - 1, Gp, down);
        *reinterpret_cast<float2 *>(&xp[w + 1][2 * tx]) = a1[kChRows - 1];
        __syncthreads();
    }
}

// One tile's K steps.  kEdge: the loaded region touches the image border or
// its last row or column (see chambolle_tile); otherwise every cell of the
// region is inside the image, so the loads, the steps and the stores need no
// bounds checks and address the image by constant row offsets.
template <int kChK, bool kEdge, bool kZsSmem>
__device__ __forceinline__ void chambolle_tile_body(const float *__restrict__ z, const float *__restrict__ p1,
                                                    const float *__restrict__ p2, float *__restrict__ q1,
                                                    float *__restrict__ q2, float lam, float inv_lam, float tau,
                                                    int nx, int ny, int ri0, int rj0, int steps, bool first,
                                                    float *__restrict__ xout, bool keep_p) {
    extern __shared__ __align__(16) float ch_smem[];
    float(*xp)[kChRW] = reinterpret_cast<float(*)[kChRW]>(ch_smem);   // xp[w + 1]: last p1 row of strip w
    float(*xg)[kChRW] = xp + (kChWarps + 1);                            // xg[w]: first G row of strip w
    float2(*zs)[kChRW / 2] = reinterpret_cast<float2(*)[kChRW / 2]>(ch_smem + kChExchange / sizeof(float));
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = kChRows * w + 1, c0 = 2 * tx + 1;      // this thread's first region row and column
    float2 zl[kChRows], a1[kChRows], a2[kChRows], m2;
    float m1[kChRows];
    // z / lam of the thread's cells (i, 0) and (i, 1)
    auto put_zl = [&](int i, float v0, float v1) {
        if constexpr (kZsSmem) {
            zs[kChRows * w + i][tx] = make_float2(v0, v1);
        } else {
            zl[i] = make_float2(v0, v1);
        }
    };
    if (!kEdge) {
        const size_t base = (size_t)(ri0 + r0) * nx + (size_t)(rj0 + c0);
        const float *zr = z + base;
#pragma unroll
        for (int i = 0; i < kChRows; ++i, zr += nx) {
            m1[i] = 1.0f;
            put_zl(i, __fmul_rn(zr[0], inv_lam), __fmul_rn(zr[1], inv_lam));
        }
        if (first) {
#pragma unroll
            for (int i = 0; i < kChRows; ++i) a1[i] = a2[i] = make_float2(0.0f, 0.0f);
        } else {
            const float *r1 = p1 + base, *r2 = p2 + base;
#pragma unroll
            for (int i = 0; i < kChRows; ++i, r1 += nx, r2 += nx) {
                a1[i] = make_float2(r1[0], r1[1]);
                a2[i] = make_float2(r2[0], r2[1]);
            }
        }
        m2 = make_float2(1.0f, 1.0f);
    } else {
        // 1 on the image's columns / rows that have a forward difference, 0 on
        // its last one and outside it
        auto has_diff = [](int g, int n) { return g >= 0 && g + 1 < n ? 1.0f : 0.0f; };
        m2 = make_float2(has_diff(rj0 + c0, nx), has_diff(rj0 + c0 + 1, nx));
#pragma unroll
        for (int i = 0; i < kChRows; ++i) {
            const int gi = ri0 + r0 + i;
            m1[i] = has_diff(gi, ny);
            float vz[2], v1s[2], v2s[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int gj = rj0 + c0 + j;
                float v1 = 0.0f, v2 = 0.0f;
                vz[j] = 0.0f;
                if (gi >= 0 && gi < ny && gj >= 0 && gj < nx) {
                    const size_t k = (size_t)gi * nx + gj;
                    vz[j] = __fmul_rn(z[k], inv_lam);
                    if (!first) {
                        v1 = p1[k];
                        v2 = p2[k];
                    }
                }
                v1s[j] = v1;
                v2s[j] = v2;
            }
            a1[i] = make_float2(v1s[0], v1s[1]);
            a2[i] = make_float2(v2s[0], v2s[1]);
            put_zl(i, vz[0], vz[1]);
        }
    }
    if (w == 0) *reinterpret_cast<float2 *>(&xp[0][2 * tx]) = make_float2(0.0f, 0.0f);
    if (w == kChWarps - 1) *reinterpret_cast<float2 *>(&xg[kChWarps][2 * tx]) = make_float2(0.0f, 0.0f);
    *reinterpret_cast<float2 *>(&xp[w + 1][2 * tx]) = a1[kChRows - 1];
    __syncthreads();
    chambolle_steps_regs<kEdge, kZsSmem>(zs, zl, a1, a2, xp, xg, tau, steps, m1, m2);
    // write the central tile: region rows kChK + 1 .. kChRH - kChK, columns kChK + 1 .. kChRW - kChK
    if (xout) {
        const float2 up = *reinterpret_cast<const float2 *>(&xp[w][2 * tx]);   // p1 row above the strip
#pragma unroll
        for (int i = 0; i < kChRows; ++i) {
            float left = __shfl_up_sync(0xffffffffu, a2[i].y, 1);
            if (tx == 0) left = 0.0f;
            const float a1r[2] = {a1[i].x, a1[i].y}, a2r[2] = {a2[i].x, a2[i].y};
            const float2 pu2 = i > 0 ? a1[i - 1] : up;
            const float pur[2] = {pu2.x, pu2.y};
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r = r0 + i, c = c0 + j, gi = ri0 + r, gj = rj0 + c;
                // inside the image the region is clear of the border: all four divergence terms exist
                if (r > kChK && r <= kChRH - kChK && c > kChK && c <= kChRW - kChK && (!kEdge || (gi < ny && gj < nx))) {
                    const size_t k = (size_t)gi * nx + gj;
                    const float pu = pur[j];
                    const float pl = j > 0 ? a2r[0] : left;
                    float dv = 0.0f;
                    if (!kEdge || gi + 1 < ny) dv += a1r[j];
                    if (!kEdge || gi > 0) dv -= pu;
                    if (!kEdge || gj + 1 < nx) dv += a2r[j];
                    if (!kEdge || gj > 0) dv -= pl;
                    xout[k] = fmaf(-lam, dv, z[k]);
                    if (keep_p) {
                        q1[k] = a1r[j];
                        q2[k] = a2r[j];
                    }
                }
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kChRows; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = r0 + i, c = c0 + j, gi = ri0 + r, gj = rj0 + c;
            if (r > kChK && r <= kChRH - kChK && c > kChK && c <= kChRW - kChK && (!kEdge || (gi < ny && gj < nx))) {
                const size_t k = (size_t)gi * nx + gj;
                q1[k] = j == 0 ? a1[i].x : a1[i].y;
                q2[k] = j == 0 ? a2[i].x : a2[i].y;
            }
        }
}

// K steps on the tile whose output corner is (i0, j0): the region loaded is
// rows i0 - K .. i0 - K - 1 + kChRH and columns j0 - K .. j0 - K - 1 + kChRW.
// xout == nullptr: write the dual field of the central tile to q1, q2.
// Otherwise (the last launch of a prox) write the prox itself to xout,
// x = z - lam div p: the divergence's four terms added in a fixed order,
// those across the image border left out, then one fma; with keep_p the
// dual field is written to q1, q2 as well (for the duality gap).
// z / lam is formed as z times the correctly rounded reciprocal of lam, and
// kept in shared memory (kZsSmem; dynamic shared memory kChSmem) or in
// registers (kChSmemRegs): the same bits either way.  Measured on the B300,
// shared memory is faster for the single-slice kernels (no spills at 64
// registers) and registers for the batched kernel.
template <int kChK, bool kZsSmem = true>
__device__ __forceinline__ void chambolle_tile(const float *__restrict__ z, const float *__restrict__ p1,
                                               const float *__restrict__ p2, float *__restrict__ q1,
                                               float *__restrict__ q2, float lam, float tau, int nx, int ny, int i0,
                                               int j0, int steps, bool first, float *__restrict__ xout = nullptr,
                                               bool keep_p = false) {
    const int ri0 = i0 - kChK - 1, rj0 = j0 - kChK - 1;   // global coordinates of region cell (0, 0)
    const float inv_lam = __frcp_rn(lam);
    // the whole region inside the image and clear of its last row and column
    const bool interior = ri0 + 1 >= 0 && ri0 + kChRH + 1 < ny && rj0 + 1 >= 0 && rj0 + kChRW + 1 < nx;
    if (interior)
        chambolle_tile_body<kChK, false, kZsSmem>(z, p1, p2, q1, q2, lam, inv_lam, tau, nx, ny, ri0, rj0, steps,
                                                  first, xout, keep_p);
    else
        chambolle_tile_body<kChK, true, kZsSmem>(z, p1, p2, q1, q2, lam, inv_lam, tau, nx, ny, ri0, rj0, steps,
                                                 first, xout, keep_p);
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
