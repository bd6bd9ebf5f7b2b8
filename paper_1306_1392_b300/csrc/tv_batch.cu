// Mixed-size batch of TV-penalised solves (Eq. 3 by ISTA/FISTA, Sec. 3.1).
//
// Slices of different sizes and angle sets run together: every stage of an
// outer iteration (gradient back-projection with the gradient step in its
// epilogue, each Chambolle launch, the last of which writes the prox,
// projection, momentum and energy) is ONE launch over the
// whole batch, each CTA taking a (slice, tile) work item from a list built on
// the host, with per-slice descriptors in device memory.  The n_iter
// iterations are captured in one CUDA graph and launched once (unless the
// caller's stream is already being captured, in which case the launches join
// the caller's capture).  The arithmetic is that of pyhst_tv_solve: one
// projection and one back-projection per iteration (P y carried by linearity),
// float64 energies from block partials summed in a fixed order.  The step
// size is estimated once per distinct geometry (same angle/axis arrays, sizes,
// centre and pixel size) by power iteration on one representative slice.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "chambolle.cuh"
#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kBT = 256;            // threads of the element-wise kernels
constexpr int kSinoBlock = 1024;    // sinogram elements per work item (4 per thread)

struct TvSlice {
    float *y, *xa, *xb, *z, *g, *p1a, *p2a, *p1b, *p2b;
    float *Axa, *Axb, *Ry;   // P x of the two iterates; Ry = P y - sino
    const float *sino;
    float *x_user;
    double *energy;
    double *gap;          // NULL, or the prox's duality gap per iteration
    int nx, ny, M;        // image size, sinogram elements
    int px_first, sn_first;
    int rep;              // representative slice of the geometry group (power iteration)
    float beta;           // weight of TV in this slice's Eq. 3
};

struct Scal {
    double *L;            // [n]
    double *ray;          // [n] ||P v||^2 of representatives
    float *invL, *lam, *invn;
};

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kBT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = (l < kBT / 32) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// Pixel work items are 32 columns x kPxRows rows; thread t of a CTA takes
// column t % 32 and rows t / 32 + 8 r (r < kPxRows / 8).
constexpr int kPxRows = 64;

// Partial-sum slots: a slice's pixel items (32 x kPxRows) and sinogram items are
// numbered from its px_first / sn_first in the order the host lists them, so
// that work lists over any subset of slices write the same slots.
__device__ __forceinline__ int px_slot(const int4 it, const TvSlice &s) {
    return s.px_first + it.z * ((s.nx + 31) / 32) + it.y;
}
__device__ __forceinline__ int sn_slot(const int4 it, const TvSlice &s) { return s.sn_first + it.y; }

// pixel (i, j) of row group r of a pixel work item; false if outside the slice
__device__ __forceinline__ bool px_of(const int4 it, const TvSlice &s, int r, int &i, int &j) {
    j = it.y * 32 + (threadIdx.x & 31);
    i = it.z * kPxRows + (threadIdx.x >> 5) + 8 * r;
    return i < s.ny && j < s.nx;
}
__device__ __forceinline__ int px_items(const TvSlice &s) { return ((s.nx + 31) / 32) * ((s.ny + kPxRows - 1) / kPxRows); }

// Launch of parity index m of the fused Chambolle steps (see chambolle.cuh;
// m = 0 starts from a zero field and writes the a buffers, m > 0 reads a for
// m odd, else b, and writes the other) on tile (items[k].y, items[k].z) of
// slice items[k].x; slices with beta = 0 skip.
template <int K>
__global__ void __launch_bounds__(kChThreads, kChMinBlocks)
b_chambolle(const TvSlice *__restrict__ d, const int4 *__restrict__ items, Scal sc, float tau, int m, int steps,
            int final_par, int keep_p) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    constexpr int Th = chambolle_tile_h(K), Tw = chambolle_tile_w(K);
    // final_par >= 0: the last launch, which writes x_new (parity as in b_prox_final)
    float *xn = final_par < 0 ? nullptr : (final_par ? s.xa : s.xb);
    if (s.beta == 0.0f) {                       // no TV term: x_new = z on this tile
        if (xn)
            for (int e = threadIdx.x; e < Th * Tw; e += kChThreads) {
                const int i = it.z * Th + e / Tw, j = it.y * Tw + e % Tw;
                if (i < s.ny && j < s.nx) xn[(size_t)i * s.nx + j] = s.z[(size_t)i * s.nx + j];
            }
        return;
    }
    const bool odd = m & 1;
    const float *s1 = odd ? s.p1a : s.p1b, *s2 = odd ? s.p2a : s.p2b;
    float *d1 = (m == 0 || !odd) ? s.p1a : s.p1b, *d2 = (m == 0 || !odd) ? s.p2a : s.p2b;
    // keep_p: the last launch also writes the final dual field, of every slice
    // (2) or of the slices that report the gap (1)
    // z / lam in registers: faster than shared memory for this kernel on the B300 (same bits)
    chambolle_tile<K, false>(s.z, s1, s2, d1, d2, sc.lam[it.x], tau, s.nx, s.ny, it.z * Th, it.y * Tw, steps, m == 0,
                             xn, keep_p == 2 || (keep_p == 1 && s.gap != nullptr));
}

template <int K>
int b_chambolle_attr_k() {
    return cudaFuncSetAttribute(b_chambolle<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChSmemRegs) ==
                   cudaSuccess
               ? PYHST_OK
               : cuda_status("Chambolle kernel shared-memory attribute");
}
int b_chambolle_attr(int K) { PYHST_CHAMBOLLE_DISPATCH(K, b_chambolle_attr_k) }

template <int K>
int b_chambolle_launches_k(int nch, const TvSlice *T, const int4 *items, int nchf, const int4 *items_f, Scal sc,
                           float tau, int n_inner, int par, int keep_p, int q0, cudaStream_t st) {
    const int Lc = chambolle_launches(n_inner, K);
    for (int m = 0; m + 1 < Lc; ++m) {
        ProfScope prof(kProfChambolle, st);
        b_chambolle<K><<<nch, kChThreads, kChSmemRegs, st>>>(T, items, sc, tau, q0 + m,
                                                             chambolle_steps(n_inner, m, K), -1, 0);
    }
    // the last launch writes x_new; it reads p one row above and one column left
    // of its tiles, so it takes the halo of K + 1 steps (same bits)
    {
        ProfScope prof(kProfChambolle, st);
        b_chambolle<K + 1><<<nchf, kChThreads, kChSmemRegs, st>>>(T, items_f, sc, tau, q0 + Lc - 1,
                                                              chambolle_steps(n_inner, Lc - 1, K), par, keep_p);
    }
    return cuda_status("batched Chambolle kernels");
}
// All launches of the Chambolle steps of one iteration, with parity indices
// q0, q0 + 1, ..; the last one writes x_new (xa for par = 1, xb for par = 0)
// instead of the dual field, and with keep_p the final dual field too (in the
// a buffers when its index is even): of every slice for keep_p = 2, of the
// slices that report the duality gap for keep_p = 1.
int b_chambolle_launches(int K, int nch, const TvSlice *T, const int4 *items, int nchf, const int4 *items_f, Scal sc,
                         float tau, int n_inner, int par, int keep_p, int q0, cudaStream_t st) {
    PYHST_CHAMBOLLE_DISPATCH(K, b_chambolle_launches_k, nch, T, items, nchf, items_f, sc, tau, n_inner, par, keep_p,
                             q0, st)
}

// Duality-gap partial of a pixel item (the prox's gap, lam * sum of
// |grad x| + p . grad x over the slice, as in pyhst_tv_prox): x_new of
// it_parity, the final dual field in the a buffers (pa_final) or b.
__global__ void b_gap_partial(const TvSlice *__restrict__ d, const int4 *__restrict__ items, int it_parity,
                              int pa_final, double *__restrict__ part) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    if (!s.gap || s.beta == 0.0f) {             // uniform over the CTA
        if (threadIdx.x == 0) part[px_slot(it, s)] = 0.0;
        return;
    }
    const float *xn = it_parity ? s.xa : s.xb;
    const float *Q1 = pa_final ? s.p1a : s.p1b, *Q2 = pa_final ? s.p2a : s.p2b;
    RunSum rs;
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (!px_of(it, s, r, i, j)) continue;
        const size_t k = (size_t)i * s.nx + j;
        const float v = xn[k];
        const float d1 = (i + 1 < s.ny) ? xn[k + s.nx] - v : 0.0f;
        const float d2 = (j + 1 < s.nx) ? xn[k + 1] - v : 0.0f;
        rs.add(sqrtf(fmaf(d1, d1, d2 * d2)) + fmaf(Q1[k], d1, Q2[k] * d2));
    }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[px_slot(it, s)] = acc;
}

// gap[k] of slice blockIdx.x: lam times its partials in a fixed order (0 for beta = 0)
__global__ void b_finalize_gap(const TvSlice *__restrict__ d, const double *__restrict__ part, Scal sc, int k) {
    const TvSlice s = d[blockIdx.x];
    if (!s.gap) return;                          // uniform over the CTA
    double t = 0.0;
    const int n_px = px_items(s);
    if (s.beta != 0.0f)
        for (int e = s.px_first + threadIdx.x; e < s.px_first + n_px; e += kBT) t += part[e];
    t = block_sum(t);
    if (threadIdx.x == 0) s.gap[(size_t)k] = s.beta == 0.0f ? 0.0 : (double)sc.lam[blockIdx.x] * t;
}

// x_new = z - lam div p (p in the buffers of `parity`); with lam = 0, x_new = z
__global__ void b_prox_final(const TvSlice *__restrict__ d, const int4 *__restrict__ items, Scal sc, int parity,
                             int it_parity, int identity) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    float *xn = it_parity ? s.xa : s.xb;
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (!px_of(it, s, r, i, j)) continue;
        const size_t k = (size_t)i * s.nx + j;
        if (identity || s.beta == 0.0f) {
            xn[k] = s.z[k];
            continue;
        }
        const float *P1 = parity ? s.p1b : s.p1a, *P2 = parity ? s.p2b : s.p2a;
        float dv = 0.0f;
        if (i + 1 < s.ny) dv += P1[k];
        if (i > 0) dv -= P1[k - s.nx];
        if (j + 1 < s.nx) dv += P2[k];
        if (j > 0) dv -= P2[k - 1];
        xn[k] = fmaf(-sc.lam[it.x], dv, s.z[k]);
    }
}

// data partial ||Axn - b||^2 and Ry = Ay - b, Ay = Axn + w (Axn - Axo) rounded first
__global__ void b_sino_update(const TvSlice *__restrict__ d, const int4 *__restrict__ items, float w, int it_parity,
                              double *__restrict__ part) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    const float *axn = it_parity ? s.Axa : s.Axb, *axo = it_parity ? s.Axb : s.Axa;
    RunSum rs;
    const int base = it.y * kSinoBlock;
    for (int e = base + threadIdx.x; e < min(base + kSinoBlock, s.M); e += kBT) {
        const float v = axn[e], b = s.sino[e];
        const float r = v - b;
        rs.add(r * r);
        const float ay = fmaf(w, v - axo[e], v);
        s.Ry[e] = ay - b;
    }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[sn_slot(it, s)] = acc;
}

// TV(xn) partial (Eq. 2) and y = xn + w (xn - xo)
__global__ void b_image_update(const TvSlice *__restrict__ d, const int4 *__restrict__ items, float w, int it_parity,
                               double *__restrict__ part) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    const float *xn = it_parity ? s.xa : s.xb, *xo = it_parity ? s.xb : s.xa;
    float tvp = 0.0f;
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (!px_of(it, s, r, i, j)) continue;
        const size_t k = (size_t)i * s.nx + j;
        const float v = xn[k];
        const float d1 = (i + 1 < s.ny) ? xn[k + s.nx] - v : 0.0f;
        const float d2 = (j + 1 < s.nx) ? xn[k + 1] - v : 0.0f;
        tvp += sqrtf(d1 * d1 + d2 * d2);
        s.y[k] = fmaf(w, v - xo[k], v);
    }
    // TV partial: each thread's terms and then each warp's in float32 (fixed
    // order and shuffle tree, relative error ~1e-7), the 8 warp sums in
    // float64 in order (FP64 is scarce here)
    for (int o = 16; o > 0; o >>= 1) tvp += __shfl_down_sync(0xffffffffu, tvp, o);
    __shared__ float wsum[kBT / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = tvp;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int q = 0; q < kBT / 32; ++q) acc += (double)wsum[q];
        part[px_slot(it, s)] = acc;
    }
}

// energy[k] of slice blockIdx.x from its partials, in a fixed order
__global__ void b_finalize_energy(const TvSlice *__restrict__ d, const double *__restrict__ part_sn,
                                  const double *__restrict__ part_px, int n_iter, int k, int n) {
    const TvSlice s = d[blockIdx.x];
    (void)n;
    double a = 0.0, t = 0.0;
    for (int e = s.sn_first + threadIdx.x; e < s.sn_first + (s.M + kSinoBlock - 1) / kSinoBlock; e += kBT)
        a += part_sn[e];
    const int n_px = px_items(s);
    for (int e = s.px_first + threadIdx.x; e < s.px_first + n_px; e += kBT) t += part_px[e];
    a = block_sum(a);
    t = block_sum(t);
    if (threadIdx.x == 0 && s.energy) s.energy[(size_t)k] = 0.5 * a + (double)s.beta * t;
}

// ||g||^2 partial of a slice's pixels (power iteration)
__global__ void b_sqnorm_g(const TvSlice *__restrict__ d, const int4 *__restrict__ items, double *__restrict__ part) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (!px_of(it, s, r, i, j)) continue;
        const float v = s.g[(size_t)i * s.nx + j];
        acc += (double)v * (double)v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[px_slot(it, s)] = acc;
}

// ||P v||^2 partial of a slice's sinogram (power iteration end)
__global__ void b_sqnorm_axa(const TvSlice *__restrict__ d, const int4 *__restrict__ items, double *__restrict__ part) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    double acc = 0.0;
    const int base = it.y * kSinoBlock;
    for (int e = base + threadIdx.x; e < min(base + kSinoBlock, s.M); e += kBT) {
        const float v = s.Axa[e];
        acc += (double)v * (double)v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[sn_slot(it, s)] = acc;
}

// per representative: invn = 1/sqrt(sum) (mode 0) or ray = sum (mode 1)
__global__ void b_finalize_norm(const TvSlice *__restrict__ d, const int *__restrict__ reps, const double *__restrict__ part,
                                Scal sc, int mode) {
    const int r = reps[blockIdx.x];
    const TvSlice s = d[r];
    double a = 0.0;
    if (mode == 0) {
        const int n_px = px_items(s);
        for (int e = s.px_first + threadIdx.x; e < s.px_first + n_px; e += kBT) a += part[e];
    } else {
        for (int e = s.sn_first + threadIdx.x; e < s.sn_first + (s.M + kSinoBlock - 1) / kSinoBlock; e += kBT)
            a += part[e];
    }
    a = block_sum(a);
    if (threadIdx.x == 0) {
        if (mode == 0) sc.invn[r] = (float)(1.0 / sqrt(a));
        else sc.ray[r] = a;
    }
}

__global__ void b_scale_v(const TvSlice *__restrict__ d, const int4 *__restrict__ items, Scal sc) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (!px_of(it, s, r, i, j)) continue;
        const size_t k = (size_t)i * s.nx + j;
        s.z[k] = s.g[k] * sc.invn[it.x];
    }
}

__global__ void b_fill_v(const TvSlice *__restrict__ d, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (px_of(it, s, r, i, j)) s.z[(size_t)i * s.nx + j] = 1.0f;
    }
}

__global__ void b_set_step(const TvSlice *__restrict__ d, Scal sc, double L_fixed, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double L = L_fixed > 0.0 ? L_fixed : 1.01 * sc.ray[d[k].rep];
    sc.L[k] = L;
    sc.invL[k] = (float)(1.0 / L);
    sc.lam[k] = (float)((double)d[k].beta / L);
}

// start: xa = x_user (warm) or 0, y = xa; result: x_user = x of the last iteration
__global__ void b_copy_x(const TvSlice *__restrict__ d, const int4 *__restrict__ items, int mode, int it_parity) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
#pragma unroll
    for (int r = 0; r < kPxRows / 8; ++r) {
        int i, j;
        if (!px_of(it, s, r, i, j)) continue;
        const size_t k = (size_t)i * s.nx + j;
        if (mode == 0) {           // cold start
            s.xa[k] = 0.0f;
            s.y[k] = 0.0f;
        } else if (mode == 1) {    // warm start
            const float v = s.x_user[k];
            s.xa[k] = v;
            s.y[k] = v;
        } else {                   // result
            s.x_user[k] = it_parity ? s.xa[k] : s.xb[k];
        }
    }
}

__global__ void b_copy_sino_start(const TvSlice *__restrict__ d, const int4 *__restrict__ items, int warm) {
    const int4 it = items[blockIdx.x];
    const TvSlice s = d[it.x];
    const int base = it.y * kSinoBlock;
    for (int e = base + threadIdx.x; e < min(base + kSinoBlock, s.M); e += kBT) {
        const float v = warm ? s.Axa[e] : 0.0f;
        s.Axa[e] = v;
        s.Ry[e] = v - s.sino[e];
    }
}

// ------------------------------------------------------------------ host plan
struct Plan {
    int n = 0;
    std::vector<int> rep;                       // representative of each slice
    std::vector<int> reps;                      // distinct representatives
    std::vector<int4> bp, proj, tr, px, sn, ch; // all slices (ch: Chambolle tiles of chK fused steps)
    std::vector<int4> chf;                      // tiles of the last Chambolle launch (chK + 1 steps of halo)
    std::vector<int4> bp_r, proj_r, tr_r, px_r, sn_r;   // representatives only
    std::vector<size_t> img_off, sino_off;      // per slice, in floats
    size_t img_total = 0, sino_total = 0;
    std::vector<int> px_first, sn_first;
    // projector items grouped by staging width (256, 384, 512 columns; each
    // slice uses the width of its single-slice solve): counts per group
    int proj_cnt[3] = {0, 0, 0}, proj_r_cnt[3] = {0, 0, 0};
    int chK = 5;     // Chambolle steps fused per launch (tuned for the largest slice)
    int bpNA = 16;   // back-projector angles per block (tuned for the geometry with the most updates)
};

size_t up4(size_t v) { return (v + 63) / 64 * 64; }   // 256-byte multiples of floats

void add_items(Plan &P, int s, const pyhst_geometry &g, bool rep_only) {
    int tx, ty;
    bp_tiles(g.nx, g.ny, &tx, &ty);
    auto &bp = rep_only ? P.bp_r : P.bp;
    for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) bp.push_back(make_int4(s, x, y, 0));
    if (rep_only) {   // the power iteration projects one slice per geometry (the pairs: make_plan)
        int nb, na;
        proj_blocks(g.n_angles, g.n_bins, &nb, &na);
        for (int a = 0; a < na; ++a)
            for (int b = 0; b < nb; ++b) P.proj_r.push_back(make_int4(s, b, a, s));
    }
    auto &tr = rep_only ? P.tr_r : P.tr;
    for (int y = 0; y < (g.ny + 63) / 64; ++y)     // the projector's transpose moves 64 x 64 tiles
        for (int x = 0; x < (g.nx + 63) / 64; ++x) tr.push_back(make_int4(s, x, y, 0));
    auto &px = rep_only ? P.px_r : P.px;
    for (int y = 0; y < (g.ny + kPxRows - 1) / kPxRows; ++y)
        for (int x = 0; x < (g.nx + 31) / 32; ++x) px.push_back(make_int4(s, x, y, 0));
    auto &sn = rep_only ? P.sn_r : P.sn;
    const int M = g.n_angles * g.n_bins;
    for (int e = 0; e < (M + kSinoBlock - 1) / kSinoBlock; ++e) sn.push_back(make_int4(s, e, 0, 0));
    if (!rep_only) {
        const int h0 = chambolle_tile_h(P.chK), w0 = chambolle_tile_w(P.chK);
        const int h1 = chambolle_tile_h(P.chK + 1), w1 = chambolle_tile_w(P.chK + 1);
        for (int y = 0; y < (g.ny + h0 - 1) / h0; ++y)
            for (int x = 0; x < (g.nx + w0 - 1) / w0; ++x) P.ch.push_back(make_int4(s, x, y, 0));
        for (int y = 0; y < (g.ny + h1 - 1) / h1; ++y)
            for (int x = 0; x < (g.nx + w1 - 1) / w1; ++x) P.chf.push_back(make_int4(s, x, y, 0));
    }
}

Plan make_plan(const pyhst_tv_item *items, int n) {
    Plan P;
    P.n = n;
    int big = 0;
    for (int s = 1; s < n; ++s)
        if ((long)items[s].geom.nx * items[s].geom.ny > (long)items[big].geom.nx * items[big].geom.ny) big = s;
    P.chK = chambolle_k_for(items[big].geom.nx, items[big].geom.ny);
    {   // the back-projector's angle block: that of the geometry (size, angle count) with the most updates
        std::map<std::tuple<int, int, int>, double> work;
        for (int s = 0; s < n; ++s) {
            const pyhst_geometry &g = items[s].geom;
            work[std::make_tuple(g.nx, g.ny, g.n_angles)] += (double)g.nx * g.ny * g.n_angles;
        }
        auto top = std::max_element(work.begin(), work.end(),
                                    [](const auto &a, const auto &b) { return a.second < b.second; });
        P.bpNA = bp_block_for(std::get<0>(top->first), std::get<1>(top->first), std::get<2>(top->first));
    }
    P.rep.resize(n);
    std::map<std::tuple<const void *, const void *, int, int, int, int, float, float, float>, int> groups;
    for (int s = 0; s < n; ++s) {
        const pyhst_geometry &g = items[s].geom;
        auto key = std::make_tuple((const void *)g.angles, (const void *)g.axis, g.n_angles, g.n_bins, g.nx, g.ny,
                                   g.cx, g.cy, g.pixel_size);
        auto f = groups.find(key);
        if (f == groups.end()) {
            groups[key] = s;
            P.rep[s] = s;
            P.reps.push_back(s);
        } else {
            P.rep[s] = f->second;
        }
        P.img_off.push_back(P.img_total);
        P.img_total += up4((size_t)g.nx * g.ny);
        P.sino_off.push_back(P.sino_total);
        P.sino_total += up4((size_t)g.n_angles * g.n_bins);
        P.px_first.push_back((int)P.px.size());
        P.sn_first.push_back((int)P.sn.size());
        add_items(P, s, g, false);
    }
    for (int r : P.reps) add_items(P, r, items[r].geom, true);
    // projector items: each CTA walks two slices of one geometry (items[k].x
    // and items[k].w), paired in list order within the geometry; an odd one
    // out is paired with itself
    {
        std::map<int, std::vector<int>> members;
        for (int s = 0; s < n; ++s) members[P.rep[s]].push_back(s);
        for (int r : P.reps) {
            const std::vector<int> &m = members[r];
            int nb, na;
            proj_blocks(items[r].geom.n_angles, items[r].geom.n_bins, &nb, &na);
            for (size_t q = 0; q < m.size(); q += 2) {
                const int s0 = m[q], s1 = q + 1 < m.size() ? m[q + 1] : m[q];
                for (int a = 0; a < na; ++a)
                    for (int b = 0; b < nb; ++b) P.proj.push_back(make_int4(s0, b, a, s1));
            }
        }
    }
    auto width_group = [&](const int4 &it) {
        const pyhst_geometry &g = items[it.x].geom;
        const int w = project_width(g.nx, g.ny, g.n_angles);
        return w == 256 ? 0 : (w == 384 ? 1 : 2);
    };
    for (auto *v : {&P.proj, &P.proj_r}) {
        std::vector<int> grp(v->size());
        for (size_t q = 0; q < v->size(); ++q) grp[q] = width_group((*v)[q]);
        std::vector<size_t> ord(v->size());
        for (size_t q = 0; q < ord.size(); ++q) ord[q] = q;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return grp[a] < grp[b]; });
        std::vector<int4> sorted(v->size());
        int *cnt = v == &P.proj ? P.proj_cnt : P.proj_r_cnt;
        for (size_t q = 0; q < ord.size(); ++q) {
            sorted[q] = (*v)[ord[q]];
            ++cnt[grp[ord[q]]];
        }
        v->swap(sorted);
    }
    // Longest items first: CTAs start roughly in list order, so the long
    // items of the large slices run early and the short ones fill the last
    // wave.  A CTA's result does not depend on its place in the list.
    auto longest_first = [](std::vector<int4>::iterator b, std::vector<int4>::iterator e, auto cost) {
        std::stable_sort(b, e, [&](const int4 &u, const int4 &v) { return cost(u) > cost(v); });
    };
    auto bp_cost = [&](const int4 &it) { return items[it.x].geom.n_angles; };       // angles per output tile
    auto proj_cost = [&](const int4 &it) {                                           // rows walked per ray
        return std::max(items[it.x].geom.nx, items[it.x].geom.ny);
    };
    longest_first(P.bp.begin(), P.bp.end(), bp_cost);
    longest_first(P.bp_r.begin(), P.bp_r.end(), bp_cost);
    for (int k = 0, o = 0, orr = 0; k < 3; o += P.proj_cnt[k], orr += P.proj_r_cnt[k], ++k) {
        longest_first(P.proj.begin() + o, P.proj.begin() + o + P.proj_cnt[k], proj_cost);
        longest_first(P.proj_r.begin() + orr, P.proj_r.begin() + orr + P.proj_r_cnt[k], proj_cost);
    }
    return P;
}

struct Layout {
    size_t desc_even, desc_odd, desc_init, desc_pow, tvs, reps, items, tabs, imgs, sinos, scal, part_px, part_sn,
        part_gap, bytes;
    size_t n_items_total;
    std::vector<size_t> tab_off;
};

Layout make_layout(const Plan &P, const pyhst_tv_item *items) {
    Layout l{};
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    l.desc_even = take(sizeof(BatchSlice) * P.n);
    l.desc_odd = take(sizeof(BatchSlice) * P.n);
    l.desc_init = take(sizeof(BatchSlice) * P.n);
    l.desc_pow = take(sizeof(BatchSlice) * P.n);
    l.tvs = take(sizeof(TvSlice) * P.n);
    l.reps = take(sizeof(int) * P.reps.size());
    l.n_items_total = P.bp.size() + P.proj.size() + P.tr.size() + P.px.size() + P.sn.size() + P.ch.size() +
                      P.chf.size() +
                      P.bp_r.size() +
                      P.proj_r.size() + P.tr_r.size() + P.px_r.size() + P.sn_r.size();
    l.items = take(sizeof(int4) * l.n_items_total);
    for (int s = 0; s < P.n; ++s) l.tab_off.push_back(take(sizeof(AngleInfo) * items[s].geom.n_angles));
    l.imgs = take(sizeof(float) * P.img_total * 10);
    l.sinos = take(sizeof(float) * P.sino_total * 3);
    l.scal = take(sizeof(double) * P.n * 2 + sizeof(float) * P.n * 3);
    l.part_px = take(sizeof(double) * P.px.size());
    l.part_sn = take(sizeof(double) * P.sn.size());
    l.part_gap = take(sizeof(double) * P.px.size());
    l.bytes = off;
    return l;
}

int check_items(const pyhst_tv_item *items, int n) {
    if (!items || n < 1) return fail(PYHST_ERR_INVALID_ARG, "need at least one batch item");
    for (int s = 0; s < n; ++s) {
        pyhst_geometry g = items[s].geom;
        g.n_slices = 1;
        int rc = check_geometry(&g);
        if (rc) {
            char inner[512];   // the message is formatted into the same per-thread buffer
            snprintf(inner, sizeof inner, "%s", pyhst_last_error());
            return fail(rc, "item %d: %s", s, inner);
        }
        if (!items[s].sino || !items[s].x) return fail(PYHST_ERR_INVALID_ARG, "item %d: sino/x pointer is NULL", s);
        if (!std::isfinite(items[s].beta)) return fail(PYHST_ERR_INVALID_ARG, "item %d: beta is not finite", s);
    }
    return PYHST_OK;
}

int check_tv_opts_b(const pyhst_tv_opts *o) {
    if (!o) return fail(PYHST_ERR_INVALID_ARG, "options are NULL");
    if (!(o->beta >= 0.0f) || !std::isfinite(o->beta)) return fail(PYHST_ERR_INVALID_ARG, "beta must be >= 0");
    if (o->n_iter < 1) return fail(PYHST_ERR_INVALID_ARG, "n_iter must be >= 1");
    if (o->n_inner < 1) return fail(PYHST_ERR_INVALID_ARG, "n_inner must be >= 1");
    if (!(o->tau > 0.0f && o->tau <= 0.25f)) return fail(PYHST_ERR_INVALID_ARG, "tau must be in (0, 1/4]");
    if (!(o->lipschitz >= 0.0) || !std::isfinite(o->lipschitz))
        return fail(PYHST_ERR_INVALID_ARG, "lipschitz must be >= 0 (0: estimate)");
    if (o->lipschitz == 0.0 && o->n_power_iter < 1)
        return fail(PYHST_ERR_INVALID_ARG, "n_power_iter must be >= 1 when lipschitz is estimated");
    if (o->warm_dual != 0 && o->warm_dual != 1) return fail(PYHST_ERR_INVALID_ARG, "warm_dual must be 0 or 1");
    return PYHST_OK;
}

}  // namespace
}  // namespace pyhst

using namespace pyhst;

extern "C" size_t pyhst_tv_batch_workspace_size(const pyhst_tv_item *items, int32_t n_items,
                                                const pyhst_tv_opts *opts) {
    (void)opts;
    if (!items || n_items < 1) return 0;
    for (int s = 0; s < n_items; ++s) {
        const pyhst_geometry &g = items[s].geom;
        if (g.n_angles < 1 || g.n_bins < 1 || g.nx < 1 || g.ny < 1) return 0;
    }
    Plan P = make_plan(items, n_items);
    return make_layout(P, items).bytes;
}

extern "C" int pyhst_tv_solve_batch(const pyhst_tv_item *items, int32_t n_items, const pyhst_tv_opts *opts,
                                    double *lipschitz_out, void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    int rc = check_items(items, n_items);
    if (rc) return rc;
    if ((rc = check_tv_opts_b(opts))) return rc;
    const Plan P = make_plan(items, n_items);
    const Layout L = make_layout(P, items);
    if (!workspace || ws_bytes < L.bytes || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", L.bytes);
    if (P.px.size() > 0x7fffffff || P.bp.size() > 0x7fffffff)
        return fail(PYHST_ERR_INVALID_ARG, "batch too large");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const int n = n_items;

    // ---- host tables
    float *imgs = reinterpret_cast<float *>(ws + L.imgs);
    float *sinos = reinterpret_cast<float *>(ws + L.sinos);
    const size_t IT = P.img_total, ST = P.sino_total;
    auto img = [&](int t, int s) { return imgs + (size_t)t * IT + P.img_off[s]; };
    auto sin = [&](int t, int s) { return sinos + (size_t)t * ST + P.sino_off[s]; };
    std::vector<TvSlice> tv(n);
    std::vector<BatchSlice> ev(n), od(n), in(n), pw(n);
    for (int s = 0; s < n; ++s) {
        const pyhst_geometry &g = items[s].geom;
        TvSlice &t = tv[s];
        t.y = img(0, s); t.xa = img(1, s); t.xb = img(2, s); t.z = img(3, s); t.g = img(4, s);
        t.p1a = img(5, s); t.p2a = img(6, s); t.p1b = img(7, s); t.p2b = img(8, s);
        t.Axa = sin(0, s); t.Axb = sin(1, s); t.Ry = sin(2, s);
        t.sino = items[s].sino;
        t.x_user = items[s].x;
        t.energy = items[s].energy;
        t.gap = items[s].gap;
        t.nx = g.nx; t.ny = g.ny; t.M = g.n_angles * g.n_bins;
        t.px_first = P.px_first[s];
        t.sn_first = P.sn_first[s];
        t.rep = P.rep[s];
        t.beta = (items[s].beta >= 0.0f) ? items[s].beta : opts->beta;
        BatchSlice b{};
        b.tab = reinterpret_cast<const AngleInfo *>(ws + L.tab_off[s]);
        b.n_angles = g.n_angles; b.n_bins = g.n_bins; b.nx = g.nx; b.ny = g.ny;
        b.cx = g.cx; b.cy = g.cy; b.pixel_size = g.pixel_size;
        b.proj_inT = img(9, s);
        b.proj_nseg = proj_segments(&g);
        // gradient back-projection of the residual P y - sino (formed by the update kernels)
        b.bp_a = t.Ry; b.bp_b = nullptr; b.bp_out = t.g;
        ev[s] = b; ev[s].proj_in = t.xb; ev[s].proj_out = t.Axb;   // even iterations write xb, Axb
        od[s] = b; od[s].proj_in = t.xa; od[s].proj_out = t.Axa;   // odd iterations write xa, Axa
        // the iterations' back-projection ends in the gradient step z = y - invL g
        const float *invL_s = reinterpret_cast<const float *>(reinterpret_cast<double *>(ws + L.scal) + 2 * n) + s;
        for (BatchSlice *e : {&ev[s], &od[s]}) {
            e->bp_out = t.z;
            e->bp_y = t.y;
            e->bp_invL = invL_s;
        }
        in[s] = b; in[s].proj_in = t.xa; in[s].proj_out = t.Axa;   // warm start
        pw[s] = b; pw[s].proj_in = t.z; pw[s].proj_out = t.Axa;    // power iteration
        pw[s].bp_a = t.Axa; pw[s].bp_b = nullptr;
    }
    std::vector<int4> all;
    auto append = [&](const std::vector<int4> &v) { size_t o = all.size(); all.insert(all.end(), v.begin(), v.end()); return o; };
    const size_t o_bp = append(P.bp), o_proj = append(P.proj), o_tr = append(P.tr), o_px = append(P.px),
                 o_sn = append(P.sn), o_ch = append(P.ch), o_chf = append(P.chf), o_bpr = append(P.bp_r), o_projr = append(P.proj_r), o_trr = append(P.tr_r),
                 o_pxr = append(P.px_r), o_snr = append(P.sn_r);
    // pageable host memory: each copy returns once its data are staged
    cudaMemcpyAsync(ws + L.desc_even, ev.data(), sizeof(BatchSlice) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ws + L.desc_odd, od.data(), sizeof(BatchSlice) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ws + L.desc_init, in.data(), sizeof(BatchSlice) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ws + L.desc_pow, pw.data(), sizeof(BatchSlice) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ws + L.tvs, tv.data(), sizeof(TvSlice) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ws + L.reps, P.reps.data(), sizeof(int) * P.reps.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ws + L.items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice, st);
    if ((rc = cuda_status("batch table upload"))) return rc;
    for (int s = 0; s < n; ++s)
        if ((rc = launch_angle_table(items[s].geom.angles, items[s].geom.axis, items[s].geom.n_angles,
                                     reinterpret_cast<AngleInfo *>(ws + L.tab_off[s]), st)))
            return rc;

    const BatchSlice *D_even = reinterpret_cast<const BatchSlice *>(ws + L.desc_even);
    const BatchSlice *D_odd = reinterpret_cast<const BatchSlice *>(ws + L.desc_odd);
    const BatchSlice *D_init = reinterpret_cast<const BatchSlice *>(ws + L.desc_init);
    const BatchSlice *D_pow = reinterpret_cast<const BatchSlice *>(ws + L.desc_pow);
    const TvSlice *T = reinterpret_cast<const TvSlice *>(ws + L.tvs);
    const int *R = reinterpret_cast<const int *>(ws + L.reps);
    const int4 *I = reinterpret_cast<const int4 *>(ws + L.items);
    double *sc_base = reinterpret_cast<double *>(ws + L.scal);
    Scal sc;
    sc.L = sc_base;
    sc.ray = sc_base + n;
    sc.invL = reinterpret_cast<float *>(sc_base + 2 * n);
    sc.lam = sc.invL + n;
    sc.invn = sc.lam + n;
    double *part_px = reinterpret_cast<double *>(ws + L.part_px);
    double *part_sn = reinterpret_cast<double *>(ws + L.part_sn);
    double *part_gap = reinterpret_cast<double *>(ws + L.part_gap);
    bool any_gap = false;
    for (int q = 0; q < n; ++q) any_gap = any_gap || items[q].gap != nullptr;
    const int Lch = chambolle_launches(opts->n_inner, P.chK);
    const int npx = (int)P.px.size(), nsn = (int)P.sn.size(), nbp = (int)P.bp.size(), npr = (int)P.proj.size(),
              ntr = (int)P.tr.size(), nch = (int)P.ch.size(), nchf = (int)P.chf.size();
    const dim3 tb(kBT);

    // ---- step size: power iteration on the representatives, or the caller's L
    if ((rc = set_proj_attr())) return rc;
    // projector: the transposes, then the items of each staging width (256, 384, 512 columns)
    // (ns: slices per projector CTA, 2 for the pairs of the solve, 1 for the
    // power iteration's one slice per geometry)
    auto project = [&](const BatchSlice *D, size_t o_items, const int *cnt, size_t o_tr, int n_tr, int ns) {
        int r = launch_project_batch(D, I + o_items, cnt[0], I + o_tr, n_tr, 256, st, ns);
        if (!r) r = launch_project_batch(D, I + o_items + cnt[0], cnt[1], nullptr, 0, 384, st, ns);
        if (!r) r = launch_project_batch(D, I + o_items + cnt[0] + cnt[1], cnt[2], nullptr, 0, 512, st, ns);
        return r;
    };
    if (opts->lipschitz == 0.0) {
        const int npxr = (int)P.px_r.size(), nsnr = (int)P.sn_r.size();
        b_fill_v<<<npxr, tb, 0, st>>>(T, I + o_pxr);
        for (int it = 0; it < opts->n_power_iter; ++it) {
            if ((rc = project(D_pow, o_projr, P.proj_r_cnt, o_trr, (int)P.tr_r.size(), 1)))
                return rc;
            if ((rc = launch_backproject_batch(D_pow, I + o_bpr, (int)P.bp_r.size(), false, st, P.bpNA))) return rc;
            b_sqnorm_g<<<npxr, tb, 0, st>>>(T, I + o_pxr, part_px);
            b_finalize_norm<<<(int)P.reps.size(), tb, 0, st>>>(T, R, part_px, sc, 0);
            b_scale_v<<<npxr, tb, 0, st>>>(T, I + o_pxr, sc);
        }
        if ((rc = project(D_pow, o_projr, P.proj_r_cnt, o_trr, (int)P.tr_r.size(), 1)))
            return rc;
        b_sqnorm_axa<<<nsnr, tb, 0, st>>>(T, I + o_snr, part_sn);
        b_finalize_norm<<<(int)P.reps.size(), tb, 0, st>>>(T, R, part_sn, sc, 1);
    }
    b_set_step<<<(n + 127) / 128, 128, 0, st>>>(T, sc, opts->lipschitz, n);
    if ((rc = cuda_status("step-size kernels"))) return rc;
    if (lipschitz_out) cudaMemcpyAsync(lipschitz_out, sc.L, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);

    // ---- start
    b_copy_x<<<npx, tb, 0, st>>>(T, I + o_px, opts->warm_start ? 1 : 0, 0);
    if (opts->warm_start)
        if ((rc = project(D_init, o_proj, P.proj_cnt, o_tr, ntr, 2))) return rc;
    b_copy_sino_start<<<nsn, tb, 0, st>>>(T, I + o_sn, opts->warm_start ? 1 : 0);
    if ((rc = cuda_status("batch start"))) return rc;

    if ((rc = b_chambolle_attr(P.chK))) return rc;
    // ---- the iterations, captured in one graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    // the legacy default stream cannot be captured: launch directly there
    const bool own_graph = cap == cudaStreamCaptureStatusNone && st != nullptr;
    if (own_graph && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_status("graph capture begin");
    double t = 1.0;
    bool dual_a = true;     // where the last prox left its dual field
    bool identity = true;   // no slice has a TV term: skip the Chambolle steps
    for (int q = 0; q < n; ++q) identity = identity && tv[q].beta == 0.0f;
    for (int k = 0; k < opts->n_iter && !rc; ++k) {
        const int par = k & 1;   // 0: x_new -> xb, 1: x_new -> xa
        rc = launch_backproject_batch(D_even, I + o_bp, nbp, false, st, P.bpNA);
        if (rc) break;
        if (!identity) {                        // the last Chambolle launch writes x_new
            // warm_dual: after the first prox, start from the field the previous
            // one kept (parity index 1 reads the a buffers, 2 the b buffers)
            const int q0 = (opts->warm_dual && k > 0) ? (dual_a ? 1 : 2) : 0;
            const int pa_final = ((q0 + Lch - 1) & 1) == 0;
            rc = b_chambolle_launches(P.chK, nch, T, I + o_ch, nchf, I + o_chf, sc, opts->tau, opts->n_inner, par,
                                      opts->warm_dual ? 2 : (any_gap ? 1 : 0), q0, st);
            if (rc) break;
            dual_a = pa_final;
            if (any_gap) b_gap_partial<<<npx, tb, 0, st>>>(T, I + o_px, par, pa_final, part_gap);
        } else {
            b_prox_final<<<npx, tb, 0, st>>>(T, I + o_px, sc, 0, par, 1);
        }
        if (any_gap) b_finalize_gap<<<n, tb, 0, st>>>(T, part_gap, sc, k);
        rc = project(par ? D_odd : D_even, o_proj, P.proj_cnt, o_tr, ntr, 2);
        if (rc) break;
        double w = 0.0;
        if (opts->use_fista) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            w = (t - 1.0) / tn;
            t = tn;
        }
        b_sino_update<<<nsn, tb, 0, st>>>(T, I + o_sn, (float)w, par, part_sn);
        b_image_update<<<npx, tb, 0, st>>>(T, I + o_px, (float)w, par, part_px);
        b_finalize_energy<<<n, tb, 0, st>>>(T, part_sn, part_px, opts->n_iter, k, n);
        rc = cuda_status("batch iteration kernels");
    }
    if (own_graph) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(PYHST_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(PYHST_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        e = cudaGraphLaunch(exec, st);
        cudaGraphExecDestroy(exec);   // released once the launched graph completes
        if (e != cudaSuccess) return fail(PYHST_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    } else if (rc) {
        return rc;
    }
    // ---- result: the last iterate
    b_copy_x<<<npx, tb, 0, st>>>(T, I + o_px, 2, (opts->n_iter - 1) & 1);
    return cuda_status("batch result copy");
}
