// Forward projector: the exact transpose of the unweighted back-projector,
//   sino[a][b] = scale * sum_{i,j} img[i][j] * max(0, 1 - |t_a(i, j) - b|),
// the operator P the iterative methods apply at every iteration (Sec. 2.3,
// last paragraph; Eq. 1 and Eq. 3).
//
// The paper keeps the volume in a texture.  Here the projector is ray-driven
// and deterministic (no atomics).  For an angle whose |cos| >= |sin| a ray
// walks the image rows; on row i the hat weight of pixel j is
// 1 - |cos| * |j - x*(i)|, x*(i) being the column where t = b, so at most
// three pixels per row are non-zero.  For |sin| > |cos| the same walk runs over
// the rows of a transposed copy of the image.
//
// A CTA takes a group of 8 consecutive angles and 128 consecutive bins (1024
// rays, 4 per thread).  A warp holds 16 consecutive bins of two neighbouring
// angles, so the pixels its lanes read in one row span at most ~26 words of
// shared memory (one wavefront per load).  The CTA walks its array in blocks
// of 32 rows (256-column staging) or 16 rows (384 or 512 columns); for each
// block it stages the rectangle of pixels that its rays can touch (for
// neighbouring angles their bands nearly coincide, so one staged pixel serves
// about eight times more rays than a one-angle band would); only the columns
// of the band are loaded.  The next block is copied from L2 into the other
// half of a double buffer by asynchronous 16-byte copies (cp.async, no
// registers held) while the current one is walked, with one barrier per
// block.  The staging buffer holds up to 512 columns, enough for the 8-angle
// bands of sparse angle sets (150 angles at 2048^2); if a group's band still
// does not fit, the CTA walks 4, 2 or 1 angles at a time; the band width is
// convex in the row, so checking the first and last blocks decides it.
// When the grid would have few CTAs (few angles, few slices) the rows are
// split into segments whose partial sinograms are added in a fixed order.
// Otherwise a CTA walks two slices of one geometry at once (two slices of a
// stack, or two batch slices that share the geometry): each slice has its own
// staged plane, while the ray positions, hat weights, bands and copies'
// index arithmetic are computed once for both; the taps of both slices are
// added by the same paired fmas a one-slice walk uses, so each slice gets
// the bits of its one-slice projection.  Half the rows per staged block keep
// the double buffer at 64 KB.
//
// x*(b, r) = X0 + b dX - r rho is computed in 32.32 fixed point (int64), so the
// staged bands, computed with the same integers, provably contain every tap
// (with one column to spare on each side).  Inside a 32-row chunk each ray
// follows x* - L0 (L0: the first staged column of the current block) in
// unsigned 9.23 fixed point (every band width), re-anchored exactly at every
// chunk and moved by whole columns between a chunk's two blocks, so a row
// costs one integer add and the error stays below 2e-6 pixel (31 steps
// rounded by at most 2^-24 each, plus the anchor's truncation below 2^-23);
// the fraction becomes a float by placing its bits in a mantissa.  Pairs of
// rays share paired float32 (f32x2) arithmetic.
// Rays that do not take part in a pass get zero weights and a fixed in-range
// position, so the walk has no branches.  The weights
// of the taps jc-1, jc, jc+1 (jc = round(x*), psi = x* - jc in [-1/2, 1/2)) are
// sat(1 - a - a psi), 1 - a |psi|, sat(1 - a + a psi) with a = |cos| (or |sin|);
// no fourth pixel can have a non-zero weight since a >= 1/sqrt(2).
#include <climits>
#include <cmath>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kPThreads = 256;
constexpr int kPG = 8;          // angles per group
constexpr int kPB = 128;        // bins per CTA
constexpr int kPR = 32;         // rows per chunk (the unit of re-anchoring, clipping and row segments)
// Staged pixels per row (band capacity): 256 for dense angle sets, 512 for
// sparse ones (image size / number of angles > 2), chosen per launch.
constexpr int kPRays = kPG / 2; // rays per thread
// Rows per staged block: a whole chunk for the 256-column staging (whose
// double buffer then still allows 3 CTAs per SM), half a chunk for the wider
// ones, and half that again when a CTA walks NS = 2 slices of one geometry
// (one staged plane per slice, the same 64 KB).  The arithmetic is per chunk,
// so the bits do not depend on it.
template <int PW, int NS = 1> __host__ __device__ constexpr int prows() { return (PW == 256 ? kPR : kPR / 2) / NS; }
template <int PW, int NS = 1> __host__ __device__ constexpr int pvec() {      // copies per thread per block and plane
    return prows<PW, NS>() * PW / 4 / kPThreads;
}
template <int PW, int NS = 1> __host__ __device__ constexpr int psmem() {     // double-buffered strips
    return 2 * NS * prows<PW, NS>() * PW * (int)sizeof(float);
}
constexpr int kPTargetCtas = 148 * 3 * 4;   // below this, the rows are split into segments
constexpr int kPBandWin = 128;              // chunks whose bands are computed at once (1 KB of shared memory)
constexpr double kFix = 4294967296.0;   // 2^32

// out = in^T for the 64 x 64 tile at (r0, c0) of a rows x cols array, by 32 x 8
// threads (16 elements each; rows of 65 floats: conflict-free both ways)
constexpr int kTT = 64;
__device__ __forceinline__ void transpose_tile(const float *__restrict__ in, float *__restrict__ out, int rows,
                                               int cols, int r0, int c0) {
    __shared__ float tile[kTT][kTT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int k = ty; k < kTT; k += 8)
#pragma unroll
        for (int h = 0; h < kTT; h += 32) {
            const int r = r0 + k, c = c0 + tx + h;
            if (r < rows && c < cols) tile[k][tx + h] = in[(size_t)r * cols + c];
        }
    __syncthreads();
#pragma unroll
    for (int k = ty; k < kTT; k += 8)
#pragma unroll
        for (int h = 0; h < kTT; h += 32) {
            const int c = c0 + k, r = r0 + tx + h;
            if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[tx + h][k];
        }
}

__global__ void transpose_kernel(const float *__restrict__ in, float *__restrict__ out, int rows,
                                 int cols) {
    const size_t off = (size_t)blockIdx.z * rows * cols;
    transpose_tile(in + off, out + off, rows, cols, blockIdx.y * kTT, blockIdx.x * kTT);
}

// One angle's walk over a row-major [R][C] array (image rows when |cos| >=
// |sin|, transposed rows otherwise): x*(b, r) = X0 + b dX - r rho in 32.32.
struct RayGeom {
    long long X0, dX, rho;
    float a;        // |cc|
    int major;      // 0: image rows, 1: transposed rows, -1: no contribution
};

__device__ RayGeom ray_geom(const AngleInfo &e, double cx, double cy) {
    RayGeom g;
    g.major = -1;
    g.X0 = g.dX = g.rho = 0;
    g.a = 0.0f;
    if (!(isfinite(e.c) && isfinite(e.s) && isfinite(e.axis))) return g;
    const bool xm = fabs(e.c) >= fabs(e.s);
    const double cc = xm ? e.c : e.s, rr = xm ? e.s : e.c;
    const double ccen = xm ? cx : cy, rcen = xm ? cy : cx;
    if (cc == 0.0) return g;
    const double X0 = ccen + (rcen * rr - e.axis) / cc;
    if (!(fabs(X0) < 1.0e9)) return g;          // rays that miss any image
    g.X0 = llrint(X0 * kFix);
    g.dX = llrint(kFix / cc);
    g.rho = llrint(rr / cc * kFix);
    g.a = (float)fabs(cc);
    g.major = xm ? 0 : 1;
    return g;
}

__device__ __forceinline__ int hi32(long long v) { return (int)(v >> 32); }

// Band of a chunk: columns [L0, H] covering every tap of the rays of the
// masked angles between rows r_first and r_last (warp 0; result in lane 0).
__device__ __forceinline__ void chunk_band(const RayGeom *rg, int mask, int b0, int bhi, int r_first, int r_last,
                                           int &L0, int &H) {
    const int lane = threadIdx.x & 31;
    int lo = INT_MAX, hi = INT_MIN;
    if (lane < kPG && ((mask >> lane) & 1)) {
        const RayGeom g = rg[lane];
        const long long p = g.X0 + (long long)b0 * g.dX, q = g.X0 + (long long)bhi * g.dX;
        const long long u = (long long)r_first * g.rho, v = (long long)r_last * g.rho;
        const long long mn = min(min(p - u, q - u), min(p - v, q - v));
        const long long mx = max(max(p - u, q - u), max(p - v, q - v));
        lo = hi32(mn) - 2;
        hi = hi32(mx) + 3;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    L0 = lo & ~3;   // float4-aligned start
    H = hi;
}

// Chunks [out[0], out[1]) outside of which no ray of the masked angles has a
// tap inside the array's columns [0, C) (warp 0; result in lane 0): on the
// rows outside, every tap reads a zero staged outside the image and adds an
// exact zero, so skipping them changes no bits.  The range is widened by
// margins (3 columns, 2 rows, one chunk), never narrowed.
__device__ __forceinline__ void chunk_clip(const RayGeom *rg, int mask, int b0, int bhi, int R, int C, int *out) {
    const int lane = threadIdx.x & 31;
    int lo = INT_MAX, hi = INT_MIN;
    if (lane < kPG && ((mask >> lane) & 1)) {
        const RayGeom g = rg[lane];
        // x*(b, r) = A_b - r rho over the bins b0 .. bhi: its extremes are at the end bins
        const double A0 = (double)(g.X0 + (long long)b0 * g.dX) / kFix;
        const double A1 = (double)(g.X0 + (long long)bhi * g.dX) / kFix;
        const double rho = (double)g.rho / kFix, amax = fmax(A0, A1), amin = fmin(A0, A1);
        double rl = 0.0, rh = (double)(R - 1);
        if (rho > 0.0) {
            rh = fmin(rh, (amax + 3.0) / rho);
            rl = fmax(rl, (amin - C - 2.0) / rho);
        } else if (rho < 0.0) {
            rl = fmax(rl, (amax + 3.0) / rho);
            rh = fmin(rh, (amin - C - 2.0) / rho);
        } else if (amax < -3.0 || amin > C + 2.0) {
            rl = 1.0;
            rh = 0.0;
        }
        if (rl <= rh) {
            lo = (int)floor(rl) - 2;
            hi = (int)ceil(rh) + 2;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        const int nch = (R + kPR - 1) / kPR;
        out[0] = lo == INT_MAX ? 0 : max(0, lo / kPR);
        out[1] = hi == INT_MIN ? 0 : min(nch, hi / kPR + 1);
    }
}

struct WalkArgs {
    const float *M[2];  // the walked array of each slice (M[0] only for one slice)
    int R, C;
    int b0, bhi, b;
    bool vec;       // float4 staging allowed (16-byte aligned rows)
};

// Walk the chunks [c_lo, c_hi) of one array for the rays of the masked
// angles, staged in blocks of prows rows (one to four per chunk).  Only the
// band of each block is staged.  The bands of up to kPBandWin blocks are
// computed at once by all threads (the same integer bounds as chunk_band)
// before those blocks are walked.  With kNS = 2 the same rays walk two
// slices of one geometry at once: one staged plane per slice, the positions
// and weights computed once for both, and each slice's sums formed exactly
// as a one-slice walk forms them (the same bits).
template <int kPW, int kNS>
__device__ __forceinline__ void walk_pass(const WalkArgs &w, const RayGeom *rg, int mask, float2 (&acc)[kNS][2],
                                          float2 (*tot)[kPThreads], float scale, int per,
                                          float (*strip)[kNS][prows<kPW, kNS>()][kPW], int2 *bands, int c_lo,
                                          int c_hi) {
    constexpr int kPVec = pvec<kPW, kNS>(), kRows = prows<kPW, kNS>(), kSub = kPR / kRows;   // kSub blocks per chunk
    constexpr int kPlane = kRows * kPW;                    // floats between two slices' staged rows
    constexpr int kFrac = 23;
    const int tid = threadIdx.x, lane = tid & 31;
    const int asub = lane >> 4;
    if (c_hi <= c_lo) return;
    const int row0 = c_lo * kPR, r_end = min(w.R, c_hi * kPR);   // rows of this pass
    const int n_blocks = (r_end - row0 + kRows - 1) / kRows;       // block k: rows row0 + k kRows, ...
    long long X64[kPRays];          // x* + 1/2 at row 0, 32.32
    float aa[kPRays], m1[kPRays], t1[kPRays], c1[kPRays];
    unsigned r32[kPRays];           // rho in 9.23 fixed point (0: ray not in this pass)
    bool act[kPRays];
#pragma unroll
    for (int k = 0; k < kPRays; ++k) {
        const RayGeom g = rg[asub + 2 * k];
        act[k] = ((mask >> (asub + 2 * k)) & 1) && w.b <= w.bhi;
        X64[k] = g.X0 + (long long)w.b * g.dX + (1LL << 31);
        aa[k] = act[k] ? g.a : 0.0f;          // inactive: all three weights 0
        m1[k] = -1.5f * aa[k];
        t1[k] = act[k] ? 1.0f - g.a : -1.0f;
        c1[k] = act[k] ? 1.0f : 0.0f;
        r32[k] = act[k] ? (unsigned)(int)((g.rho + (1LL << (31 - kFrac))) >> (32 - kFrac)) : 0u;
    }
    int win0 = 0;                          // first block of the current band window
    // block k -> strip[sbuf], band columns only, by asynchronous copies
    // (a source size of 0 fills zeros outside the array); completed by the
    // wait before the next barrier
    auto load = [&](int k, int sbuf) {
        const int2 bd = bands[k - win0];
        const int r0 = row0 + k * kRows, nr = min(kRows, r_end - r0), L0 = bd.x & ~3, width = bd.y - L0 + 4;
        // one copy of 16 (or 4 x 4) bytes into every slice's plane; a source
        // size of 0 (outside the array or past the pass's rows) writes zeros
        auto copy16 = [&](uint32_t dst, size_t off, bool in) {
#pragma unroll
            for (int q = 0; q < kNS; ++q)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst + q * kPlane * 4),
                             "l"(in ? w.M[q] + off : w.M[0]), "r"(in ? 16u : 0u) : "memory");
        };
        auto copy4x4 = [&](uint32_t dst, size_t off, int j, bool row_in) {
#pragma unroll
            for (int q = 0; q < kNS; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool in = row_in && (unsigned)(j + e) < (unsigned)w.C;
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + q * kPlane * 4 + 4 * e),
                                 "l"(in ? w.M[q] + off + e : w.M[0]), "r"(in ? 4u : 0u) : "memory");
                }
        };
        if constexpr ((4 * kPThreads) % kPW == 0) {
            // a thread copies the same 4 columns of rows rr0, rr0 + kStep, ...
            constexpr int kStep = 4 * kPThreads / kPW;
            const int col = (4 * tid) % kPW, rr0 = (4 * tid) / kPW, j = L0 + col;
            if (col < width) {
                uint32_t dst = smem_addr(&strip[sbuf][0][rr0][col]);
                size_t off = (size_t)(r0 + rr0) * w.C + j;
                const size_t off_step = (size_t)kStep * w.C;
                if (w.vec) {
                    const bool jin = j >= 0 && j + 3 < w.C;
#pragma unroll
                    for (int v = 0; v < kPVec; ++v, dst += kStep * kPW * 4, off += off_step)
                        copy16(dst, off, jin && rr0 + v * kStep < nr);
                } else {
#pragma unroll
                    for (int v = 0; v < kPVec; ++v, dst += kStep * kPW * 4, off += off_step)
                        copy4x4(dst, off, j, rr0 + v * kStep < nr);
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < kPVec; ++v) {
                const int e = (tid + v * kPThreads) * 4, rr = e / kPW, col = e - rr * kPW;
                const int j = L0 + col;
                if (col < width) {
                    const uint32_t dst = smem_addr(&strip[sbuf][0][rr][col]);
                    const size_t off = (size_t)(r0 + rr) * w.C + j;
                    if (w.vec)
                        copy16(dst, off, rr < nr && j >= 0 && j + 3 < w.C);
                    else
                        copy4x4(dst, off, j, rr < nr);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto wait_loads = [] { asm volatile("cp.async.wait_group 0;" ::: "memory"); };
    // bands of blocks [win0, win0 + n), all threads at once: min / max over the
    // masked angles of the end bins' positions at the block's first and last rows
    auto bands_for = [&](int n) {
        for (int k = tid; k < n; k += kPThreads) bands[k] = make_int2(INT_MAX, INT_MIN);
        __syncthreads();
        for (int idx = tid; idx < n * kPG; idx += kPThreads) {
            const int k = idx / kPG, a = idx % kPG;
            if (!((mask >> a) & 1)) continue;
            const RayGeom g = rg[a];
            const int r_first = row0 + (win0 + k) * kRows, r_last = min(r_first + kRows, r_end) - 1;
            const long long p = g.X0 + (long long)w.b0 * g.dX, q = g.X0 + (long long)w.bhi * g.dX;
            const long long u = (long long)r_first * g.rho, v = (long long)r_last * g.rho;
            const long long mn = min(min(p - u, q - u), min(p - v, q - v));
            const long long mx = max(max(p - u, q - u), max(p - v, q - v));
            atomicMin(&bands[k].x, hi32(mn) - 2);
            atomicMax(&bands[k].y, hi32(mx) + 3);
        }
        __syncthreads();
    };
    // Ray positions x* + 1/2 - L0 in unsigned 9.23 fixed point (the block's
    // band keeps them inside (2.5, kPW - 5.5), so below 2^32 for every
    // width), anchored from the exact 32.32 value at the first row of every
    // chunk, so 32 rounded row steps add at most 2e-6 bins.  A chunk's second
    // block moves them by the change of L0, an exact integer; L0 only shifts
    // the integer part, so the bits do not depend on the blocking.
    unsigned x32[kPRays];
    int L0_prev = 0;
    int seg_left = per - c_lo % per;       // chunks until the current row segment ends
    for (; win0 < n_blocks; win0 += kPBandWin) {
        const int win_end = min(n_blocks, win0 + kPBandWin);
        bands_for(win_end - win0);
        load(win0, 0);
        wait_loads();
        __syncthreads();
        for (int c = win0; c < win_end; ++c) {
            const int cur = (c - win0) & 1;
            const bool more = c + 1 < win_end;
            if (more) load(c + 1, cur ^ 1);   // the barrier that ended block c - 1 freed that buffer
            const int r0 = row0 + c * kRows, nr = min(kRows, r_end - r0), L0 = bands[c - win0].x & ~3;
            if (kSub == 1 || c % kSub == 0) {
#pragma unroll
                for (int k = 0; k < kPRays; ++k) {
                    const long long rel = X64[k] - (long long)r0 * rg[asub + 2 * k].rho - ((long long)L0 << 32);
                    x32[k] = act[k] ? (unsigned)(rel >> (32 - kFrac)) : (3u << kFrac);
                }
            } else {
                const unsigned d = (unsigned)(L0_prev - L0) << kFrac;
#pragma unroll
                for (int k = 0; k < kPRays; ++k) x32[k] += act[k] ? d : 0u;
            }
            L0_prev = L0;
            const float *S = &strip[cur][0][0][0];
            auto row = [&](const float *Sr) {   // one staged row: three taps per ray and slice
                float v[kPRays], q0[kNS][kPRays], q1[kNS][kPRays], q2[kNS][kPRays];
#pragma unroll
                for (int k = 0; k < kPRays; ++k) {
                    const float *q = Sr + (x32[k] >> kFrac) - 1;
                    v[k] = __uint_as_float((x32[k] & 0x7FFFFFu) | 0x3F800000u);   // 1 + frac in [1, 2)
#pragma unroll
                    for (int n = 0; n < kNS; ++n) {
                        q0[n][k] = q[n * kPlane];
                        q1[n][k] = q[n * kPlane + 1];
                        q2[n][k] = q[n * kPlane + 2];
                    }
                    x32[k] -= r32[k];
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int k = 2 * p;
                    // a psi = a (1 + frac) - 3a/2, psi in [-1/2, 1/2)
                    const float2 ap = fma2(make_float2(aa[k], aa[k + 1]), make_float2(v[k], v[k + 1]),
                                           make_float2(m1[k], m1[k + 1]));
                    const float2 wl = make_float2(__saturatef(t1[k] - ap.x), __saturatef(t1[k + 1] - ap.y));
                    const float2 wc = make_float2(c1[k] - fabsf(ap.x), c1[k + 1] - fabsf(ap.y));
                    const float2 wr = make_float2(__saturatef(t1[k] + ap.x), __saturatef(t1[k + 1] + ap.y));
#pragma unroll
                    for (int n = 0; n < kNS; ++n) {
                        acc[n][p] = fma2(wl, make_float2(q0[n][k], q0[n][k + 1]), acc[n][p]);
                        acc[n][p] = fma2(wc, make_float2(q1[n][k], q1[n][k + 1]), acc[n][p]);
                        acc[n][p] = fma2(wr, make_float2(q2[n][k], q2[n][k + 1]), acc[n][p]);
                    }
                }
            };
            if (nr == kRows) {                  // full block: rows at constant offsets
#pragma unroll
                for (int rr = 0; rr < kRows; ++rr) row(S + rr * kPW);
            } else {
                for (int rr = 0; rr < nr; ++rr) row(S + rr * kPW);
            }
            // end of a chunk that ends a row segment: its scaled sum joins the
            // total (in segment order)
            const bool last = c + 1 == n_blocks;
            if ((kSub == 1 || c % kSub == kSub - 1 || last) && (--seg_left == 0 || last)) {
                seg_left = per;
                const float2 s2 = make_float2(scale, scale);
#pragma unroll
                for (int n = 0; n < kNS; ++n)
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        tot[2 * n + p][tid] = add2(tot[2 * n + p][tid], mul2(s2, acc[n][p]));
                        acc[n][p] = make_float2(0.0f, 0.0f);
                    }
            }
            if (more) wait_loads();
            __syncthreads();
        }
    }
}

// One CTA: angles [g0, g0 + 8) x bins [b0, b0 + 128) of one slice;
// img/imgT are that slice's image and its transpose.  The rows of each walk
// fall into nseg segments of equal chunk counts (the last one shorter), and
// a ray's value is the sum, in segment order, of its scaled per-segment sums.
// seg >= 0: this CTA walks segment seg only and writes that partial (the
// partials are added in order afterwards); seg < 0: it walks all segments and
// adds them itself.  Both give the same bits, so the segmentation (a
// property of the slice geometry) and not the launch decides the rounding.
// The CTA projects the kNS slices of one geometry in S (S.img[n], its
// transpose S.imgT[n] -> S.sino[n]); every slice gets the bits of a one-slice
// CTA.
struct ProjSlices {
    const float *img[2], *imgT[2];
    float *sino[2];
};

template <int kPW, int kNS>
__device__ __forceinline__ void proj_cta(const AngleInfo *__restrict__ tab, const ProjSlices &S, int n_angles,
                                         int n_bins, int nx, int ny, double cx, double cy, float scale, int g0,
                                         int b0, int seg, int nseg) {
    extern __shared__ __align__(16) float proj_smem[];
    constexpr int kRows = prows<kPW, kNS>();
    float (*strip)[kNS][kRows][kPW] = reinterpret_cast<float (*)[kNS][kRows][kPW]>(proj_smem);
    __shared__ RayGeom rg[kPG];
    __shared__ int2 bands_s[kPBandWin];
    __shared__ int phase_mask[2], fits_s, clip_s[2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = b0 + 16 * warp + (lane & 15);
    const int asub = lane >> 4;
    const int bhi = min(b0 + kPB, n_bins) - 1;

    if (tid < kPG) {
        RayGeom g;
        g.major = -1; g.X0 = g.dX = g.rho = 0; g.a = 0.0f;
        if (g0 + tid < n_angles) g = ray_geom(tab[g0 + tid], cx, cy);
        rg[tid] = g;
    }
    if (tid < 2) phase_mask[tid] = 0;
    __syncthreads();
    if (tid < kPG && rg[tid].major >= 0) atomicOr(&phase_mask[rg[tid].major], 1 << tid);
    __syncthreads();

    float2 acc[kNS][2];                     // per slice, rays (0,1), (2,3): segment sums
    __shared__ float2 tot[2 * kNS][kPThreads];  // per thread: scaled sums of its finished segments
#pragma unroll
    for (int n = 0; n < kNS; ++n) {
        acc[n][0] = acc[n][1] = make_float2(0.0f, 0.0f);
        tot[2 * n][tid] = tot[2 * n + 1][tid] = make_float2(0.0f, 0.0f);
    }

    for (int major = 0; major < 2; ++major) {
        const int mask_all = phase_mask[major];
        if (!mask_all) continue;
        WalkArgs w;
        w.R = major == 0 ? ny : nx;
        w.C = major == 0 ? nx : ny;
        w.b0 = b0; w.bhi = bhi; w.b = b;
        w.vec = w.C % 4 == 0;
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            w.M[n] = major == 0 ? S.img[n < kNS ? n : 0] : S.imgT[n < kNS ? n : 0];
            w.vec = w.vec && (reinterpret_cast<uintptr_t>(w.M[n]) & 15) == 0;
        }
        // Largest subset of consecutive angles (8, 4, 2, 1) whose bands fit:
        // the band of rows [r, r + n - 1] (n rows per staged block) has a
        // width convex in r, every block lies within the range of the first
        // and last n-row windows, and the float4 alignment of a block's start
        // adds at most 3 columns.  A single angle always fits
        // (127 sqrt 2 + 32 + 8 < 256).
        if (warp == 0) {
            int gs = kPG;
            const int last0 = max(0, w.R - kRows);
            for (; gs > 1; gs >>= 1) {
                bool ok = true;
                for (int s0 = 0; s0 < kPG; s0 += gs) {
                    const int m = mask_all & (((1 << gs) - 1) << s0);
                    if (!m) continue;
                    int L0a, Ha, L0b, Hb;
                    chunk_band(rg, m, b0, bhi, 0, min(kRows, w.R) - 1, L0a, Ha);
                    chunk_band(rg, m, b0, bhi, last0, w.R - 1, L0b, Hb);
                    ok = ok && (Ha - L0a + 4 <= kPW) && (Hb - L0b + 4 <= kPW);
                }
                if (ok) break;
            }
            if (lane == 0) fits_s = gs;
        }
        __syncthreads();
        const int gs = fits_s;
        const int nch = (w.R + kPR - 1) / kPR, per = (nch + nseg - 1) / nseg;
        const int c_lo = seg >= 0 ? seg * per : 0, c_hi = seg >= 0 ? min(nch, c_lo + per) : nch;
        for (int s0 = 0; s0 < kPG; s0 += gs) {
            const int m = mask_all & (((1 << gs) - 1) << s0);
            if (!m) continue;
            // only the chunks where some ray of the subset meets the image
            if (warp == 0) chunk_clip(rg, m, b0, bhi, w.R, w.C, clip_s);
            __syncthreads();
            const int cl = max(c_lo, clip_s[0]), ch = min(c_hi, clip_s[1]);
            __syncthreads();
            walk_pass<kPW, kNS>(w, rg, m, acc, tot, scale, per, strip, bands_s, cl, ch);
        }
        __syncthreads();
    }
    if (b <= bhi) {
#pragma unroll
        for (int n = 0; n < kNS; ++n) {
            const float r[kPRays] = {tot[2 * n][tid].x, tot[2 * n][tid].y, tot[2 * n + 1][tid].x,
                                     tot[2 * n + 1][tid].y};
#pragma unroll
            for (int k = 0; k < kPRays; ++k) {
                const int a = g0 + asub + 2 * k;
                if (a < n_angles) S.sino[n][(size_t)a * n_bins + b] = r[k];
            }
        }
    }
}

// split: blockIdx.z = slice * nseg + segment, and the output is the partial
// sinogram of the segment, part[slice][segment][angle][bin]; otherwise
// blockIdx.z = slice (NS = 1) or the pair of slices 2 z, 2 z + 1 (NS = 2; the
// last slice of an odd count is walked twice, both planes giving its bits)
// and the CTA adds the segments itself.
template <int PW, int NS>
__global__ void __launch_bounds__(kPThreads, 3)
proj_kernel(const AngleInfo *__restrict__ tab, const float *__restrict__ img, const float *__restrict__ imgT,
            float *__restrict__ sino, int n_angles, int n_bins, int nx, int ny, double cx, double cy,
            float scale, int nseg, int split, int n_slices) {
    const int bz = (int)blockIdx.z;
    const size_t img_sz = (size_t)nx * ny, sino_sz = (size_t)n_angles * n_bins;
    ProjSlices S;
    if (NS == 1) {
        const int slice = split ? bz / nseg : bz;
        S.img[0] = S.img[1] = img + slice * img_sz;
        S.imgT[0] = S.imgT[1] = imgT + slice * img_sz;
        S.sino[0] = S.sino[1] = sino + (size_t)bz * sino_sz;
    } else {
        const int s0 = 2 * bz, s1 = min(2 * bz + 1, n_slices - 1);
        S.img[0] = img + s0 * img_sz;
        S.img[1] = img + s1 * img_sz;
        S.imgT[0] = imgT + s0 * img_sz;
        S.imgT[1] = imgT + s1 * img_sz;
        S.sino[0] = sino + s0 * sino_sz;
        S.sino[1] = sino + s1 * sino_sz;
    }
    proj_cta<PW, NS>(tab, S, n_angles, n_bins, nx, ny, cx, cy, scale, blockIdx.y * kPG, blockIdx.x * kPB,
                     NS == 1 && split ? bz % nseg : -1, nseg);
}

// sino[s][k] = sum over segments (in order) of part[s][seg][k]
__global__ void proj_reduce_kernel(const float *__restrict__ part, float *__restrict__ sino, size_t per_slice,
                                   int nseg) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= per_slice) return;
    const float *p = part + (size_t)blockIdx.y * nseg * per_slice + k;
    float acc = 0.0f;
    for (int g = 0; g < nseg; ++g) acc += p[(size_t)g * per_slice];
    sino[(size_t)blockIdx.y * per_slice + k] = acc;
}

// Mixed batch: CTA k projects angle group items[k].z, bin block items[k].y of
// slice items[k].x and, with NS = 2, of slice items[k].w too, a slice of the
// same geometry (or items[k].x again).
template <int PW, int NS>
__global__ void __launch_bounds__(kPThreads, 3)
proj_batch_kernel(const BatchSlice *__restrict__ slices, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    const BatchSlice s = slices[it.x];
    ProjSlices S;
    S.img[0] = S.img[1] = s.proj_in;
    S.imgT[0] = S.imgT[1] = s.proj_inT;
    S.sino[0] = S.sino[1] = s.proj_out;
    if (NS == 2) {
        const BatchSlice &t = slices[it.w];
        S.img[1] = t.proj_in;
        S.imgT[1] = t.proj_inT;
        S.sino[1] = t.proj_out;
    }
    proj_cta<PW, NS>(s.tab, S, s.n_angles, s.n_bins, s.nx, s.ny, s.cx, s.cy, s.pixel_size, it.z * kPG, it.y * kPB,
                     -1, s.proj_nseg);
}

// Mixed batch transpose: CTA k moves 64 x 64 tile (items[k].y, items[k].z) of slice items[k].x.
__global__ void transpose_batch_kernel(const BatchSlice *__restrict__ slices, const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    const BatchSlice s = slices[it.x];
    transpose_tile(s.proj_in, s.proj_inT, s.ny, s.nx, it.z * kTT, it.y * kTT);
}

}  // namespace

// Staging width (256, 384 or 512 columns): the autotuned choice for the
// geometry (pyhst_autotune_project, pyhst_set_project_staging) if there is
// one; else sparse angle sets (image size / number of angles > 2) take 512
// columns, since their 8-angle bands rarely fit 256, and the others 256.
// Every width walks every ray with the same fixed-point positions and sum
// order, so the choice changes no bits.
namespace {
std::mutex g_pw_mu;
std::map<std::tuple<int, int, int, int>, int> g_pw_tune;   // (device, nx, ny, n_angles) -> 256 or 512
}  // namespace

int project_width(int nx, int ny, int n_angles) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_pw_mu);
        auto it = g_pw_tune.find(std::make_tuple(dev, nx, ny, n_angles));
        if (it != g_pw_tune.end()) return it->second;
    }
    return (double)std::max(nx, ny) > 2.0 * n_angles ? 512 : 256;
}

namespace {
template <int PW, int NS>
bool proj_attr_pw() {
    return cudaFuncSetAttribute(proj_kernel<PW, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem<PW, NS>()) ==
               cudaSuccess &&
           cudaFuncSetAttribute(proj_batch_kernel<PW, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                psmem<PW, NS>()) == cudaSuccess;
}
}  // namespace

int set_proj_attr() {
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status("cudaGetDevice");
    if (dev >= 0 && dev < 64 && done[dev]) return PYHST_OK;
    if (!(proj_attr_pw<256, 1>() && proj_attr_pw<384, 1>() && proj_attr_pw<512, 1>() && proj_attr_pw<256, 2>() &&
          proj_attr_pw<384, 2>() && proj_attr_pw<512, 2>()))
        return cuda_status("projection kernel shared-memory attribute");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return PYHST_OK;
}

int proj_blocks(int n_angles, int n_bins, int *nb, int *na) {
    *nb = (n_bins + kPB - 1) / kPB;
    *na = (n_angles + kPG - 1) / kPG;
    return *nb * *na;
}

namespace {
template <int NS>
void proj_batch_launch(int width, const BatchSlice *slices, const int4 *items, int n, cudaStream_t st) {
    if (width == 512)
        proj_batch_kernel<512, NS><<<n, kPThreads, psmem<512, NS>(), st>>>(slices, items);
    else if (width == 384)
        proj_batch_kernel<384, NS><<<n, kPThreads, psmem<384, NS>(), st>>>(slices, items);
    else
        proj_batch_kernel<256, NS><<<n, kPThreads, psmem<256, NS>(), st>>>(slices, items);
}
}  // namespace

int launch_project_batch(const BatchSlice *slices, const int4 *proj_items, int n_proj_items,
                         const int4 *tr_items, int n_tr_items, int width, cudaStream_t st, int ns) {
    if (n_tr_items > 0) {
        transpose_batch_kernel<<<n_tr_items, dim3(32, 8), 0, st>>>(slices, tr_items);
        int rc = cuda_status("batched transpose kernel");
        if (rc) return rc;
    }
    if (n_proj_items <= 0) return PYHST_OK;
    int rc = set_proj_attr();
    if (rc) return rc;
    ProfScope prof(kProfProject, st);
    if (ns == 2)
        proj_batch_launch<2>(width, slices, proj_items, n_proj_items, st);
    else
        proj_batch_launch<1>(width, slices, proj_items, n_proj_items, st);
    return cuda_status("batched projection kernel");
}

// Row segments of a slice geometry: when one slice gives few CTAs, enough
// segments to fill the GPU a few times (at least 4 waves of 3 CTAs per SM),
// at least 2 chunks (64 rows) each; between that count and twice it, the one
// whose last wave is fullest.  A property of the slice geometry alone (not of
// how many slices a call holds), since the segments fix the order of the
// float32 sums.
int proj_segments(const pyhst_geometry *g) {
    const long ctas = (long)((g->n_bins + kPB - 1) / kPB) * ((g->n_angles + kPG - 1) / kPG);
    if (ctas >= kPTargetCtas) return 1;
    const long cap = std::max(1, std::min(g->nx, g->ny) / (kPR * 2));
    const long lo = std::min(cap, (kPTargetCtas + ctas - 1) / ctas), hi = std::min(cap, 2 * lo);
    constexpr long wave = kPTargetCtas / 4;
    long best = lo;
    double best_eff = 0.0;
    for (long n = lo; n <= hi; ++n) {
        const long c = ctas * n;
        const double eff = (double)c / (double)(wave * ((c + wave - 1) / wave));
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = n;
        }
    }
    return (int)std::max(1L, best);
}

namespace {
// Segments as separate CTAs (partials added afterwards) when the call has
// few CTAs; otherwise each CTA adds its own segments (same bits).
bool proj_split(const pyhst_geometry *g, int nseg) {
    const long ctas = (long)((g->n_bins + kPB - 1) / kPB) * ((g->n_angles + kPG - 1) / kPG) * g->n_slices;
    return nseg > 1 && ctas < kPTargetCtas && (long)g->n_slices * nseg <= 65535;
}
}  // namespace

// Transposed image, then (for split launches) the partial sinograms; the
// partials of a 1-slice call fit too, since callers also project single
// slices of their geometry.
size_t project_scratch_bytes(const pyhst_geometry *g) {
    pyhst_geometry g1 = *g;
    g1.n_slices = 1;
    const int ns = proj_segments(g);
    const size_t part = std::max(proj_split(g, ns) ? (size_t)ns * g->n_slices : 0,
                                 proj_split(&g1, ns) ? (size_t)ns : 0) *
                        (size_t)g->n_angles * g->n_bins;
    return align_up(sizeof(float) * (size_t)g->nx * g->ny * g->n_slices) + align_up(sizeof(float) * part);
}

namespace {
template <int NS>
void proj_launch(int width, dim3 grid, cudaStream_t st, const AngleInfo *tab, const float *img, const float *xt,
                 float *dst, const pyhst_geometry *g, float scale, int nseg, int split) {
    if (width == 512)
        proj_kernel<512, NS><<<grid, kPThreads, psmem<512, NS>(), st>>>(tab, img, xt, dst, g->n_angles, g->n_bins, g->nx,
                                                                        g->ny, g->cx, g->cy, scale, nseg, split,
                                                                        g->n_slices);
    else if (width == 384)
        proj_kernel<384, NS><<<grid, kPThreads, psmem<384, NS>(), st>>>(tab, img, xt, dst, g->n_angles, g->n_bins, g->nx,
                                                                        g->ny, g->cx, g->cy, scale, nseg, split,
                                                                        g->n_slices);
    else
        proj_kernel<256, NS><<<grid, kPThreads, psmem<256, NS>(), st>>>(tab, img, xt, dst, g->n_angles, g->n_bins, g->nx,
                                                                        g->ny, g->cx, g->cy, scale, nseg, split,
                                                                        g->n_slices);
}
}  // namespace

int launch_project(const pyhst_geometry *g, const AngleInfo *tab, const float *img, float *sino,
                   float scale, float *xt, cudaStream_t st, int staging) {
    if (g->n_slices > 65535) return fail(PYHST_ERR_INVALID_ARG, "too many slices in one call (%d)", g->n_slices);
    dim3 tb(32, 8), tg((g->nx + kTT - 1) / kTT, (g->ny + kTT - 1) / kTT, g->n_slices);
    transpose_kernel<<<tg, tb, 0, st>>>(img, xt, g->ny, g->nx);
    int rc = cuda_status("transpose kernel");
    if (rc) return rc;
    if ((rc = set_proj_attr())) return rc;
    const int nseg = proj_segments(g);
    const bool split = proj_split(g, nseg);
    float *part = xt + align_up(sizeof(float) * (size_t)g->nx * g->ny * g->n_slices) / sizeof(float);
    // two slices per CTA unless the rows are split into segment CTAs
    const int ns = !split && g->n_slices >= 2 ? 2 : 1;
    dim3 grid((g->n_bins + kPB - 1) / kPB, (g->n_angles + kPG - 1) / kPG,
              ns == 2 ? (g->n_slices + 1) / 2 : g->n_slices * (split ? nseg : 1));
    {
        ProfScope prof(kProfProject, st);
        float *dst = split ? part : sino;
        const int width = staging > 0 ? staging : project_width(g->nx, g->ny, g->n_angles);
        if (ns == 2)
            proj_launch<2>(width, grid, st, tab, img, xt, dst, g, scale, nseg, 0);
        else
            proj_launch<1>(width, grid, st, tab, img, xt, dst, g, scale, nseg, split ? 1 : 0);
    }
    if ((rc = cuda_status("projection kernel"))) return rc;
    if (split) {
        const size_t per = (size_t)g->n_angles * g->n_bins;
        proj_reduce_kernel<<<dim3((unsigned)((per + 255) / 256), g->n_slices), 256, 0, st>>>(part, sino, per, nseg);
        rc = cuda_status("projection segment sum");
    }
    return rc;
}

}  // namespace pyhst

extern "C" int pyhst_set_project_staging(int32_t nx, int32_t ny, int32_t n_angles, int32_t width) {
    using namespace pyhst;
    if (nx < 1 || ny < 1 || n_angles < 1) return fail(PYHST_ERR_INVALID_ARG, "image %d x %d, %d angles", nx, ny, n_angles);
    if (width != 0 && width != 256 && width != 384 && width != 512)
        return fail(PYHST_ERR_INVALID_ARG, "staging width %d: need 256, 384 or 512 (0 clears)", width);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status("cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_pw_mu);
    const auto key = std::make_tuple(dev, (int)nx, (int)ny, (int)n_angles);
    if (width == 0)
        g_pw_tune.erase(key);
    else
        g_pw_tune[key] = width;
    return PYHST_OK;
}

extern "C" int pyhst_autotune_project(const pyhst_geometry *g, const float *img, float *sino, void *workspace,
                                      size_t ws_bytes, int32_t *best, pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if (!img || !sino) return fail(PYHST_ERR_INVALID_ARG, "img/sino pointer is NULL");
    const size_t need = pyhst_workspace_size(g, PYHST_OP_PROJECT);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv(workspace, ws_bytes);
    AngleInfo *tab = cv.take<AngleInfo>(g->n_angles);
    float *xt = cv.take<float>(project_scratch_bytes(g) / sizeof(float));
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_status("autotune events");
    }
    int pick = project_width(g->nx, g->ny, g->n_angles);
    float best_ms = 1e30f;
    for (int width : {256, 384, 512}) {
        if ((rc = launch_project(g, tab, img, sino, g->pixel_size, xt, st, width))) break;   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && !rc; ++r) rc = launch_project(g, tab, img, sino, g->pixel_size, xt, st, width);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = cuda_status("autotune timing");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            pick = width;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best) *best = pick;
    return pyhst_set_project_staging(g->nx, g->ny, g->n_angles, pick);
}

extern "C" int pyhst_project(const pyhst_geometry *g, const float *img, float *sino, void *workspace,
                             size_t ws_bytes, pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if (!img || !sino) return fail(PYHST_ERR_INVALID_ARG, "img/sino pointer is NULL");
    const size_t need = pyhst_workspace_size(g, PYHST_OP_PROJECT);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv(workspace, ws_bytes);
    AngleInfo *tab = cv.take<AngleInfo>(g->n_angles);
    float *xt = cv.take<float>(project_scratch_bytes(g) / sizeof(float));
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    return launch_project(g, tab, img, sino, g->pixel_size, xt, st);
}
