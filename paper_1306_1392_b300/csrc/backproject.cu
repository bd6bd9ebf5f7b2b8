// Pixel-driven back-projection with linear interpolation (Sec. 2.3).
//
//   img[i][j] = weight * sum_a L(q_a, t_a(i, j)),
//   t_a(i, j) = (j - cx) cos(th_a) + (i - cy) sin(th_a) + axis_a,
//   L(q, t)   = (1 - f) q[floor t] + f q[floor t + 1], zero outside the detector.
//
// The paper's kernel reads the sinogram through the texture unit with hardware
// interpolation, one output tile per thread block.  Hardware filtering keeps
// only 8 fractional bits of the weight, too coarse for float32 parity, so
// here each CTA owns a 64 x 32 output tile and, for blocks of 32 angles,
// stages in shared memory the window of each filtered row that the tile can
// reach.  Each window entry k holds (dq, c0) = (q[g+1] - q[g], q[g] - k dq)
// for bin g = w0 + k, so that at the tile-local coordinate u (k <= u < k+1)
//   L = c0 + u * dq     (one FMA),
// and floor(u) comes from one add rounded toward -inf (see add_rd).  The
// tile-local coordinate u = (T0 - w0) + dx cos + dy sin is small (< 76), so
// float32 keeps ~4e-6 bins of accuracy; T0, the coordinate of the tile origin,
// is formed in float64 once per (tile, angle).
#include <climits>
#include <cmath>

#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kThreads = 256;
constexpr int kTX = 64, kTY = 32;   // CTA output tile (x, y)
constexpr int kRX = 4, kRY = 2;     // pixels per thread: x stride 8, y stride 4
constexpr int kNA = 32;             // angles staged per pass
constexpr int kW = 76;              // window entries per angle: ceil(hypot(63, 31)) + 4, rounded up

struct __align__(16) StageInfo {
    float base;   // u at the tile origin
    float cf, sf; // float32 cos, sin
    int w0;       // detector bin of window entry 0
};

template <bool kResidual>
__global__ void __launch_bounds__(kThreads, 4)
bp_kernel(const AngleInfo *__restrict__ tab, const float *__restrict__ srcA,
          const float *__restrict__ srcB, float *__restrict__ img, int n_angles, int n_bins,
          int nx, int ny, double cx, double cy, float weight, int tiles_x) {
    __shared__ __align__(16) float2 win[kNA * kW];
    __shared__ StageInfo info[kNA];

    const int slice = blockIdx.y;
    const int X0 = (blockIdx.x % tiles_x) * kTX;
    const int Y0 = (blockIdx.x / tiles_x) * kTY;
    const size_t sino_off = (size_t)slice * n_angles * n_bins;
    const float *A = srcA + sino_off;
    const float *B = kResidual ? srcB + sino_off : nullptr;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = (warp & 1) * 32 + (lane & 7);   // first pixel of this thread in the tile
    const int py = (warp >> 1) * 8 + (lane >> 3);
    const float fpx = (float)px, fpy = (float)py;
    const uint32_t win_s = smem_addr(win);

    float acc[kRY][kRX];
#pragma unroll
    for (int ry = 0; ry < kRY; ++ry)
#pragma unroll
        for (int rx = 0; rx < kRX; ++rx) acc[ry][rx] = 0.0f;

    for (int a0 = 0; a0 < n_angles; a0 += kNA) {
        const int na = min(kNA, n_angles - a0);
        if (threadIdx.x < kNA) {
            StageInfo si;
            si.base = 0.0f; si.w0 = 0;
            if ((int)threadIdx.x < na) {
                const AngleInfo e = tab[a0 + threadIdx.x];
                const double T0 = ((double)X0 - cx) * e.c + ((double)Y0 - cy) * e.s + e.axis;
                const double tmin = T0 + fmin(0.0, (kTX - 1) * e.c) + fmin(0.0, (kTY - 1) * e.s);
                const double w0 = floor(tmin) - 1.0;       // one guard entry below
                si.base = (float)(T0 - w0);
                si.cf = e.cf;
                si.sf = e.sf;
                si.w0 = (int)w0;
            }
            // Padding angles of the last block, and angles whose coordinates
            // are not finite or beyond any detector (|t| >= 1e9 bins), read
            // an all-zero window at a fixed in-range position.
            if ((int)threadIdx.x >= na || !(fabs(si.base) < 1.0e3f) || !(fabs((double)si.w0) < 1.0e9)) {
                si.base = 1.5f; si.cf = 0.0f; si.sf = 0.0f; si.w0 = INT_MIN / 2;
            }
            info[threadIdx.x] = si;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kNA * kW; k += kThreads) {
            const int a = k / kW, e = k - a * kW;
            float2 v = make_float2(0.0f, 0.0f);
            if (a < na) {
                const int g = info[a].w0 + e;
                const size_t row = (size_t)(a0 + a) * n_bins;
                float q0 = 0.0f, q1 = 0.0f;
                if (g >= 0 && g < n_bins) {
                    q0 = A[row + g];
                    if (kResidual) q0 -= B[row + g];
                }
                if (g + 1 >= 0 && g + 1 < n_bins) {
                    q1 = A[row + g + 1];
                    if (kResidual) q1 -= B[row + g + 1];
                }
                const float dq = q1 - q0;
                v = make_float2(dq, fmaf(-(float)e, dq, q0));
            }
            win[k] = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int a = 0; a < na; ++a) {
            const StageInfo si = info[a];
            const uint32_t wb = win_s + (uint32_t)(a * kW * 8) - (kMagicBits << 3);
            const float r0 = fmaf(fpy, si.sf, fmaf(fpx, si.cf, si.base));
#pragma unroll
            for (int ry = 0; ry < kRY; ++ry) {
                const float rb = fmaf((float)(4 * ry), si.sf, r0);
#pragma unroll
                for (int rx = 0; rx < kRX; ++rx) {
                    const float u = fmaf((float)(8 * rx), si.cf, rb);
                    const uint32_t bits = __float_as_uint(add_rd(u, kMagic));
                    const float2 w = lds64(wb + (bits << 3));
                    acc[ry][rx] += fmaf(u, w.x, w.y);
                }
            }
        }
        __syncthreads();
    }

    float *out = img + (size_t)slice * nx * ny;
#pragma unroll
    for (int ry = 0; ry < kRY; ++ry)
#pragma unroll
        for (int rx = 0; rx < kRX; ++rx) {
            const int x = X0 + px + 8 * rx, y = Y0 + py + 4 * ry;
            if (x < nx && y < ny) out[(size_t)y * nx + x] = weight * acc[ry][rx];
        }
}

}  // namespace

int launch_backproject(const pyhst_geometry *g, const AngleInfo *tab, BpSource src, float *img,
                       float weight, cudaStream_t st) {
    const int tiles_x = (g->nx + kTX - 1) / kTX;
    const int tiles_y = (g->ny + kTY - 1) / kTY;
    dim3 grid(tiles_x * tiles_y, g->n_slices);
    if (grid.y > 65535) return fail(PYHST_ERR_INVALID_ARG, "too many slices in one call (%d)", g->n_slices);
    ProfScope prof(kProfBackproject, st);
    if (src.b)
        bp_kernel<true><<<grid, kThreads, 0, st>>>(tab, src.a, src.b, img, g->n_angles, g->n_bins, g->nx,
                                                   g->ny, g->cx, g->cy, weight, tiles_x);
    else
        bp_kernel<false><<<grid, kThreads, 0, st>>>(tab, src.a, nullptr, img, g->n_angles, g->n_bins,
                                                    g->nx, g->ny, g->cx, g->cy, weight, tiles_x);
    return cuda_status("back-projection kernel");
}

}  // namespace pyhst

extern "C" int pyhst_backproject(const pyhst_geometry *g, const float *sino, float *img, float weight,
                                 void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if (!sino || !img) return fail(PYHST_ERR_INVALID_ARG, "sino/img pointer is NULL");
    if (!std::isfinite(weight)) return fail(PYHST_ERR_INVALID_ARG, "weight is not finite");
    const size_t need = pyhst_workspace_size(g, PYHST_OP_BACKPROJECT);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv(workspace, ws_bytes);
    AngleInfo *tab = cv.take<AngleInfo>(g->n_angles);
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    return launch_backproject(g, tab, BpSource{sino, nullptr}, img, weight, st);
}
