// Forward projector: the exact transpose of the unweighted back-projector,
//   sino[a][b] = scale * sum_{i,j} img[i][j] * max(0, 1 - |t_a(i, j) - b|),
// the operator P the iterative methods apply at every iteration (Sec. 2.3,
// last paragraph; Eq. 1 and Eq. 3).
//
// The paper keeps the volume in a texture.  Here the projector is ray-driven
// and deterministic (no atomics): one thread per (angle, bin).  For an angle
// whose |cos| >= |sin| the ray walks the image rows; on row i the hat weight of
// pixel j is 1 - |cos| * |j - x*(i)|, with x*(i) the column where t = b, so at
// most three pixels per row are non-zero.  For |sin| > |cos| the same walk runs
// over the rows of a transposed copy of the image, so warps always read
// consecutive pixels.  x*(i) is anchored in float64 every 64 rows and followed
// in float32 as a small fractional offset inside the block, which keeps the
// weights within a few 1e-6 of their float64 values (the back-projector's own
// accuracy), so the pair stays adjoint to float32 rounding.
#include <cmath>

#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kRayThreads = 128;
constexpr int kAnchor = 64;   // rows per float64 anchor

__global__ void transpose_kernel(const float *__restrict__ in, float *__restrict__ out, int rows,
                                 int cols) {
    __shared__ float tile[32][33];
    const size_t off = (size_t)blockIdx.z * rows * cols;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[off + (size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[off + (size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

// One ray (angle a, bin b) per thread.
__global__ void __launch_bounds__(kRayThreads)
ray_kernel(const AngleInfo *__restrict__ tab, const float *__restrict__ img,
           const float *__restrict__ imgT, float *__restrict__ sino, int n_angles, int n_bins, int nx,
           int ny, double cx, double cy, float scale) {
    const int b = blockIdx.x * kRayThreads + threadIdx.x;
    const int a = blockIdx.y;
    const int slice = blockIdx.z;
    if (b >= n_bins) return;
    const AngleInfo e = tab[a];
    float acc = 0.0f;
    // Walk geometry: rows r of a row-major [R][C] array M; the column
    // coefficient cc multiplies the column index, rr the row index.
    const bool xmajor = fabs(e.c) >= fabs(e.s);
    const float *M = xmajor ? img + (size_t)slice * nx * ny : imgT + (size_t)slice * nx * ny;
    const int R = xmajor ? ny : nx, C = xmajor ? nx : ny;
    const double cc = xmajor ? e.c : e.s, rr = xmajor ? e.s : e.c;
    const double ccen = xmajor ? cx : cy, rcen = xmajor ? cy : cx;
    if (isfinite(cc) && isfinite(rr) && isfinite(e.axis) && cc != 0.0) {
        // x*(r) = ccen + (b - axis - (r - rcen) rr) / cc = X - r rho
        const double inv = 1.0 / cc, rho = rr * inv;
        const double X = ccen + ((double)b - e.axis + rcen * rr) * inv;
        // rows where x* lies in [-2, C + 1]: the only rows with non-zero weights
        int r_lo = 0, r_hi = R - 1;
        if (rho != 0.0) {
            double ra = (X + 2.0) / rho, rb = (X - (C + 1.0)) / rho;
            double lo = fmin(ra, rb), hi = fmax(ra, rb);
            lo = fmax(lo, 0.0);
            hi = fmin(hi, (double)(R - 1));
            r_lo = (lo > hi) ? 1 : (int)ceil(lo);
            r_hi = (lo > hi) ? 0 : (int)floor(hi);
        } else if (!(X >= -2.0 && X <= C + 1.0)) {
            r_lo = 1; r_hi = 0;
        }
        const float rhof = (float)rho;
        const float acf = (float)fabs(cc);
        for (int r0 = r_lo; r0 <= r_hi; r0 += kAnchor) {
            const double xs = X - (double)r0 * rho;
            const double J0d = floor(xs);
            const int J0 = (int)J0d;
            const float phi0 = (float)(xs - J0d);
            const int rend = min(r_hi, r0 + kAnchor - 1);
            const float *row = M + (size_t)r0 * C;
            for (int r = r0; r <= rend; ++r, row += C) {
                const float xr = fmaf(-(float)(r - r0), rhof, phi0);   // x*(r) - J0
                const float tm = add_rd(xr, kMagic);
                const float fl = tm - kMagic;                          // floor(xr), exact
                const float phi = xr - fl;                             // in [0, 1)
                const int J = J0 + (int)(__float_as_uint(tm) - kMagicBits);
                // at most three non-zero weights: J-1..J+1 when phi < 1/2, J..J+2 otherwise
                const int sh = phi < 0.5f ? 0 : 1;
                const int j0 = J - 1 + sh;
                const float d0 = (float)(sh - 1) - phi;                // j0 - x*
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int j = j0 + k;
                    const float w = fmaxf(0.0f, fmaf(-acf, fabsf(d0 + (float)k), 1.0f));
                    if ((unsigned)j < (unsigned)C) acc = fmaf(w, __ldg(row + j), acc);
                }
            }
        }
    }
    sino[((size_t)slice * n_angles + a) * n_bins + b] = scale * acc;
}

}  // namespace

size_t project_scratch_bytes(const pyhst_geometry *g) {
    return align_up(sizeof(float) * (size_t)g->nx * g->ny * g->n_slices);
}

int launch_project(const pyhst_geometry *g, const AngleInfo *tab, const float *img, float *sino,
                   float scale, float *xt, cudaStream_t st) {
    if (g->n_slices > 65535) return fail(PYHST_ERR_INVALID_ARG, "too many slices in one call (%d)", g->n_slices);
    dim3 tb(32, 8), tg((g->nx + 31) / 32, (g->ny + 31) / 32, g->n_slices);
    transpose_kernel<<<tg, tb, 0, st>>>(img, xt, g->ny, g->nx);
    int rc = cuda_status("transpose kernel");
    if (rc) return rc;
    dim3 grid((g->n_bins + kRayThreads - 1) / kRayThreads, g->n_angles, g->n_slices);
    ProfScope prof(kProfProject, st);
    ray_kernel<<<grid, kRayThreads, 0, st>>>(tab, img, xt, sino, g->n_angles, g->n_bins, g->nx, g->ny,
                                             g->cx, g->cy, scale);
    return cuda_status("projection kernel");
}

}  // namespace pyhst

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
    float *xt = cv.take<float>((size_t)g->nx * g->ny * g->n_slices);
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    return launch_project(g, tab, img, sino, g->pixel_size, xt, st);
}
