// Pixel-driven back-projection with linear interpolation (Sec. 2.3).
//
//   img[i][j] = weight * sum_a L(q_a, t_a(i, j)),
//   t_a(i, j) = (j - cx) cos(th_a) + (i - cy) sin(th_a) + axis_a,
//   L(q, t)   = (1 - f) q[floor t] + f q[floor t + 1], zero outside the detector.
//
// The paper's kernel reads the sinogram through the texture unit with hardware
// interpolation, one output tile per thread block.  Hardware filtering keeps
// only 8 fractional bits of the weight, too coarse for float32 parity, so
// here each CTA owns a 64 x 64 output tile and, for blocks of 16 angles,
// stages in shared memory the window of each filtered row that the tile can
// reach.  Each window entry k holds (dq, c0) = (q[g+1] - q[g], q[g] - k dq)
// for bin g = w0 + k, so that at the tile-local coordinate u (k <= u < k+1)
//   L = c0 + u * dq     (one FMA),
// and floor(u) comes from one add rounded toward -inf (see add_rd).  The
// tile-local coordinate u = (T0 - w0) + dx cos + dy sin is small (< 96), so
// float32 keeps ~1e-5 bins of accuracy; T0, the coordinate of the tile origin,
// is formed in float64 once per (tile, angle).
//
// Throughput: the inner loop reads one 8-byte window entry per update, which
// the shared-memory data pipe serves in two wavefronts per warp, so the kernel
// is bound by shared memory (128 B/clk/SM).  Everything else is kept off that
// pipe and off the issue slots: 16 pixels per thread amortise the per-angle
// set-up, paired float32 instructions (f32x2) form the floors and the
// accumulations, and the next block's windows are prefetched into registers
// from L2 while the current block is computed, with one barrier per block.
#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kThreads = 256;
constexpr int kTX = 64, kTY = 64;   // CTA output tile (x, y)
constexpr int kRX = 4, kRY = 4;     // pixels per thread: x stride 8, y stride 4 (warp: 32 x 16)
constexpr int kW = 96;              // window entries per angle: ceil(hypot(63, 63)) + 4, rounded up
// Angles staged per block (NA): 8, 16 or 24, a tuning parameter (the
// per-pixel sums run over the angles in the same order for every NA, and the
// padding slots of a last, partial block add +0 -- or, in the kPartial
// instantiation, are not walked: a sum that starts at +0 is never -0, so
// adding +0 changes no bit -- so results are identical);
// each thread fills NA * kW / kThreads window entries per block.
static_assert(kW % 32 == 0, "fill mapping");

struct __align__(16) StageInfo {
    float base;   // u at the tile origin
    float cf, sf; // float32 cos, sin
    int w0;       // detector bin of window entry 0
};

// Per-(tile, angle) set-up in float64.  Padding angles (past n_angles) and
// angles whose coordinates are not finite or beyond any detector read an
// all-zero window at a fixed in-range position.
__device__ __forceinline__ StageInfo stage_info(const AngleInfo *tab, int a, int n_angles, int X0, int Y0,
                                                double cx, double cy) {
    StageInfo si;
    si.base = 1.5f; si.cf = 0.0f; si.sf = 0.0f; si.w0 = INT_MIN / 2;
    if (a < n_angles) {
        const AngleInfo e = tab[a];
        const double T0 = ((double)X0 - cx) * e.c + ((double)Y0 - cy) * e.s + e.axis;
        const double tmin = T0 + fmin(0.0, (kTX - 1) * e.c) + fmin(0.0, (kTY - 1) * e.s);
        const double w0 = floor(tmin) - 1.0;       // one guard entry below
        if (fabs(T0) < 1.0e9) {
            si.base = (float)(T0 - w0);
            si.cf = e.cf;
            si.sf = e.sf;
            si.w0 = (int)w0;
        }
    }
    return si;
}

// One CTA: the 64 x 64 tile at (X0, Y0) of one slice.  A (and B in residual
// mode) are that slice's rows, out its image.
// With ystep given, out receives the gradient step z = ystep - invL * g of
// g = weight * back-projection, rounded as a separate pass would round it.
template <int kNA, bool kResidual, bool kPartial>
__device__ __forceinline__ void bp_tile(const AngleInfo *__restrict__ tab, const float *__restrict__ A,
                                        const float *__restrict__ B, float *__restrict__ out, int n_angles,
                                        int n_bins, int nx, int ny, double cx, double cy, float weight,
                                        int X0, int Y0, const float *__restrict__ ystep = nullptr,
                                        float invL = 0.0f) {
    static_assert(kNA % (kThreads / 32) == 0, "fill mapping");
    constexpr int kFill = kNA * kW / kThreads;   // window entries each thread fills per block
    __shared__ __align__(16) float2 win[2][kNA * kW];
    __shared__ StageInfo info[3][kNA];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int px = (warp & 1) * 32 + (lane & 7);   // first pixel of this thread in the tile
    const int py = (warp >> 1) * 16 + (lane >> 3);
    const float fpx = (float)px, fpy = (float)py;
    const int n_blocks = (n_angles + kNA - 1) / kNA;

    // Window fill: warp w fills angles w and w + 8 of a block, lanes the entries.
    float q0r[kFill], q1r[kFill];
    auto prefetch = [&](int blk) {
        const StageInfo *ib = info[blk % 3];
#pragma unroll
        for (int j = 0; j < kFill; ++j) {
            const int a = warp + (j / 3) * (kThreads / 32), e = lane + 32 * (j % 3);
            const int g = ib[a].w0 + e;
            const int ag = blk * kNA + a;
            const size_t row = (size_t)min(ag, n_angles - 1) * n_bins;
            float v0 = 0.0f, v1 = 0.0f;
            if (g >= 0 && g < n_bins) {
                v0 = __ldg(A + row + g);
                if (kResidual) v0 -= __ldg(B + row + g);
            }
            if (g + 1 >= 0 && g + 1 < n_bins) {
                v1 = __ldg(A + row + g + 1);
                if (kResidual) v1 -= __ldg(B + row + g + 1);
            }
            q0r[j] = v0;
            q1r[j] = v1;
        }
    };
    auto commit = [&](int buf) {
#pragma unroll
        for (int j = 0; j < kFill; ++j) {
            const int a = warp + (j / 3) * (kThreads / 32), e = lane + 32 * (j % 3);
            const float dq = q1r[j] - q0r[j];
            win[buf][a * kW + e] = make_float2(dq, fmaf(-(float)e, dq, q0r[j]));
        }
    };

    float2 acc[kRY][kRX / 2];
#pragma unroll
    for (int ry = 0; ry < kRY; ++ry)
#pragma unroll
        for (int rp = 0; rp < kRX / 2; ++rp) acc[ry][rp] = make_float2(0.0f, 0.0f);
    const float2 magic2 = make_float2(kMagic, kMagic);

    // prologue: info of blocks 0 and 1, window of block 0
    if (tid < kNA) info[0][tid] = stage_info(tab, tid, n_angles, X0, Y0, cx, cy);
    __syncthreads();
    prefetch(0);
    commit(0);
    if (tid < kNA) info[1][tid] = stage_info(tab, kNA + tid, n_angles, X0, Y0, cx, cy);
    __syncthreads();

    for (int blk = 0; blk < n_blocks; ++blk) {
        const int cur = blk & 1;
        const bool more = blk + 1 < n_blocks;
        if (more) prefetch(blk + 1);
        if (tid < kNA && blk + 2 < n_blocks)
            info[(blk + 2) % 3][tid] = stage_info(tab, (blk + 2) * kNA + tid, n_angles, X0, Y0, cx, cy);
        const StageInfo *ib = info[blk % 3];
        const uint32_t wbase = smem_addr(win[cur]) - (kMagicBits << 3);
        // kPartial: the last block walks its real angles only (a loop with a
        // run-time bound, slower on geometries without a partial block)
        const int na_blk = kPartial ? min(kNA, n_angles - blk * kNA) : kNA;
#pragma unroll 2
        for (int a = 0; a < na_blk; ++a) {
            const StageInfo si = ib[a];
            const uint32_t wb = wbase + (uint32_t)(a * kW * 8);
            const float r0 = fmaf(fpy, si.sf, fmaf(fpx, si.cf, si.base));
#pragma unroll
            for (int ry = 0; ry < kRY; ++ry) {
                const float rb = fmaf((float)(4 * ry), si.sf, r0);
#pragma unroll
                for (int rp = 0; rp < kRX / 2; ++rp) {
                    const float u0 = fmaf((float)(16 * rp), si.cf, rb);
                    const float u1 = fmaf((float)(16 * rp + 8), si.cf, rb);
                    const float2 tm = add2_rd(make_float2(u0, u1), magic2);
                    const float2 w0 = lds64(wb + (__float_as_uint(tm.x) << 3));
                    const float2 w1 = lds64(wb + (__float_as_uint(tm.y) << 3));
                    acc[ry][rp] = add2(acc[ry][rp], make_float2(fmaf(u0, w0.x, w0.y), fmaf(u1, w1.x, w1.y)));
                }
            }
        }
        if (more) commit(cur ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int ry = 0; ry < kRY; ++ry)
#pragma unroll
        for (int rp = 0; rp < kRX / 2; ++rp) {
            const int y = Y0 + py + 4 * ry;
            const int x0 = X0 + px + 16 * rp;
            if (y < ny) {
                const size_t k = (size_t)y * nx + x0;
                if (ystep) {
                    if (x0 < nx) out[k] = fmaf(-(weight * acc[ry][rp].x), invL, ystep[k]);
                    if (x0 + 8 < nx) out[k + 8] = fmaf(-(weight * acc[ry][rp].y), invL, ystep[k + 8]);
                } else {
                    if (x0 < nx) out[k] = weight * acc[ry][rp].x;
                    if (x0 + 8 < nx) out[k + 8] = weight * acc[ry][rp].y;
                }
            }
        }
}

template <int kNA, bool kResidual, bool kPartial>
__global__ void __launch_bounds__(kThreads, 3)
bp_kernel(const AngleInfo *__restrict__ tab, const float *__restrict__ srcA,
          const float *__restrict__ srcB, float *__restrict__ img, int n_angles, int n_bins,
          int nx, int ny, double cx, double cy, float weight, int tiles_x, const float *__restrict__ ystep,
          const float *__restrict__ invL) {
    const int slice = blockIdx.y;
    const size_t sino_off = (size_t)slice * n_angles * n_bins, img_off = (size_t)slice * nx * ny;
    bp_tile<kNA, kResidual, kPartial>(tab, srcA + sino_off, kResidual ? srcB + sino_off : nullptr, img + img_off,
                       n_angles, n_bins, nx, ny, cx, cy, weight, (blockIdx.x % tiles_x) * kTX,
                       (blockIdx.x / tiles_x) * kTY, ystep ? ystep + img_off : nullptr, ystep ? invL[slice] : 0.0f);
}

// Mixed batch: CTA k reconstructs tile (items[k].y, items[k].z) of slice items[k].x
// (the slices' angle counts differ, so the partial last blocks are walked short).
template <int kNA, bool kResidual>
__global__ void __launch_bounds__(kThreads, 3)
bp_batch_kernel(const BatchSlice *__restrict__ slices, const int4 *__restrict__ items, float weight_scale) {
    const int4 it = items[blockIdx.x];
    const BatchSlice s = slices[it.x];
    bp_tile<kNA, kResidual, true>(s.tab, s.bp_a, s.bp_b, s.bp_out, s.n_angles, s.n_bins, s.nx, s.ny, s.cx, s.cy,
                       weight_scale * s.pixel_size, it.y * kTX, it.z * kTY, s.bp_y, s.bp_y ? *s.bp_invL : 0.0f);
}

template <int kNA>
int launch_bp_batch_na(const BatchSlice *slices, const int4 *items, int n_items, bool residual, cudaStream_t st) {
    if (residual)
        bp_batch_kernel<kNA, true><<<n_items, kThreads, 0, st>>>(slices, items, 1.0f);
    else
        bp_batch_kernel<kNA, false><<<n_items, kThreads, 0, st>>>(slices, items, 1.0f);
    return cuda_status("batched back-projection kernel");
}

template <int kNA, bool kPartial>
void launch_bp_na_p(const pyhst_geometry *g, const AngleInfo *tab, BpSource src, float *img, float weight,
                    dim3 grid, int tiles_x, cudaStream_t st) {
    if (src.b)
        bp_kernel<kNA, true, kPartial><<<grid, kThreads, 0, st>>>(tab, src.a, src.b, img, g->n_angles, g->n_bins,
                                                                  g->nx, g->ny, g->cx, g->cy, weight, tiles_x, src.y,
                                                                  src.invL);
    else
        bp_kernel<kNA, false, kPartial><<<grid, kThreads, 0, st>>>(tab, src.a, nullptr, img, g->n_angles, g->n_bins,
                                                                   g->nx, g->ny, g->cx, g->cy, weight, tiles_x,
                                                                   src.y, src.invL);
}

// The short walk of a partial last block only where there is one: its loop
// bound is a run-time value, which costs a little on full blocks.
template <int kNA>
int launch_bp_na(const pyhst_geometry *g, const AngleInfo *tab, BpSource src, float *img, float weight, dim3 grid,
                 int tiles_x, cudaStream_t st) {
    if (g->n_angles % kNA)
        launch_bp_na_p<kNA, true>(g, tab, src, img, weight, grid, tiles_x, st);
    else
        launch_bp_na_p<kNA, false>(g, tab, src, img, weight, grid, tiles_x, st);
    return cuda_status("back-projection kernel");
}

}  // namespace

int bp_tiles(int nx, int ny, int *tx, int *ty) {
    *tx = (nx + kTX - 1) / kTX;
    *ty = (ny + kTY - 1) / kTY;
    return *tx * *ty;
}

bool bp_block_supported(int na) { return na == 8 || na == 16 || na == 24; }

int launch_backproject_batch(const BatchSlice *slices, const int4 *items, int n_items, bool residual,
                             cudaStream_t st, int angle_block) {
    if (n_items <= 0) return PYHST_OK;
    ProfScope prof(kProfBackproject, st);
    switch (angle_block) {
        case 8: return launch_bp_batch_na<8>(slices, items, n_items, residual, st);
        case 24: return launch_bp_batch_na<24>(slices, items, n_items, residual, st);
        default: return launch_bp_batch_na<16>(slices, items, n_items, residual, st);
    }
}

int launch_backproject(const pyhst_geometry *g, const AngleInfo *tab, BpSource src, float *img,
                       float weight, cudaStream_t st, int angle_block) {
    const int tiles_x = (g->nx + kTX - 1) / kTX;
    const int tiles_y = (g->ny + kTY - 1) / kTY;
    dim3 grid(tiles_x * tiles_y, g->n_slices);
    if (grid.y > 65535) return fail(PYHST_ERR_INVALID_ARG, "too many slices in one call (%d)", g->n_slices);
    if (angle_block <= 0) angle_block = bp_block_for(g->nx, g->ny, g->n_angles);
    ProfScope prof(kProfBackproject, st);
    switch (angle_block) {
        case 8: return launch_bp_na<8>(g, tab, src, img, weight, grid, tiles_x, st);
        case 24: return launch_bp_na<24>(g, tab, src, img, weight, grid, tiles_x, st);
        default: return launch_bp_na<16>(g, tab, src, img, weight, grid, tiles_x, st);
    }
}

namespace {
std::mutex g_bp_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_bp_tune;   // (device, nx, ny, n_angles) -> angles per block
}  // namespace

int bp_block_for(int nx, int ny, int n_angles) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bp_tune_mu);
    auto it = g_bp_tune.find(std::make_tuple(dev, nx, ny, n_angles));
    return it == g_bp_tune.end() ? 16 : it->second;
}

}  // namespace pyhst

extern "C" int pyhst_set_backproject_block(int32_t nx, int32_t ny, int32_t n_angles, int32_t angles_per_block) {
    using namespace pyhst;
    if (nx < 1 || ny < 1 || n_angles < 1) return fail(PYHST_ERR_INVALID_ARG, "image %d x %d, %d angles", nx, ny, n_angles);
    if (angles_per_block != 0 && !bp_block_supported(angles_per_block))
        return fail(PYHST_ERR_INVALID_ARG, "angles per block %d: need 8, 16 or 24 (0 clears)", angles_per_block);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status("cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_bp_tune_mu);
    const auto key = std::make_tuple(dev, (int)nx, (int)ny, (int)n_angles);
    if (angles_per_block == 0)
        g_bp_tune.erase(key);
    else
        g_bp_tune[key] = angles_per_block;
    return PYHST_OK;
}

extern "C" int pyhst_autotune_backproject(const pyhst_geometry *g, const float *sino, float *img, void *workspace,
                                          size_t ws_bytes, int32_t *best, pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if (!sino || !img) return fail(PYHST_ERR_INVALID_ARG, "sino/img pointer is NULL");
    const size_t need = pyhst_workspace_size(g, PYHST_OP_BACKPROJECT);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv(workspace, ws_bytes);
    AngleInfo *tab = cv.take<AngleInfo>(g->n_angles);
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_status("autotune events");
    }
    int pick = 16;
    float best_ms = 1e30f;
    for (int na : {8, 16, 24}) {
        if ((rc = launch_backproject(g, tab, BpSource{sino, nullptr}, img, 1.0f, st, na))) break;   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && !rc; ++r) rc = launch_backproject(g, tab, BpSource{sino, nullptr}, img, 1.0f, st, na);
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
            pick = na;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best) *best = pick;
    return pyhst_set_backproject_block(g->nx, g->ny, g->n_angles, pick);
}

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
