// Estimators of beta without ground truth (Sec. 4).
//
// A beta scan reconstructs one slice for every beta of a grid in a single
// batched FISTA-TV solve (pyhst_tv_solve_batch, one item per beta), with the
// projection at one angle index held out, then evaluates
//   cross-validation:  || P_k x(beta) - y_k ||^2, the squared distance between
//                      the held-out data and the projection of the
//                      reconstruction at that angle;
//   decoherence:       E_cohe(beta) = Cos(I(beta) - I(0+), I(beta))  (Eq. 11),
//                      with I(0+) the reconstruction at the first beta of the
//                      grid (the caller puts a very small beta first).
// Both are float64 reductions in a fixed order.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kET = 256;

__device__ __forceinline__ double bsum(double v) {
    __shared__ double red[kET / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = (l < kET / 32) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// block b: cv[b] = sum_j (rows[b][j] - y[j])^2
__global__ void cv_kernel(const float *__restrict__ rows, const float *__restrict__ y, int nb, double *__restrict__ cv) {
    double a = 0.0;
    const float *r = rows + (size_t)blockIdx.x * nb;
    for (int j = threadIdx.x; j < nb; j += kET) {
        const double d = (double)r[j] - (double)y[j];
        a += d * d;
    }
    a = bsum(a);
    if (threadIdx.x == 0) cv[blockIdx.x] = a;
}

// block b: Cos(x_b - x_0, x_b)
__global__ void ecohe_kernel(const float *__restrict__ x, size_t n, double *__restrict__ out) {
    const float *xb = x + (size_t)blockIdx.x * n;
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (size_t k = threadIdx.x; k < n; k += kET) {
        const double b = xb[k];
        const double a = b - (double)x[k];
        ab += a * b;
        aa += a * a;
        bb += b * b;
    }
    ab = bsum(ab);
    aa = bsum(aa);
    bb = bsum(bb);
    if (threadIdx.x == 0) out[blockIdx.x] = (aa == 0.0 || bb == 0.0) ? NAN : ab / (sqrt(aa) * sqrt(bb));
}

struct ScanLayout {
    size_t red_ang, red_ax, red_sino, batch, tab1, xt, rows, bytes, batch_bytes;
};

ScanLayout scan_layout(const pyhst_geometry *g, int n_beta, int held_out, const pyhst_tv_opts *opts) {
    ScanLayout l{};
    const int na = held_out >= 0 ? g->n_angles - 1 : g->n_angles;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    l.red_ang = take(sizeof(float) * na);
    l.red_ax = take(sizeof(float) * na);
    l.red_sino = take(sizeof(float) * (size_t)na * g->n_bins);
    std::vector<pyhst_tv_item> items(n_beta);
    for (auto &it : items) {
        it.geom = *g;
        it.geom.n_angles = na;
        it.geom.n_slices = 1;
        it.geom.angles = reinterpret_cast<const float *>(1);   // same (placeholder) arrays for every item
        it.geom.axis = reinterpret_cast<const float *>(2);
        it.sino = nullptr; it.x = nullptr; it.energy = nullptr; it.gap = nullptr; it.beta = 0.0f;
    }
    l.batch_bytes = pyhst_tv_batch_workspace_size(items.data(), n_beta, opts);
    l.batch = take(l.batch_bytes);
    l.tab1 = take(sizeof(AngleInfo));
    {
        pyhst_geometry gk = *g;
        gk.n_angles = 1;
        gk.n_slices = n_beta;
        l.xt = take(project_scratch_bytes(&gk));
    }
    l.rows = take(sizeof(float) * (size_t)g->n_bins * n_beta);
    l.bytes = off;
    return l;
}

}  // namespace
}  // namespace pyhst

using namespace pyhst;

extern "C" size_t pyhst_beta_scan_workspace_size(const pyhst_geometry *g, int32_t n_beta, int32_t held_out,
                                                 const pyhst_tv_opts *opts) {
    if (!g || n_beta < 1 || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1) return 0;
    if (held_out >= g->n_angles || (held_out >= 0 && g->n_angles < 2)) return 0;
    return scan_layout(g, n_beta, held_out, opts).bytes;
}

extern "C" int pyhst_beta_scan(const pyhst_geometry *g, const float *sino, const float *betas, int32_t n_beta,
                               int32_t held_out, const pyhst_tv_opts *opts, float *x, double *cv, double *ecohe,
                               void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    pyhst_geometry g1 = g ? *g : pyhst_geometry{};
    g1.n_slices = 1;
    int rc = check_geometry(g ? &g1 : nullptr);
    if (rc) return rc;
    if (!sino || !x || !betas) return fail(PYHST_ERR_INVALID_ARG, "sino/x/betas pointer is NULL");
    if (n_beta < 1) return fail(PYHST_ERR_INVALID_ARG, "n_beta must be >= 1");
    if (held_out < -1 || held_out >= g->n_angles || (held_out >= 0 && g->n_angles < 2))
        return fail(PYHST_ERR_INVALID_ARG, "held_out %d: need -1 or an angle index (with >= 2 angles)", held_out);
    if (cv && held_out < 0) return fail(PYHST_ERR_INVALID_ARG, "cross-validation needs a held-out angle");
    for (int k = 0; k < n_beta; ++k)
        if (!(betas[k] >= 0.0f) || !std::isfinite(betas[k])) return fail(PYHST_ERR_INVALID_ARG, "beta %d invalid", k);
    if (!opts) return fail(PYHST_ERR_INVALID_ARG, "options are NULL");
    const ScanLayout L = scan_layout(g, n_beta, held_out, opts);
    if (!workspace || ws_bytes < L.bytes || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", L.bytes);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const int na = g->n_angles, nb = g->n_bins;
    const size_t N = (size_t)g->nx * g->ny;

    // the data with the projection at held_out removed
    pyhst_geometry gr = g1;
    const float *sino_r = sino;
    if (held_out >= 0) {
        float *ra = reinterpret_cast<float *>(ws + L.red_ang), *rx = reinterpret_cast<float *>(ws + L.red_ax);
        float *rs = reinterpret_cast<float *>(ws + L.red_sino);
        const int k = held_out, after = na - k - 1;
        if (k > 0) {
            cudaMemcpyAsync(ra, g->angles, sizeof(float) * k, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(rx, g->axis, sizeof(float) * k, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(rs, sino, sizeof(float) * (size_t)k * nb, cudaMemcpyDeviceToDevice, st);
        }
        if (after > 0) {
            cudaMemcpyAsync(ra + k, g->angles + k + 1, sizeof(float) * after, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(rx + k, g->axis + k + 1, sizeof(float) * after, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(rs + (size_t)k * nb, sino + (size_t)(k + 1) * nb, sizeof(float) * (size_t)after * nb,
                            cudaMemcpyDeviceToDevice, st);
        }
        if ((rc = cuda_status("held-out copies"))) return rc;
        gr.n_angles = na - 1;
        gr.angles = ra;
        gr.axis = rx;
        sino_r = rs;
    }
    std::vector<pyhst_tv_item> items(n_beta);
    for (int k = 0; k < n_beta; ++k) {
        items[k].geom = gr;
        items[k].sino = sino_r;
        items[k].x = x + (size_t)k * N;
        items[k].energy = nullptr;
        items[k].gap = nullptr;
        items[k].beta = betas[k];
    }
    rc = pyhst_tv_solve_batch(items.data(), n_beta, opts, nullptr, ws + L.batch, L.batch_bytes, stream);
    if (rc) return rc;

    if (cv) {
        pyhst_geometry gk = g1;
        gk.n_angles = 1;
        gk.angles = g->angles + held_out;
        gk.axis = g->axis + held_out;
        gk.n_slices = n_beta;
        AngleInfo *tab1 = reinterpret_cast<AngleInfo *>(ws + L.tab1);
        float *rows = reinterpret_cast<float *>(ws + L.rows);
        if ((rc = launch_angle_table(gk.angles, gk.axis, 1, tab1, st))) return rc;
        if ((rc = launch_project(&gk, tab1, x, rows, g->pixel_size, reinterpret_cast<float *>(ws + L.xt), st))) return rc;
        cv_kernel<<<n_beta, kET, 0, st>>>(rows, sino + (size_t)held_out * nb, nb, cv);
        if ((rc = cuda_status("cross-validation kernel"))) return rc;
    }
    if (ecohe) {
        ecohe_kernel<<<n_beta, kET, 0, st>>>(x, N, ecohe);
        if ((rc = cuda_status("decoherence kernel"))) return rc;
    }
    return PYHST_OK;
}
