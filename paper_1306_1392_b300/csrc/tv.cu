// TV-penalised least squares (Eq. 3) by ISTA/FISTA (Sec. 3.1) with the
// isotropic TV (Eq. 2) prox computed by Chambolle's dual fixed point.
//
//   x_k = prox_{(beta/L) TV}( y_k - (1/L) P^T (P y_k - sino) )
//   FISTA: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, w_k = (t_k - 1) / t_{k+1},
//          y_{k+1} = x_k + w_k (x_k - x_{k-1});   ISTA: w_k = 0.
//   energy_k = 1/2 ||P x_k - sino||^2 + beta TV(x_k)   (Eq. 3, float64)
//
// Each iteration makes one projection and one back-projection: the solver
// projects x_k (which the energy needs anyway) and carries P y_{k+1} =
// P x_k + w_k (P x_k - P x_{k-1}) by linearity in sinogram space, keeping
// the residual P y_{k+1} - sino (formed by the update kernel), so the
// gradient step back-projects that residual directly (the back-projector
// writes z = y_k - g/L itself), and the last Chambolle launch writes x_k.  Reductions (energy,
// norms) are float64, per block then in fixed order: bitwise reproducible.
// L comes from the caller or from power iteration on P^T P started from the
// all-ones image (float64 norms), L = 1.01 * ||P v||^2 for the final unit v.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "chambolle.cuh"
#include "common.cuh"

namespace pyhst {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 256;  // partial sums per slice (= kRedThreads: one per finalize thread)

// ----------------------------------------------------------------- layout
struct TvLayout {
    size_t tab, xt, img[9], sino[3], scal, part[3], bytes;
};

// images: y, xa, xb, z, g, p1a, p2a, p1b, p2b; sinograms: Axa, Axb, Ry (the residual P y - sino);
// scalars per slice: L (double), invL, lam, invnorm (float)
TvLayout tv_layout(const pyhst_geometry *g) {
    TvLayout l{};
    const size_t S = (size_t)g->n_slices, N = (size_t)g->nx * g->ny, M = (size_t)g->n_angles * g->n_bins;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    l.tab = take(sizeof(AngleInfo) * g->n_angles);
    l.xt = take(project_scratch_bytes(g));
    for (auto &o : l.img) o = take(sizeof(float) * N * S);
    for (auto &o : l.sino) o = take(sizeof(float) * M * S);
    l.scal = take(sizeof(double) * 4 * S);
    for (auto &o : l.part) o = take(sizeof(double) * kRedBlocks * S);
    l.bytes = off;
    return l;
}

struct Scalars {   // per-slice solver scalars in the workspace
    double *L;     // [S]
    float *invL;   // [S]
    float *lam;    // [S] beta / L
    float *invn;   // [S] 1 / ||w|| of the power iteration
};

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = (l < kRedThreads / 32) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;   // valid in thread 0
}

// sum over the slice of (a - b)^2 (b may be NULL) -> part[slice][block]
__global__ void sqdiff_partial(const float *__restrict__ a, const float *__restrict__ b, size_t n,
                               double *__restrict__ part) {
    const size_t off = (size_t)blockIdx.y * n;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = b ? a[off + i] - b[off + i] : a[off + i];
        acc += (double)d * (double)d;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.y * kRedBlocks + blockIdx.x] = acc;
}

__device__ double sum_partials(const double *part) {
    double v = threadIdx.x < kRedBlocks ? part[blockIdx.x * kRedBlocks + threadIdx.x] : 0.0;
    return block_sum(v);
}

// mode 0: L = 1.01 * sum (power iteration end) and derived scalars;
// mode 1: invnorm = 1 / sqrt(sum)
__global__ void finalize_scalar(const double *__restrict__ part, Scalars sc, float beta, int mode,
                                int broadcast) {
    const double s = sum_partials(part);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            const double L = 1.01 * s;
            for (int k = 0; k < broadcast; ++k) {
                sc.L[k] = L;
                sc.invL[k] = (float)(1.0 / L);
                sc.lam[k] = (float)((double)beta / L);
            }
        } else {
            sc.invn[blockIdx.x] = (float)(1.0 / sqrt(s));
        }
    }
}

__global__ void set_lipschitz(Scalars sc, double L, float beta, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        sc.L[k] = L;
        sc.invL[k] = (float)(1.0 / L);
        sc.lam[k] = (float)((double)beta / L);
    }
}

__global__ void finalize_energy(const double *__restrict__ data_part, const double *__restrict__ tv_part,
                                float beta, double *__restrict__ energy, int n_iter, int k) {
    const double d = sum_partials(data_part);
    const double t = sum_partials(tv_part);
    if (threadIdx.x == 0 && energy) energy[(size_t)blockIdx.x * n_iter + k] = 0.5 * d + (double)beta * t;
}

__global__ void scale_kernel(const float *__restrict__ w, const float *__restrict__ invn, float *__restrict__ v,
                             size_t n) {
    const size_t off = (size_t)blockIdx.y * n;
    const float s = invn[blockIdx.y];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[off + i] = w[off + i] * s;
}

// r = a - b (element-wise, all slices)
__global__ void diff_kernel(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ r, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        r[i] = a[i] - b[i];
}

__global__ void fill_kernel(float *__restrict__ v, float val, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[i] = val;
}

// n_inner Chambolle steps in launches of up to K fused steps (see
// chambolle.cuh).  m is the launch's parity index: m = 0 starts from a zero
// field and writes the "a" buffers, m > 0 reads a (m odd) or b and writes the
// other, so a chain of launches with consecutive indices hands the field on.
template <int K>
__global__ void __launch_bounds__(kChThreads, kChMinBlocks)
chambolle_fused_kernel(const float *__restrict__ z, float *pa1, float *pa2, float *pb1, float *pb2,
                       const float *__restrict__ lam, float tau, int nx, int ny, int m, int steps, int tiles_x,
                       float *__restrict__ x, bool keep_p) {
    const size_t off = (size_t)blockIdx.y * nx * ny;
    const bool odd = m & 1;
    const float *s1 = (odd ? pa1 : pb1) + off, *s2 = (odd ? pa2 : pb2) + off;
    float *d1 = (m == 0 || !odd ? pa1 : pb1) + off, *d2 = (m == 0 || !odd ? pa2 : pb2) + off;
    constexpr int Th = chambolle_tile_h(K), Tw = chambolle_tile_w(K);
    chambolle_tile<K>(z + off, s1, s2, d1, d2, lam[blockIdx.y], tau, nx, ny, (blockIdx.x / tiles_x) * Th,
                      (blockIdx.x % tiles_x) * Tw, steps, m == 0, x ? x + off : nullptr, keep_p);
}

template <int K>
int launch_chambolle_k(const float *z, float *pa1, float *pa2, float *pb1, float *pb2, const float *lam, float tau,
                       int nx, int ny, int n_slices, int n_inner, bool *final_a, cudaStream_t st, float *x,
                       bool keep_p, int q0) {
    constexpr int Th = chambolle_tile_h(K), Tw = chambolle_tile_w(K);
    const int tx = (nx + Tw - 1) / Tw, ty = (ny + Th - 1) / Th;
    const int L = chambolle_launches(n_inner, K);
    for (int m = 0; m < L; ++m) {
        ProfScope prof(kProfChambolle, st);
        const int steps = chambolle_steps(n_inner, m, K);
        if (m + 1 == L && x) {
            // The prox x = z - lam div p of a tile reads p one row above and one
            // column left of it, so the last launch takes the halo of K + 1 steps
            // (tiles two rows and columns smaller); its <= K steps give the same bits.
            constexpr int Th1 = chambolle_tile_h(K + 1), Tw1 = chambolle_tile_w(K + 1);
            const int tx1 = (nx + Tw1 - 1) / Tw1, ty1 = (ny + Th1 - 1) / Th1;
            chambolle_fused_kernel<K + 1><<<dim3(tx1 * ty1, n_slices), kChThreads, kChSmem, st>>>(
                z, pa1, pa2, pb1, pb2, lam, tau, nx, ny, q0 + m, steps, tx1, x, keep_p);
        } else {
            chambolle_fused_kernel<K><<<dim3(tx * ty, n_slices), kChThreads, kChSmem, st>>>(
                z, pa1, pa2, pb1, pb2, lam, tau, nx, ny, q0 + m, steps, tx, nullptr, false);
        }
    }
    *final_a = ((q0 + L - 1) & 1) == 0;
    return cuda_status("Chambolle kernels");
}

// Enqueue n_inner steps with K fused steps per launch (K <= 0: the tuned or
// default choice for the size); returns through *final_a whether the dual
// field ends in the a buffers.  With x given, the last launch writes the prox
// x = z - lam div p there instead of the dual field (the divergence with
// the Neumann boundary of Eq. 2, then one fma), and with keep_p the final
// dual field as well.  q0 is the parity index of the first launch: 0 starts
// from a zero field; q0 > 0 starts from the field in the a buffers (q0 odd)
// or b, such as the field a previous chain kept.
int launch_chambolle(const float *z, float *pa1, float *pa2, float *pb1, float *pb2, const float *lam, float tau,
                     int nx, int ny, int n_slices, int n_inner, bool *final_a, cudaStream_t st, int K = 0,
                     float *x = nullptr, bool keep_p = false, int q0 = 0) {
    if (K <= 0) K = chambolle_k_for(nx, ny);
    PYHST_CHAMBOLLE_DISPATCH(K, launch_chambolle_k, z, pa1, pa2, pb1, pb2, lam, tau, nx, ny, n_slices, n_inner,
                             final_a, st, x, keep_p, q0)
}

// ROF duality gap of the prox (Eq. 2 with the quadratic term of the prox):
// for x = z - lam div p with |p| <= 1 pixelwise,
//   primal 1/2 ||x - z||^2 + lam TV(x)  -  dual 1/2 ||z||^2 - 1/2 ||x||^2
//     = lam TV(x) - <x, z - x> = lam (TV(x) + <p, grad x>)
// (z - x = lam div p and div = -grad^T), a sum of per-pixel terms
// |grad x| + p . grad x >= 0.  Summing those terms avoids the cancellation of
// the two nearly equal halves of the first form.  Partial of slice
// blockIdx.y per block (float32 terms in runs of 8, float64 beyond).
__global__ void gap_partial(const float *__restrict__ x, const float *__restrict__ p1, const float *__restrict__ p2,
                            int nx, int ny, double *__restrict__ part) {
    const size_t n = (size_t)nx * ny, off = (size_t)blockIdx.y * n;
    const float *X = x + off, *Q1 = p1 + off, *Q2 = p2 + off;
    RunSum rs;
    for (int i = blockIdx.x; i < ny; i += gridDim.x)
        for (int j = threadIdx.x; j < nx; j += blockDim.x) {
            const size_t k = (size_t)i * nx + j;
            const float v = X[k];
            const float d1 = (i + 1 < ny) ? X[k + nx] - v : 0.0f;
            const float d2 = (j + 1 < nx) ? X[k + 1] - v : 0.0f;
            rs.add(sqrtf(fmaf(d1, d1, d2 * d2)) + fmaf(Q1[k], d1, Q2[k] * d2));
        }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[blockIdx.y * kRedBlocks + blockIdx.x] = acc;
}

// gap[slice * stride + k] = lam[slice] * (sum of the slice's partials)
__global__ void finalize_gap(const double *__restrict__ part, const float *__restrict__ lam, double *__restrict__ gap,
                             int stride, int k) {
    const double s = sum_partials(part);
    if (threadIdx.x == 0) gap[(size_t)blockIdx.x * stride + k] = (double)lam[blockIdx.x] * s;
}

__global__ void zero_gap(double *__restrict__ gap, int S, int stride, int k) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < S) gap[(size_t)q * stride + k] = 0.0;
}

// data partial of ||Axn - b||^2 and the residual of the next y,
// ry = Ay - b with Ay = Axn + w (Axn - Axo) rounded to float32 first; the
// gradient step back-projects ry
__global__ void sino_update_kernel(const float *__restrict__ axn, const float *__restrict__ axo,
                                   const float *__restrict__ b, float *__restrict__ ry, float w, size_t n,
                                   double *__restrict__ part) {
    const size_t off = (size_t)blockIdx.y * n;
    RunSum rs;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = axn[off + i], bi = b[off + i];
        const float d = v - bi;
        rs.add(d * d);
        const float ay = fmaf(w, v - axo[off + i], v);
        ry[off + i] = ay - bi;
    }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[blockIdx.y * kRedBlocks + blockIdx.x] = acc;
}

// TV(xn) partial (Eq. 2) and y = xn + w (xn - xo)
__global__ void image_update_kernel(const float *__restrict__ xn, const float *__restrict__ xo,
                                    float *__restrict__ y, float w, int nx, int ny,
                                    double *__restrict__ part) {
    const size_t n = (size_t)nx * ny, off = (size_t)blockIdx.y * n;
    const float *X = xn + off;
    RunSum rs;
    for (int i = blockIdx.x; i < ny; i += gridDim.x)      // block: rows; threads: columns
        for (int j = threadIdx.x; j < nx; j += blockDim.x) {
            const size_t k = (size_t)i * nx + j;
            const float v = X[k];
            const float d1 = (i + 1 < ny) ? X[k + nx] - v : 0.0f;
            const float d2 = (j + 1 < nx) ? X[k + 1] - v : 0.0f;
            rs.add(sqrtf(d1 * d1 + d2 * d2));
            y[off + k] = fmaf(w, v - xo[off + k], v);
        }
    const double acc = block_sum(rs.total());
    if (threadIdx.x == 0) part[blockIdx.y * kRedBlocks + blockIdx.x] = acc;
}

struct Bufs {
    AngleInfo *tab;
    float *xt;
    float *img[9];
    float *sino[3];
    Scalars sc;
    double *part[3];
};

Bufs carve(const pyhst_geometry *g, void *ws) {
    const TvLayout l = tv_layout(g);
    char *b = static_cast<char *>(ws);
    Bufs r;
    r.tab = reinterpret_cast<AngleInfo *>(b + l.tab);
    r.xt = reinterpret_cast<float *>(b + l.xt);
    for (int i = 0; i < 9; ++i) r.img[i] = reinterpret_cast<float *>(b + l.img[i]);
    for (int i = 0; i < 3; ++i) r.sino[i] = reinterpret_cast<float *>(b + l.sino[i]);
    double *sc = reinterpret_cast<double *>(b + l.scal);
    const int S = g->n_slices;
    r.sc.L = sc;
    r.sc.invL = reinterpret_cast<float *>(sc + S);
    r.sc.lam = r.sc.invL + S;
    r.sc.invn = r.sc.lam + S;
    for (int i = 0; i < 3; ++i) r.part[i] = reinterpret_cast<double *>(b + l.part[i]);
    return r;
}

}  // namespace

size_t tv_workspace_bytes(const pyhst_geometry *g, const pyhst_tv_opts *) {
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    return tv_layout(g).bytes;
}

int check_tv_opts(const pyhst_tv_opts *o) {
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

// Optional changes to the iteration: a learned prox in place of the TV prox
// (the residual CNN of cnn.cu), and copies of the prox input z at chosen
// iterations.
struct SolveHooks {
    const float *cnn_params = nullptr;     // non-NULL: x_k = CNN(z_k)
    void *cnn_ws = nullptr;
    int n_capture = 0;
    const int32_t *capture_iters = nullptr; // host, 1-based iteration numbers
    float *capture = nullptr;              // [n_capture][n_slices][ny][nx]
};

// Enqueue the whole solve on `st`.
int tv_solve_enqueue(const pyhst_geometry *g, const float *sino, const pyhst_tv_opts *o, float *x,
                     double *energy, double *lip_out, void *ws, cudaStream_t st, const SolveHooks &hk = SolveHooks(),
                     double *gap = nullptr) {
    int rc;
    Bufs B = carve(g, ws);
    const int S = g->n_slices;
    const size_t N = (size_t)g->nx * g->ny, M = (size_t)g->n_angles * g->n_bins;
    const float s = g->pixel_size;
    float *y = B.img[0], *xa = B.img[1], *xb = B.img[2], *z = B.img[3], *gr = B.img[4];
    float *p1a = B.img[5], *p2a = B.img[6], *p1b = B.img[7], *p2b = B.img[8];
    float *Axa = B.sino[0], *Axb = B.sino[1], *Ry = B.sino[2];
    // reduction kernels always run kRedBlocks blocks per slice (every partial is written)
    const dim3 eg(kRedBlocks, S), sg(kRedBlocks, S);

    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, B.tab, st))) return rc;

    // ---- step size
    if (o->lipschitz > 0.0) {
        set_lipschitz<<<(S + 127) / 128, 128, 0, st>>>(B.sc, o->lipschitz, o->beta, S);
    } else {
        // the operator is the same for every slice: iterate on slice 0 only
        pyhst_geometry g1 = *g;
        g1.n_slices = 1;
        const dim3 rg1(kRedBlocks, 1), eg1(kRedBlocks, 1);
        fill_kernel<<<256, 256, 0, st>>>(z, 1.0f, N);
        for (int it = 0; it < o->n_power_iter; ++it) {
            if ((rc = launch_project(&g1, B.tab, z, Axa, s, B.xt, st))) return rc;
            if ((rc = launch_backproject(&g1, B.tab, BpSource{Axa, nullptr}, gr, s, st))) return rc;
            sqdiff_partial<<<rg1, kRedThreads, 0, st>>>(gr, nullptr, N, B.part[0]);
            finalize_scalar<<<1, kRedThreads, 0, st>>>(B.part[0], B.sc, o->beta, 1, 0);
            scale_kernel<<<eg1, kRedThreads, 0, st>>>(gr, B.sc.invn, z, N);
        }
        if ((rc = launch_project(&g1, B.tab, z, Axa, s, B.xt, st))) return rc;
        sqdiff_partial<<<rg1, kRedThreads, 0, st>>>(Axa, nullptr, M, B.part[0]);
        finalize_scalar<<<1, kRedThreads, 0, st>>>(B.part[0], B.sc, o->beta, 0, S);
    }
    if (lip_out) cudaMemcpyAsync(lip_out, B.sc.L, sizeof(double) * S, cudaMemcpyDeviceToDevice, st);
    if ((rc = cuda_status("step-size kernels"))) return rc;

    // ---- start: x_0 = x (warm) or 0; y_1 = x_0; P y_1 = P x_0
    float *xo = xa, *xn = xb, *Axo = Axa, *Axn = Axb;
    if (o->warm_start) {
        cudaMemcpyAsync(xo, x, sizeof(float) * N * S, cudaMemcpyDeviceToDevice, st);
        if ((rc = launch_project(g, B.tab, xo, Axo, s, B.xt, st))) return rc;
    } else {
        cudaMemsetAsync(xo, 0, sizeof(float) * N * S, st);
        cudaMemsetAsync(Axo, 0, sizeof(float) * M * S, st);
    }
    cudaMemcpyAsync(y, xo, sizeof(float) * N * S, cudaMemcpyDeviceToDevice, st);
    diff_kernel<<<256, 256, 0, st>>>(Axo, sino, Ry, M * S);   // P y_1 - sino
    if ((rc = cuda_status("solver start"))) return rc;

    double t = 1.0;
    bool dual_a = true;   // where the last prox left its dual field
    for (int k = 0; k < o->n_iter; ++k) {
        // gradient step: z = y - (1/L) P^T (P y - sino)
        if ((rc = launch_backproject(g, B.tab, BpSource{Ry, nullptr, y, B.sc.invL}, z, s, st))) return rc;
        for (int c = 0; c < hk.n_capture; ++c)
            if (hk.capture_iters[c] == k + 1)
                cudaMemcpyAsync(hk.capture + (size_t)c * N * S, z, sizeof(float) * N * S, cudaMemcpyDeviceToDevice, st);
        // prox of (beta/L) TV, or the learned prox
        if (hk.cnn_params) {
            if ((rc = cnn_forward(hk.cnn_params, z, xn, S, g->ny, g->nx, hk.cnn_ws, st))) return rc;
        } else if (o->beta > 0.0f) {
            // warm_dual: after the first prox, start from the field the previous
            // one kept (q0 = 1 reads the a buffers, 2 the b buffers)
            const int q0 = (o->warm_dual && k > 0) ? (dual_a ? 1 : 2) : 0;
            bool fa;
            if ((rc = launch_chambolle(z, p1a, p2a, p1b, p2b, B.sc.lam, o->tau, g->nx, g->ny, S, o->n_inner, &fa, st,
                                       0, xn, gap != nullptr || o->warm_dual, q0)))
                return rc;
            dual_a = fa;
            if (gap) {
                gap_partial<<<eg, kRedThreads, 0, st>>>(xn, fa ? p1a : p1b, fa ? p2a : p2b, g->nx, g->ny, B.part[2]);
                finalize_gap<<<S, kRedThreads, 0, st>>>(B.part[2], B.sc.lam, gap, o->n_iter, k);
            }
        } else {
            cudaMemcpyAsync(xn, z, sizeof(float) * N * S, cudaMemcpyDeviceToDevice, st);
            if (gap) zero_gap<<<(S + 127) / 128, 128, 0, st>>>(gap, S, o->n_iter, k);   // the identity prox
        }
        if ((rc = cuda_status("prox kernels"))) return rc;
        if ((rc = launch_project(g, B.tab, xn, Axn, s, B.xt, st))) return rc;
        double w = 0.0;
        if (o->use_fista) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            w = (t - 1.0) / tn;
            t = tn;
        }
        sino_update_kernel<<<sg, kRedThreads, 0, st>>>(Axn, Axo, sino, Ry, (float)w, M, B.part[0]);
        image_update_kernel<<<eg, kRedThreads, 0, st>>>(xn, xo, y, (float)w, g->nx, g->ny, B.part[1]);
        finalize_energy<<<S, kRedThreads, 0, st>>>(B.part[0], B.part[1], o->beta, energy, o->n_iter, k);
        if ((rc = cuda_status("update kernels"))) return rc;
        std::swap(xn, xo);
        std::swap(Axn, Axo);
    }
    cudaMemcpyAsync(x, xo, sizeof(float) * N * S, cudaMemcpyDeviceToDevice, st);
    return cuda_status("solver result copy");
}

size_t tv_prox_workspace_bytes(int nx, int ny, int n_slices) {
    if (nx < 1 || ny < 1 || n_slices < 1) return 0;
    return 4 * align_up(sizeof(float) * (size_t)nx * ny * n_slices) + align_up(sizeof(float) * n_slices) +
           align_up(sizeof(double) * kRedBlocks * n_slices);
}

__global__ void fill_lam(float *lam, float v, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) lam[k] = v;
}

int tv_prox_enqueue(const float *z, int nx, int ny, int S, float lam, int n_inner, float tau, float *x, void *ws,
                    cudaStream_t st, double *gap = nullptr) {
    Carver cv(ws, tv_prox_workspace_bytes(nx, ny, S));
    const size_t n = (size_t)nx * ny * S;
    float *p1a = cv.take<float>(n), *p2a = cv.take<float>(n), *p1b = cv.take<float>(n), *p2b = cv.take<float>(n);
    float *lamd = cv.take<float>(S);
    double *part = cv.take<double>((size_t)kRedBlocks * S);
    if (lam == 0.0f) {
        cudaMemcpyAsync(x, z, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
        if (gap) zero_gap<<<(S + 127) / 128, 128, 0, st>>>(gap, S, 1, 0);   // the identity prox
        return cuda_status("prox copy");
    }
    fill_lam<<<(S + 127) / 128, 128, 0, st>>>(lamd, lam, S);
    bool fa;
    int rc = launch_chambolle(z, p1a, p2a, p1b, p2b, lamd, tau, nx, ny, S, n_inner, &fa, st, 0, x, gap != nullptr);
    if (rc) return rc;
    if (gap) {
        gap_partial<<<dim3(kRedBlocks, S), kRedThreads, 0, st>>>(x, fa ? p1a : p1b, fa ? p2a : p2b, nx, ny, part);
        finalize_gap<<<S, kRedThreads, 0, st>>>(part, lamd, gap, 1, 0);
    }
    return cuda_status("prox kernels");
}

}  // namespace pyhst

extern "C" size_t pyhst_tv_workspace_size(const pyhst_geometry *g, const pyhst_tv_opts *opts) {
    return pyhst::tv_workspace_bytes(g, opts);
}

extern "C" int pyhst_tv_solve(const pyhst_geometry *g, const float *sino, const pyhst_tv_opts *opts, float *x,
                              double *energy, double *gap, double *lipschitz_out, void *workspace, size_t ws_bytes,
                              pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if ((rc = check_tv_opts(opts))) return rc;
    if (!sino || !x) return fail(PYHST_ERR_INVALID_ARG, "sino/x pointer is NULL");
    const size_t need = tv_workspace_bytes(g, opts);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    return tv_solve_enqueue(g, sino, opts, x, energy, lipschitz_out, workspace,
                            reinterpret_cast<cudaStream_t>(stream), SolveHooks(), gap);
}

extern "C" size_t pyhst_tv_prox_workspace_size(int32_t nx, int32_t ny, int32_t n_slices) {
    return pyhst::tv_prox_workspace_bytes(nx, ny, n_slices);
}

extern "C" int pyhst_tv_prox(const float *z, int32_t nx, int32_t ny, int32_t n_slices, float lam, int32_t n_inner,
                             float tau, float *x, double *gap, void *workspace, size_t ws_bytes,
                             pyhst_stream_t stream) {
    using namespace pyhst;
    if (!z || !x) return fail(PYHST_ERR_INVALID_ARG, "z/x pointer is NULL");
    if (nx < 1 || ny < 1 || n_slices < 1 || nx > 16384 || ny > 16384 || n_slices > 65535)
        return fail(PYHST_ERR_INVALID_ARG, "image %d x %d x %d out of range", nx, ny, n_slices);
    if (!(lam >= 0.0f) || !std::isfinite(lam)) return fail(PYHST_ERR_INVALID_ARG, "lam must be >= 0");
    if (n_inner < 1) return fail(PYHST_ERR_INVALID_ARG, "n_inner must be >= 1");
    if (!(tau > 0.0f && tau <= 0.25f)) return fail(PYHST_ERR_INVALID_ARG, "tau must be in (0, 1/4]");
    {   // every launch reads z around its tiles while the last one writes x
        const uintptr_t bytes = sizeof(float) * (size_t)nx * ny * n_slices;
        const uintptr_t xa = reinterpret_cast<uintptr_t>(x), za = reinterpret_cast<uintptr_t>(z);
        if (xa < za + bytes && za < xa + bytes) return fail(PYHST_ERR_INVALID_ARG, "x overlaps z");
    }
    const size_t need = tv_prox_workspace_bytes(nx, ny, n_slices);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    return tv_prox_enqueue(z, nx, ny, n_slices, lam, n_inner, tau, x, workspace,
                           reinterpret_cast<cudaStream_t>(stream), gap);
}

extern "C" int pyhst_tv_solve_capture(const pyhst_geometry *g, const float *sino, const pyhst_tv_opts *opts, float *x,
                                      int32_t n_capture, const int32_t *capture_iters, float *capture,
                                      void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if ((rc = check_tv_opts(opts))) return rc;
    if (!sino || !x) return fail(PYHST_ERR_INVALID_ARG, "sino/x pointer is NULL");
    if (n_capture < 0 || (n_capture > 0 && (!capture_iters || !capture)))
        return fail(PYHST_ERR_INVALID_ARG, "captures need iteration numbers and an output buffer");
    for (int c = 0; c < n_capture; ++c)
        if (capture_iters[c] < 1 || capture_iters[c] > opts->n_iter)
            return fail(PYHST_ERR_INVALID_ARG, "capture iteration %d outside [1, n_iter]", capture_iters[c]);
    const size_t need = tv_workspace_bytes(g, opts);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    SolveHooks hk;
    hk.n_capture = n_capture;
    hk.capture_iters = capture_iters;
    hk.capture = capture;
    return tv_solve_enqueue(g, sino, opts, x, nullptr, nullptr, workspace, reinterpret_cast<cudaStream_t>(stream), hk);
}

namespace {
pyhst_tv_opts pnp_opts(const pyhst_tv_opts *o) {
    pyhst_tv_opts r = *o;
    r.beta = 0.0f;          // no functional: the energy is the data term 1/2 ||sino - P x||^2
    r.n_inner = 1;
    r.tau = 0.125f;
    return r;
}
}  // namespace

extern "C" size_t pyhst_pnp_workspace_size(const pyhst_geometry *g) {
    using namespace pyhst;
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    const size_t c = cnn_workspace_size(g->n_slices, g->ny, g->nx);
    if (!c) return 0;
    return align_up(tv_workspace_bytes(g, nullptr)) + c;
}

extern "C" int pyhst_pnp_solve(const pyhst_geometry *g, const float *sino, const float *params,
                               const pyhst_tv_opts *opts, float *x, double *energy, double *lipschitz_out,
                               void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if (!opts) return fail(PYHST_ERR_INVALID_ARG, "options are NULL");
    const pyhst_tv_opts o = pnp_opts(opts);
    if ((rc = check_tv_opts(&o))) return rc;
    if (!sino || !x || !params) return fail(PYHST_ERR_INVALID_ARG, "sino/x/params pointer is NULL");
    if (g->n_slices > 65535) return fail(PYHST_ERR_INVALID_ARG, "n_slices %d > 65535", g->n_slices);
    const size_t need = pyhst_pnp_workspace_size(g);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    SolveHooks hk;
    hk.cnn_params = params;
    hk.cnn_ws = static_cast<char *>(workspace) + align_up(tv_workspace_bytes(g, nullptr));
    return tv_solve_enqueue(g, sino, &o, x, energy, lipschitz_out, workspace, reinterpret_cast<cudaStream_t>(stream),
                            hk);
}

namespace pyhst {

// ----------------------------------------------------------------- autotuned K
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tune;   // (device, nx, ny) -> steps fused per launch

int chambolle_k_for(int nx, int ny) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto f = g_tune.find(std::make_tuple(dev, nx, ny));
    return f == g_tune.end() ? kChKDefault : f->second;
}

void chambolle_k_set(int nx, int ny, int K) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (K <= 0)
        g_tune.erase(std::make_tuple(dev, nx, ny));
    else
        g_tune[std::make_tuple(dev, nx, ny)] = K;
}

}  // namespace pyhst

extern "C" int pyhst_set_tv_prox_steps(int32_t nx, int32_t ny, int32_t steps) {
    using namespace pyhst;
    if (nx < 1 || ny < 1) return fail(PYHST_ERR_INVALID_ARG, "image size must be positive");
    if (steps > 0 && !chambolle_k_supported(steps))
        return fail(PYHST_ERR_INVALID_ARG, "steps per launch %d: supported 2, 3, 4, 5, 6, 8 (0 clears)", steps);
    chambolle_k_set(nx, ny, steps);
    return PYHST_OK;
}

extern "C" int pyhst_autotune_tv_prox(const float *z, int32_t nx, int32_t ny, int32_t n_slices, float lam,
                                      int32_t n_inner, float tau, void *workspace, size_t ws_bytes,
                                      int32_t *best_steps, pyhst_stream_t stream) {
    using namespace pyhst;
    if (!z || !best_steps) return fail(PYHST_ERR_INVALID_ARG, "z/best_steps pointer is NULL");
    if (nx < 1 || ny < 1 || n_slices < 1 || nx > 16384 || ny > 16384 || n_slices > 65535)
        return fail(PYHST_ERR_INVALID_ARG, "image %d x %d x %d out of range", nx, ny, n_slices);
    if (!(lam >= 0.0f) || !std::isfinite(lam)) return fail(PYHST_ERR_INVALID_ARG, "lam must be >= 0");
    if (n_inner < 1) return fail(PYHST_ERR_INVALID_ARG, "n_inner must be >= 1");
    if (!(tau > 0.0f && tau <= 0.25f)) return fail(PYHST_ERR_INVALID_ARG, "tau must be in (0, 1/4]");
    const size_t need = tv_prox_workspace_bytes(nx, ny, n_slices);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t img = align_up(sizeof(float) * (size_t)nx * ny * n_slices);
    char *b = static_cast<char *>(workspace);
    float *p1a = reinterpret_cast<float *>(b), *p2a = reinterpret_cast<float *>(b + img);
    float *p1b = reinterpret_cast<float *>(b + 2 * img), *p2b = reinterpret_cast<float *>(b + 3 * img);
    float *lamd = reinterpret_cast<float *>(b + 4 * img);
    fill_lam<<<(n_slices + 127) / 128, 128, 0, st>>>(lamd, lam, n_slices);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand[] = {2, 3, 4, 5, 6, 8};
    int best = kChKDefault;
    float best_ms = 1e30f;
    int rc = PYHST_OK;
    for (int K : cand) {
        bool fa;
        if ((rc = launch_chambolle(z, p1a, p2a, p1b, p2b, lamd, tau, nx, ny, n_slices, n_inner, &fa, st, K))) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && !rc; ++r)
            rc = launch_chambolle(z, p1a, p2a, p1b, p2b, lamd, tau, nx, ny, n_slices, n_inner, &fa, st, K);
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
            best = K;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    chambolle_k_set(nx, ny, best);
    *best_steps = best;
    return PYHST_OK;
}
