// Filtered back-projection with the paper's preprocessing variants (Sec. 2.3),
// in its order: dark/flat correction with flats interpolated in time, the
// hot-spot median filter, -ln, rearrangement into sinograms, the ring filter,
// then the Ram-Lak filter and back-projection of pyhst_fbp.
//
// For each chunk of slices a preprocessing kernel reads the raw radiography
// stack in place, forms r = (I - D) / (F(t) - D) for a sample and (with the
// hot-spot filter) its up to 8 neighbours in the (z, bin) plane of its
// projection, replaces r by the neighbours' median where that median is below
// r - threshold, and writes p = -ln(max(r, 1e-6)) as sinograms into the
// workspace.  The ring filter takes each sinogram's mean over angles s(b),
// subtracts its moving average (the high-pass part s - m), and removes that
// from every row.  The filter and back-projector then run as in pyhst_fbp.
// The hot-spot decision is taken in float32 (the kernel's precision).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pyhst {

size_t filter_table_bytes(int P);
int launch_filter_tables(int P, int filter, void *tables, cudaStream_t st);
int launch_filter(int kind, const void *data, int64_t slice_stride, int64_t angle_stride, const float *flat,
                  const float *dark, int z0, int n_slices_chunk, int n_angles, int n_bins, int P,
                  const void *tables, float *q, cudaStream_t st);
int default_pad(int n_bins);

namespace {

constexpr int kPreThreads = 256;

struct PreArgs {
    const void *data;
    int64_t ss, as;          // slice / angle strides of the raw stack (elements)
    const float *flats;      // [nf][nz][nb]
    const float *pos;        // [na] or NULL
    const float *dark;       // [nz][nb]
    int nf, nz, na, nb;
    float thr;
};

template <int kKind>
__device__ __forceinline__ float raw_at(const PreArgs &A, int z, int a, int b) {
    const int64_t i = (int64_t)z * A.ss + (int64_t)a * A.as + b;
    return kKind == PYHST_U16_RAW ? (float)static_cast<const uint16_t *>(A.data)[i]
                                  : static_cast<const float *>(A.data)[i];
}

// r = (I - D) / (F - D) at (z, a, b); 1 where F - D <= 0
template <int kKind>
__device__ __forceinline__ float ratio_at(const PreArgs &A, int z, int a, int b, int f0, float w) {
    const size_t k = (size_t)z * A.nb + b;
    float F = A.flats[(size_t)f0 * A.nz * A.nb + k];
    if (A.nf > 1) F = fmaf(w, A.flats[(size_t)(f0 + 1) * A.nz * A.nb + k] - F, F);
    const float D = A.dark[k];
    const float den = F - D;
    return den > 0.0f ? (raw_at<kKind>(A, z, a, b) - D) / den : 1.0f;
}

__device__ __forceinline__ void cswap(float &a, float &b) {
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

// p [chunk][na][nb] for slices z0 .. z0 + gridDim.z - 1
template <int kKind, bool kHot>
__global__ void __launch_bounds__(kPreThreads) pre_kernel(PreArgs A, int z0, float *__restrict__ p) {
    const int b = blockIdx.x * kPreThreads + threadIdx.x;
    const int a = blockIdx.y, zl = blockIdx.z, z = z0 + zl;
    if (b >= A.nb) return;
    float ps = A.nf > 1 ? A.pos[a] : 0.0f;
    ps = fminf(fmaxf(ps, 0.0f), (float)(A.nf - 1));
    int f0 = (int)floorf(ps);
    f0 = min(f0, max(A.nf - 2, 0));
    const float w = ps - (float)f0;
    float r = ratio_at<kKind>(A, z, a, b, f0, w);
    if (kHot) {
        float v[8];
        int n = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int db = -1; db <= 1; ++db) {
                if (dz == 0 && db == 0) continue;
                const int zz = z + dz, bb = b + db;
                const bool ok = zz >= 0 && zz < A.nz && bb >= 0 && bb < A.nb;
                v[n++] = ok ? ratio_at<kKind>(A, zz, a, bb, f0, w) : INFINITY;
            }
        int cnt = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int db = -1; db <= 1; ++db)
                if (!(dz == 0 && db == 0) && z + dz >= 0 && z + dz < A.nz && b + db >= 0 && b + db < A.nb) ++cnt;
        // sort the 8 values (missing neighbours are +inf, so the k present come first)
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 7 - i; ++j) cswap(v[j], v[j + 1]);
        float med = r;
        if (cnt > 0) {
            // v[cnt/2] and v[cnt/2 - 1] without dynamic register indexing
            float hi = v[0], lo = v[0];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i == cnt / 2) hi = v[i];
                if (i == cnt / 2 - 1) lo = v[i];
            }
            med = (cnt & 1) ? hi : 0.5f * (lo + hi);
        }
        if (med < r - A.thr) r = med;
    }
    p[((size_t)zl * A.na + a) * A.nb + b] = -logf(fmaxf(r, 1e-6f));
}

// ring: s(b) = mean over angles, hp(b) = s(b) - moving average of s; p -= hp
__global__ void ring_mean_kernel(const float *__restrict__ p, int na, int nb, float *__restrict__ s) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int zl = blockIdx.y;
    if (b >= nb) return;
    const float *P = p + (size_t)zl * na * nb;
    double acc = 0.0;
    for (int a = 0; a < na; ++a) acc += (double)P[(size_t)a * nb + b];
    s[(size_t)zl * nb + b] = (float)(acc / (double)na);
}

__global__ void ring_hp_kernel(const float *__restrict__ s, int nb, int h, float *__restrict__ hp) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int zl = blockIdx.y;
    if (b >= nb) return;
    const float *S = s + (size_t)zl * nb;
    double acc = 0.0;
    int cnt = 0;
    for (int c = max(0, b - h); c <= min(nb - 1, b + h); ++c) {
        acc += (double)S[c];
        ++cnt;
    }
    hp[(size_t)zl * nb + b] = (float)((double)S[b] - acc / (double)cnt);
}

__global__ void ring_sub_kernel(float *__restrict__ p, const float *__restrict__ hp, int na, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y, zl = blockIdx.z;
    if (b >= nb) return;
    p[((size_t)zl * na + a) * nb + b] -= hp[(size_t)zl * nb + b];
}

}  // namespace
}  // namespace pyhst

using namespace pyhst;

static size_t pre_bytes(const pyhst_geometry *g, int P, int S) {
    const size_t per_p = sizeof(float) * (size_t)g->n_angles * g->n_bins;
    return angle_table_bytes(g->n_angles) + filter_table_bytes(P) + align_up(per_p * S) /* q */ +
           align_up(per_p * S) /* p */ + 2 * align_up(sizeof(float) * (size_t)S * g->n_bins);
}

extern "C" size_t pyhst_fbp_pre_workspace_size(const pyhst_geometry *g, int32_t pad_len, int32_t slices_per_pass) {
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    const int P = pad_len == 0 ? default_pad(g->n_bins) : pad_len;
    if (P < 2 * g->n_bins || P > 16384 || (P & (P - 1)) || P < 64) return 0;
    return pre_bytes(g, P, std::max(1, std::min<int>(slices_per_pass, g->n_slices)));
}

extern "C" int pyhst_fbp_pre(const pyhst_geometry *g, int input_type, const void *data, int64_t slice_stride,
                             int64_t angle_stride, const float *dark, const pyhst_preproc *pre, int filter,
                             int32_t pad_len, float *out, void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    int rc = check_geometry(g);
    if (rc) return rc;
    if (input_type != PYHST_U16_RAW && input_type != PYHST_F32_RAW)
        return fail(PYHST_ERR_INVALID_ARG, "pyhst_fbp_pre needs raw counts (PYHST_U16_RAW or PYHST_F32_RAW)");
    if (filter < PYHST_RAMLAK || filter > PYHST_HANN) return fail(PYHST_ERR_INVALID_ARG, "unknown filter %d", filter);
    if (!data || !out || !dark || !pre || !pre->flats) return fail(PYHST_ERR_INVALID_ARG, "NULL pointer argument");
    if (pre->n_flats < 1 || (pre->n_flats > 1 && !pre->flat_pos))
        return fail(PYHST_ERR_INVALID_ARG, "n_flats >= 1, and flat_pos is needed for more than one flat");
    if (!(pre->hotspot_threshold >= 0.0f) || !std::isfinite(pre->hotspot_threshold))
        return fail(PYHST_ERR_INVALID_ARG, "hotspot_threshold must be >= 0");
    if (pre->ring_window != 0 && (pre->ring_window < 3 || !(pre->ring_window & 1)))
        return fail(PYHST_ERR_INVALID_ARG, "ring_window must be 0 or an odd number >= 3");
    const int P = pad_len == 0 ? default_pad(g->n_bins) : pad_len;
    if (P < 2 * g->n_bins || P > 16384 || (P & (P - 1)) || P < 64)
        return fail(PYHST_ERR_INVALID_ARG, "pad_len %d: need a power of two in [max(64, 2 n_bins), 16384]", P);
    const size_t per_p = sizeof(float) * (size_t)g->n_angles * g->n_bins;
    const size_t one = pre_bytes(g, P, 1);
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < one)
        return fail(PYHST_ERR_WORKSPACE, "workspace needs at least %zu bytes, 256-byte aligned", one);
    int S = 1;
    while (S < g->n_slices && pre_bytes(g, P, S + 1) <= ws_bytes) ++S;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv(workspace, ws_bytes);
    AngleInfo *tab = cv.take<AngleInfo>(g->n_angles);
    void *tables = cv.take<char>(filter_table_bytes(P));
    float *q = cv.take<float>(per_p / sizeof(float) * S);
    float *p = cv.take<float>(per_p / sizeof(float) * S);
    float *sbuf = cv.take<float>((size_t)S * g->n_bins);
    float *hp = cv.take<float>((size_t)S * g->n_bins);
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    if ((rc = launch_filter_tables(P, filter, tables, st))) return rc;

    PreArgs A;
    A.data = data; A.ss = slice_stride; A.as = angle_stride;
    A.flats = pre->flats; A.pos = pre->flat_pos; A.dark = dark;
    A.nf = pre->n_flats; A.nz = g->n_slices; A.na = g->n_angles; A.nb = g->n_bins;
    A.thr = pre->hotspot_threshold;
    const bool hot = pre->hotspot_threshold > 0.0f;
    const float weight = (float)(M_PI / ((double)g->n_angles * (double)g->pixel_size));
    const int bx = (g->n_bins + kPreThreads - 1) / kPreThreads;
    for (int z0 = 0; z0 < g->n_slices; z0 += S) {
        const int n = std::min(S, g->n_slices - z0);
        const dim3 grid(bx, g->n_angles, n);
        if (input_type == PYHST_U16_RAW) {
            if (hot) pre_kernel<PYHST_U16_RAW, true><<<grid, kPreThreads, 0, st>>>(A, z0, p);
            else pre_kernel<PYHST_U16_RAW, false><<<grid, kPreThreads, 0, st>>>(A, z0, p);
        } else {
            if (hot) pre_kernel<PYHST_F32_RAW, true><<<grid, kPreThreads, 0, st>>>(A, z0, p);
            else pre_kernel<PYHST_F32_RAW, false><<<grid, kPreThreads, 0, st>>>(A, z0, p);
        }
        if ((rc = cuda_status("preprocessing kernel"))) return rc;
        if (pre->ring_window > 0) {
            ring_mean_kernel<<<dim3(bx, n), kPreThreads, 0, st>>>(p, g->n_angles, g->n_bins, sbuf);
            ring_hp_kernel<<<dim3(bx, n), kPreThreads, 0, st>>>(sbuf, g->n_bins, (pre->ring_window - 1) / 2, hp);
            ring_sub_kernel<<<grid, kPreThreads, 0, st>>>(p, hp, g->n_angles, g->n_bins);
            if ((rc = cuda_status("ring filter kernels"))) return rc;
        }
        rc = launch_filter(PYHST_F32_SINO, p, (int64_t)g->n_angles * g->n_bins, g->n_bins, nullptr, nullptr, 0, n,
                           g->n_angles, g->n_bins, P, tables, q, st);
        if (rc) return rc;
        pyhst_geometry gc = *g;
        gc.n_slices = n;
        rc = launch_backproject(&gc, tab, BpSource{q, nullptr}, out + (size_t)z0 * g->nx * g->ny, weight, st);
        if (rc) return rc;
    }
    return PYHST_OK;
}
