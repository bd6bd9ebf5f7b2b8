// Filtered back-projection driver (Sec. 2.3) and workspace sizing.
//
// The stack is processed in chunks of slices: the fused normalise + filter
// kernel writes the chunk's filtered rows q [chunk][n_angles][n_bins] into the
// workspace (sized to stay L2-resident), then the back-projector reconstructs
// the chunk's slices from q.  The sinogram of a detector row is read in place
// from the radiography stack through the caller's strides, so no
// rearrangement pass is made.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pyhst {

size_t filter_table_bytes(int P);
int launch_filter_tables(int P, void *tables, cudaStream_t st);
int launch_filter(int kind, const void *data, int64_t slice_stride, int64_t angle_stride, const float *flat,
                  const float *dark, int z0, int n_slices_chunk, int n_angles, int n_bins, int P,
                  const void *tables, float *q, cudaStream_t st);
size_t tv_workspace_bytes(const pyhst_geometry *g, const pyhst_tv_opts *o);

static constexpr int kFbpDefaultChunk = 4;

int default_pad(int n_bins) {
    int P = 64;
    while (P < 2 * n_bins) P <<= 1;
    return P;
}

static size_t fbp_fixed_bytes(const pyhst_geometry *g, int P) {
    return angle_table_bytes(g->n_angles) + filter_table_bytes(P);
}

static size_t q_slice_bytes(const pyhst_geometry *g) {
    return sizeof(float) * (size_t)g->n_angles * g->n_bins;
}

}  // namespace pyhst

extern "C" size_t pyhst_workspace_size(const pyhst_geometry *g, int op) {
    using namespace pyhst;
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    switch (op) {
        case PYHST_OP_FBP: {
            const int P = default_pad(g->n_bins);
            const int S = g->n_slices < kFbpDefaultChunk ? g->n_slices : kFbpDefaultChunk;
            return fbp_fixed_bytes(g, P) + align_up(q_slice_bytes(g) * S);
        }
        case PYHST_OP_BACKPROJECT:
            return angle_table_bytes(g->n_angles);
        case PYHST_OP_PROJECT:
            return angle_table_bytes(g->n_angles) + project_scratch_bytes(g);
        case PYHST_OP_TV_SOLVE: {
            pyhst_tv_opts o{};
            return tv_workspace_bytes(g, &o);
        }
        default:
            return 0;
    }
}

extern "C" size_t pyhst_fbp_workspace_size(const pyhst_geometry *g, int32_t pad_len, int32_t slices_per_pass) {
    using namespace pyhst;
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    const int P = pad_len == 0 ? default_pad(g->n_bins) : pad_len;
    if (P < 2 * g->n_bins || P > 16384 || (P & (P - 1)) || P < 64) return 0;
    const int S = std::max(1, std::min<int>(slices_per_pass, g->n_slices));
    return fbp_fixed_bytes(g, P) + align_up(q_slice_bytes(g) * S);
}

extern "C" int pyhst_fbp(const pyhst_geometry *g, int input_type, const void *data, int64_t slice_stride,
                         int64_t angle_stride, const float *flat, const float *dark, int filter,
                         int32_t pad_len, float *out, void *workspace, size_t ws_bytes,
                         pyhst_stream_t stream) {
    using namespace pyhst;
    int rc = check_geometry(g);
    if (rc) return rc;
    if (input_type < PYHST_U16_RAW || input_type > PYHST_BF16_SINO)
        return fail(PYHST_ERR_INVALID_ARG, "unknown input kind %d", input_type);
    if (filter != PYHST_RAMLAK) return fail(PYHST_ERR_INVALID_ARG, "unknown filter %d", filter);
    if (!data || !out) return fail(PYHST_ERR_INVALID_ARG, "data/out pointer is NULL");
    const bool raw = input_type == PYHST_U16_RAW || input_type == PYHST_F32_RAW;
    if (raw && (!flat || !dark)) return fail(PYHST_ERR_INVALID_ARG, "raw input needs flat and dark fields");
    int P = pad_len;
    if (P == 0) P = default_pad(g->n_bins);
    if (P < 2 * g->n_bins || P > 16384 || (P & (P - 1)) || P < 64)
        return fail(PYHST_ERR_INVALID_ARG, "pad_len %d: need a power of two in [max(64, 2 n_bins), 16384]", P);
    const size_t fixed = fbp_fixed_bytes(g, P);
    const size_t per = q_slice_bytes(g);
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < fixed + align_up(per))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs at least %zu bytes, 256-byte aligned",
                    fixed + align_up(per));
    size_t room = ws_bytes - fixed;
    int S = (int)std::min<size_t>((size_t)g->n_slices, std::max<size_t>(1, (room - kAlign) / per));
    if (S < 1) S = 1;
    const float weight = (float)(M_PI / ((double)g->n_angles * (double)g->pixel_size));

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Carver cv(workspace, ws_bytes);
    AngleInfo *tab = cv.take<AngleInfo>(g->n_angles);
    void *tables = cv.take<char>(filter_table_bytes(P));
    float *q = cv.take<float>((size_t)S * g->n_angles * g->n_bins);
    if ((rc = launch_angle_table(g->angles, g->axis, g->n_angles, tab, st))) return rc;
    if ((rc = launch_filter_tables(P, tables, st))) return rc;
    for (int z0 = 0; z0 < g->n_slices; z0 += S) {
        const int n = std::min(S, g->n_slices - z0);
        rc = launch_filter(input_type, data, slice_stride, angle_stride, flat, dark, z0, n, g->n_angles,
                           g->n_bins, P, tables, q, st);
        if (rc) return rc;
        pyhst_geometry gc = *g;
        gc.n_slices = n;
        rc = launch_backproject(&gc, tab, BpSource{q, nullptr}, out + (size_t)z0 * g->nx * g->ny, weight, st);
        if (rc) return rc;
    }
    return PYHST_OK;
}
