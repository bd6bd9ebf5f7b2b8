// Filtered back-projection drivers (Sec. 2.3) and workspace sizing.
//
// The stack is processed in chunks of slices: the fused normalise + filter
// kernel writes the chunk's filtered rows q [chunk][n_angles][n_bins] into the
// workspace (a few slices, so q stays L2-resident), then the back-projector
// reconstructs the chunk's slices from q.  The sinogram of a detector row is
// read in place from the radiography stack through the caller's strides, so
// no rearrangement pass is made (Sec. 2.3 rearranges radiographies into
// sinograms; here that is only an indexing choice).
//
// pyhst_fbp_host streams host data through the device: chunks of slices are
// copied in on one stream, reconstructed on the caller's stream and copied
// out on a third, double-buffered so that copies overlap compute.
#include <algorithm>
#include <cmath>

#include <vector>

#include "common.cuh"

namespace pyhst {

size_t filter_table_bytes(int P);
int launch_filter_tables(int P, int filter, void *tables, cudaStream_t st);
int launch_filter(int kind, const void *data, int64_t slice_stride, int64_t angle_stride, const float *flat,
                  const float *dark, int z0, int n_slices_chunk, int n_angles, int n_bins, int P,
                  const void *tables, float *q, cudaStream_t st);
size_t tv_workspace_bytes(const pyhst_geometry *g, const pyhst_tv_opts *o);

static constexpr int kFbpDefaultChunk = 4;
// The host-streamed FBP filters and back-projects each copied chunk in one
// pass of up to this many slices (a 2048^2 slice is 1024 back-projection
// CTAs: 8 slices make 18.4 waves of 444, so the partly filled last wave
// costs less than with 4).
static constexpr int kFbpHostPass = 16;

int default_pad(int n_bins) {
    int P = 64;
    while (P < 2 * n_bins) P <<= 1;
    return P;
}

bool valid_pad(int P, int n_bins) { return P >= 2 * n_bins && P <= 16384 && !(P & (P - 1)) && P >= 64; }

static size_t q_slice_bytes(const pyhst_geometry *g) { return sizeof(float) * (size_t)g->n_angles * g->n_bins; }

static size_t fbp_fixed_bytes(const pyhst_geometry *g, int P) {
    return angle_table_bytes(g->n_angles) + filter_table_bytes(P);
}

static size_t input_elem_bytes(int kind) {
    switch (kind) {
        case PYHST_U16_RAW: case PYHST_F16_SINO: case PYHST_BF16_SINO: return 2;
        default: return 4;
    }
}

// Workspace carve of one FBP: angle table, filter tables, q for S slices.
struct FbpPlan {
    AngleInfo *tab;
    void *tables;
    float *q;
    int S, P, filter;
};

static int fbp_plan(const pyhst_geometry *g, int P, void *ws, size_t ws_bytes, FbpPlan *pl) {
    const size_t fixed = fbp_fixed_bytes(g, P), per = q_slice_bytes(g);
    if (!ws || ((uintptr_t)ws % kAlign) || ws_bytes < fixed + align_up(per))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs at least %zu bytes, 256-byte aligned", fixed + align_up(per));
    const size_t room = ws_bytes - fixed;
    pl->S = (int)std::min<size_t>({(size_t)g->n_slices, std::max<size_t>(1, room / per), (size_t)max_slices_per_pass(g->n_angles)});
    pl->P = P;
    Carver cv(ws, ws_bytes);
    pl->tab = cv.take<AngleInfo>(g->n_angles);
    pl->tables = cv.take<char>(filter_table_bytes(P));
    pl->q = cv.take<float>((size_t)pl->S * g->n_angles * g->n_bins);
    return PYHST_OK;
}

static int fbp_prepare(const pyhst_geometry *g, const FbpPlan &pl, cudaStream_t st) {
    int rc = launch_angle_table(g->angles, g->axis, g->n_angles, pl.tab, st);
    if (rc) return rc;
    return launch_filter_tables(pl.P, pl.filter, pl.tables, st);
}

// Reconstruct slices [0, g->n_slices) of `data` (z indices relative to data,
// flat and dark).
static int fbp_run(const pyhst_geometry *g, int kind, const void *data, int64_t ss, int64_t as,
                   const float *flat, const float *dark, const FbpPlan &pl, float *out, cudaStream_t st) {
    const float weight = (float)(M_PI / ((double)g->n_angles * (double)g->pixel_size));
    for (int z0 = 0; z0 < g->n_slices; z0 += pl.S) {
        const int n = std::min(pl.S, g->n_slices - z0);
        int rc = launch_filter(kind, data, ss, as, flat, dark, z0, n, g->n_angles, g->n_bins, pl.P, pl.tables,
                               pl.q, st);
        if (rc) return rc;
        pyhst_geometry gc = *g;
        gc.n_slices = n;
        rc = launch_backproject(&gc, pl.tab, BpSource{pl.q, nullptr}, out + (size_t)z0 * g->nx * g->ny, weight, st);
        if (rc) return rc;
    }
    return PYHST_OK;
}

int check_fbp_args(const pyhst_geometry *g, int kind, const void *data, const float *flat,
                          const float *dark, int filter, int *P, const void *out) {
    int rc = check_geometry(g);
    if (rc) return rc;
    if (kind < PYHST_U16_RAW || kind > PYHST_BF16_SINO) return fail(PYHST_ERR_INVALID_ARG, "unknown input kind %d", kind);
    if (filter < PYHST_RAMLAK || filter > PYHST_HANN) return fail(PYHST_ERR_INVALID_ARG, "unknown filter %d", filter);
    if (!data || !out) return fail(PYHST_ERR_INVALID_ARG, "data/out pointer is NULL");
    const bool raw = kind == PYHST_U16_RAW || kind == PYHST_F32_RAW;
    if (raw && (!flat || !dark)) return fail(PYHST_ERR_INVALID_ARG, "raw input needs flat and dark fields");
    if (*P == 0) *P = default_pad(g->n_bins);
    if (!valid_pad(*P, g->n_bins))
        return fail(PYHST_ERR_INVALID_ARG, "pad_len %d: need a power of two in [max(64, 2 n_bins), 16384]", *P);
    return PYHST_OK;
}

static size_t host_chunk_in_bytes(const pyhst_geometry *g, int kind, int S) {
    return align_up(input_elem_bytes(kind) * (size_t)S * g->n_angles * g->n_bins);
}
static size_t host_chunk_out_bytes(const pyhst_geometry *g, int S) {
    return align_up(sizeof(float) * (size_t)S * g->nx * g->ny);
}
static size_t host_chunk_field_bytes(const pyhst_geometry *g, int S) {
    return align_up(sizeof(float) * (size_t)S * g->n_bins);
}
static size_t host_plan_bytes(const pyhst_geometry *g, int P, int S) {
    pyhst_geometry gc = *g;
    gc.n_slices = S;
    return fbp_fixed_bytes(&gc, P) + align_up(q_slice_bytes(&gc) * std::min(S, kFbpHostPass));
}
static size_t fbp_host_bytes(const pyhst_geometry *g, int kind, int P, int S) {
    return host_plan_bytes(g, P, S) +
           2 * (host_chunk_in_bytes(g, kind, S) + host_chunk_out_bytes(g, S) + 2 * host_chunk_field_bytes(g, S));
}

}  // namespace pyhst

using namespace pyhst;

extern "C" size_t pyhst_workspace_size(const pyhst_geometry *g, int op) {
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    switch (op) {
        case PYHST_OP_FBP: {
            const int P = default_pad(g->n_bins);
            const int S = std::min(g->n_slices, kFbpDefaultChunk);
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
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    const int P = pad_len == 0 ? default_pad(g->n_bins) : pad_len;
    if (!valid_pad(P, g->n_bins)) return 0;
    const int S = std::max(1, std::min<int>(slices_per_pass, g->n_slices));
    return fbp_fixed_bytes(g, P) + align_up(q_slice_bytes(g) * S);
}

extern "C" int pyhst_fbp(const pyhst_geometry *g, int input_type, const void *data, int64_t slice_stride,
                         int64_t angle_stride, const float *flat, const float *dark, int filter,
                         int32_t pad_len, float *out, void *workspace, size_t ws_bytes,
                         pyhst_stream_t stream) {
    int P = pad_len;
    int rc = check_fbp_args(g, input_type, data, flat, dark, filter, &P, out);
    if (rc) return rc;
    FbpPlan pl;
    if ((rc = fbp_plan(g, P, workspace, ws_bytes, &pl))) return rc;
    pl.filter = filter;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = fbp_prepare(g, pl, st))) return rc;
    return fbp_run(g, input_type, data, slice_stride, angle_stride, flat, dark, pl, out, st);
}

// ------------------------------------------------------------------ filter only
extern "C" size_t pyhst_filter_workspace_size(const pyhst_geometry *g, int32_t pad_len) {
    if (!g || g->n_bins < 1) return 0;
    const int P = pad_len == 0 ? default_pad(g->n_bins) : pad_len;
    if (!valid_pad(P, g->n_bins)) return 0;
    return filter_table_bytes(P);
}

extern "C" int pyhst_filter(const pyhst_geometry *g, int input_type, const void *data, int64_t slice_stride,
                            int64_t angle_stride, const float *flat, const float *dark, int filter, int32_t pad_len,
                            float *q, void *workspace, size_t ws_bytes, pyhst_stream_t stream) {
    int P = pad_len;
    int rc = check_fbp_args(g, input_type, data, flat, dark, filter, &P, q);
    if (rc) return rc;
    const size_t need = filter_table_bytes(P);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = launch_filter_tables(P, filter, workspace, st))) return rc;
    // at most 2^30 rows per launch (the kernel's grid is rows / 2)
    const int per = std::max(1, (1 << 30) / g->n_angles);
    for (int z0 = 0; z0 < g->n_slices; z0 += per) {
        const int n = std::min(per, g->n_slices - z0);
        rc = launch_filter(input_type, data, slice_stride, angle_stride, flat, dark, z0, n, g->n_angles, g->n_bins,
                           P, workspace, q + (size_t)z0 * g->n_angles * g->n_bins, st);
        if (rc) return rc;
    }
    return PYHST_OK;
}

// ------------------------------------------------------------------ host-streamed FBP
// Chunk sizes of a host-streamed call on n slices with chunks of at most S:
// 1, 4, 16, ... (below S) at both ends and chunks of S between (a shorter one
// first), so that the first compute waits only for one slice's copy and the
// last copy back is one slice's, while every other copy is smaller than the
// compute it overlaps (a slice's copies take about a tenth of its FBP).
static std::vector<int> host_chunks(int n, int S) {
    std::vector<int> head;
    int left = n;
    for (int c = 1; c < S && left > 2 * c; c *= 4) {
        head.push_back(c);
        left -= 2 * c;
    }
    std::vector<int> out = head;
    if (left % S) out.push_back(left % S);
    for (int k = 0; k < left / S; ++k) out.push_back(S);
    out.insert(out.end(), head.rbegin(), head.rend());
    return out;
}

extern "C" size_t pyhst_fbp_host_workspace_size(const pyhst_geometry *g, int input_type, int32_t pad_len,
                                                int32_t slices_per_chunk) {
    if (!g || g->n_angles < 1 || g->n_bins < 1 || g->nx < 1 || g->ny < 1 || g->n_slices < 1) return 0;
    if (input_type < PYHST_U16_RAW || input_type > PYHST_BF16_SINO || slices_per_chunk < 1) return 0;
    const int P = pad_len == 0 ? default_pad(g->n_bins) : pad_len;
    if (!valid_pad(P, g->n_bins)) return 0;
    return fbp_host_bytes(g, input_type, P, std::min<int>(slices_per_chunk, g->n_slices));
}

extern "C" int pyhst_fbp_host(const pyhst_geometry *g, int input_type, const void *host_data, int64_t slice_stride,
                              int64_t angle_stride, const float *host_flat, const float *host_dark, int filter,
                              int32_t pad_len, float *host_out, int32_t slices_per_chunk, void *workspace,
                              size_t ws_bytes, pyhst_stream_t stream) {
    int P = pad_len;
    int rc = check_fbp_args(g, input_type, host_data, host_flat, host_dark, filter, &P, host_out);
    if (rc) return rc;
    if (slices_per_chunk < 1) return fail(PYHST_ERR_INVALID_ARG, "slices_per_chunk must be >= 1");
    const int S = std::min<int>(slices_per_chunk, g->n_slices);
    const size_t need = fbp_host_bytes(g, input_type, P, S);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign))
        return fail(PYHST_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    const bool raw = input_type == PYHST_U16_RAW || input_type == PYHST_F32_RAW;
    const size_t es = input_elem_bytes(input_type);
    const int na = g->n_angles, nb = g->n_bins;

    // carve: FBP plan for chunks of S slices, then two buffers of each chunk array
    pyhst_geometry gs = *g;
    gs.n_slices = S;
    const size_t plan_bytes = host_plan_bytes(g, P, S);
    FbpPlan pl;
    if ((rc = fbp_plan(&gs, P, workspace, plan_bytes, &pl))) return rc;
    pl.filter = filter;
    Carver cv(static_cast<char *>(workspace) + plan_bytes, ws_bytes - plan_bytes);
    char *in[2];
    float *outb[2], *fl[2], *dk[2];
    for (int b = 0; b < 2; ++b) {
        in[b] = cv.take<char>(host_chunk_in_bytes(g, input_type, S));
        outb[b] = cv.take<float>((size_t)S * g->nx * g->ny);
        fl[b] = cv.take<float>((size_t)S * nb);
        dk[b] = cv.take<float>((size_t)S * nb);
    }

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ready[2] = {}, done[2] = {}, drained[2] = {}, fin = nullptr, start = nullptr;
    auto cleanup = [&]() {
        // CUDA defers destroying streams and events that still have work pending
        for (int b = 0; b < 2; ++b) {
            if (ready[b]) cudaEventDestroy(ready[b]);
            if (done[b]) cudaEventDestroy(done[b]);
            if (drained[b]) cudaEventDestroy(drained[b]);
        }
        if (fin) cudaEventDestroy(fin);
        if (start) cudaEventDestroy(start);
        if (h2d) cudaStreamDestroy(h2d);
        if (d2h) cudaStreamDestroy(d2h);
    };
    bool ok = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&fin, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&ready[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&drained[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cleanup();
        return cuda_status("fbp_host stream/event creation");
    }
    // the copy streams start after the work already queued on the caller's stream
    cudaEventRecord(start, st);
    cudaStreamWaitEvent(h2d, start, 0);
    cudaStreamWaitEvent(d2h, start, 0);
    rc = fbp_prepare(&gs, pl, st);
    const char *src = static_cast<const char *>(host_data);
    const std::vector<int> chunks = host_chunks(g->n_slices, S);
    for (int i = 0, z0 = 0; !rc && i < (int)chunks.size(); z0 += chunks[i], ++i) {
        const int b = i & 1, n = chunks[i];
        if (i >= 2) cudaStreamWaitEvent(h2d, done[b], 0);   // compute has finished reading in[b]
        int64_t dss, das;                                     // strides of the device chunk
        if (slice_stride == nb) {
            // the chunk's slices are contiguous within each projection: one 2-D copy [na][n * nb]
            dss = nb;
            das = (int64_t)n * nb;
            cudaMemcpy2DAsync(in[b], (size_t)n * nb * es, src + (size_t)z0 * nb * es, (size_t)angle_stride * es,
                              (size_t)n * nb * es, na, cudaMemcpyHostToDevice, h2d);
        } else {
            // general strides: one 2-D copy per slice into [n][na][nb]
            dss = (int64_t)na * nb;
            das = nb;
            for (int z = 0; z < n; ++z)
                cudaMemcpy2DAsync(in[b] + (size_t)z * na * nb * es, (size_t)nb * es,
                                  src + (size_t)(z0 + z) * slice_stride * es, (size_t)angle_stride * es,
                                  (size_t)nb * es, na, cudaMemcpyHostToDevice, h2d);
        }
        if (raw) {
            cudaMemcpyAsync(fl[b], host_flat + (size_t)z0 * nb, sizeof(float) * n * nb, cudaMemcpyHostToDevice, h2d);
            cudaMemcpyAsync(dk[b], host_dark + (size_t)z0 * nb, sizeof(float) * n * nb, cudaMemcpyHostToDevice, h2d);
        }
        cudaEventRecord(ready[b], h2d);
        cudaStreamWaitEvent(st, ready[b], 0);
        if (i >= 2) cudaStreamWaitEvent(st, drained[b], 0);   // out[b] has been copied back
        pyhst_geometry gc = *g;
        gc.n_slices = n;
        rc = fbp_run(&gc, input_type, in[b], dss, das, fl[b], dk[b], pl, outb[b], st);
        cudaEventRecord(done[b], st);
        cudaStreamWaitEvent(d2h, done[b], 0);
        cudaMemcpyAsync(host_out + (size_t)z0 * g->nx * g->ny, outb[b], sizeof(float) * n * g->nx * g->ny,
                        cudaMemcpyDeviceToHost, d2h);
        cudaEventRecord(drained[b], d2h);
    }
    cudaEventRecord(fin, d2h);
    cudaStreamWaitEvent(st, fin, 0);   // completion is ordered on the caller's stream
    if (!rc) rc = cuda_status("fbp_host pipeline");
    cleanup();
    return rc;
}
