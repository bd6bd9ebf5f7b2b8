// Opt-in per-kernel timing with CUDA events on the launch stream.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace pyhst {
namespace {

struct Record {
    int kind;
    cudaEvent_t a, b;
};

thread_local bool g_on = false;
thread_local std::vector<Record> g_recs;
thread_local std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

const char *kNames[kProfKinds] = {"backproject", "filter", "project", "chambolle"};

}  // namespace

ProfScope::ProfScope(int k, cudaStream_t s) : kind(k), st(s), end(nullptr), flags(cudaEventRecordDefault) {
    if (!g_on) return;
    cudaEvent_t a = get_event(), b = get_event();
    if (!a || !b) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        flags = cudaEventRecordExternal;   // an event-record node of the captured graph
    cudaEventRecordWithFlags(a, st, flags);
    g_recs.push_back(Record{kind, a, b});
    end = reinterpret_cast<void *>(b);
}

ProfScope::~ProfScope() {
    if (end) cudaEventRecordWithFlags(reinterpret_cast<cudaEvent_t>(end), st, flags);
}

}  // namespace pyhst

extern "C" int pyhst_profile_enable(int on) {
    pyhst::g_on = on != 0;
    return PYHST_OK;
}

extern "C" int pyhst_profile_read(const char *kernel, double *total_ms, int64_t *launches) {
    using namespace pyhst;
    int kind = -1;
    for (int k = 0; k < kProfKinds; ++k)
        if (kernel && std::strcmp(kernel, kNames[k]) == 0) kind = k;
    if (kind < 0 || !total_ms || !launches) return fail(PYHST_ERR_INVALID_ARG, "unknown kernel name");
    double ms = 0.0;
    int64_t n = 0;
    std::vector<Record> keep;
    for (const Record &r : g_recs) {
        if (r.kind != kind) {
            keep.push_back(r);
            continue;
        }
        if (cudaEventSynchronize(r.b) != cudaSuccess) return cuda_status("profile event");
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return cuda_status("profile event");
        ms += t;
        ++n;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.swap(keep);
    *total_ms = ms;
    *launches = n;
    return PYHST_OK;
}
