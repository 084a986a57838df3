// prof.cu -- opt-in CUDA-event timing of every kernel class the library launches
// (rqrcp_profile_begin / rqrcp_profile_end).  Host code only.
#include <vector>

#include "internal.cuh"

namespace rq {
namespace {

struct Record {
    int cls;
    cudaEvent_t e0, e1;
    double flops, bytes;
};

bool g_on = false;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;
int g_open_cls = -1;
cudaEvent_t g_open_ev = nullptr;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

const char* const kNames[RQRCP_PROFILE_CLASSES] = {
    "omega", "sketch_gemm", "sketch_reduce", "pivot", "swap", "panel",
    "wy_gemm_tn", "tform", "reduce_y", "wy_update", "bupdate", "lowrank_misc", "backward", "batched",
};

}  // namespace

bool prof_on() { return g_on; }

void prof_begin(int cls, cudaStream_t s)
{
    g_open_cls = cls;
    g_open_ev = take_event();
    cudaEventRecord(g_open_ev, s);
}

void prof_end(int cls, double flops, double bytes, cudaStream_t s)
{
    if (g_open_cls != cls || g_open_ev == nullptr) return;
    cudaEvent_t e1 = take_event();
    cudaEventRecord(e1, s);
    g_records.push_back({cls, g_open_ev, e1, flops, bytes});
    g_open_ev = nullptr;
    g_open_cls = -1;
}

}  // namespace rq

using namespace rq;

extern "C" {

__attribute__((visibility("default"))) int rqrcp_profile_begin(void)
{
    for (const Record& r : g_records) {
        g_pool.push_back(r.e0);
        g_pool.push_back(r.e1);
    }
    g_records.clear();
    g_on = true;
    return RQRCP_OK;
}

__attribute__((visibility("default"))) int rqrcp_profile_end(int nmax, int64_t* launches, double* ms, double* flops,
                                                             double* bytes)
{
    g_on = false;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    const int nc = nmax < RQRCP_PROFILE_CLASSES ? nmax : RQRCP_PROFILE_CLASSES;
    for (int c = 0; c < nc; ++c) {
        if (launches) launches[c] = 0;
        if (ms) ms[c] = 0.0;
        if (flops) flops[c] = 0.0;
        if (bytes) bytes[c] = 0.0;
    }
    for (const Record& r : g_records) {
        if (r.cls >= nc) continue;
        float t = 0.f;
        cudaEventElapsedTime(&t, r.e0, r.e1);
        if (launches) launches[r.cls] += 1;
        if (ms) ms[r.cls] += t;
        if (flops) flops[r.cls] += r.flops;
        if (bytes) bytes[r.cls] += r.bytes;
    }
    for (const Record& r : g_records) {
        g_pool.push_back(r.e0);
        g_pool.push_back(r.e1);
    }
    g_records.clear();
    return RQRCP_OK;
}

__attribute__((visibility("default"))) const char* rqrcp_profile_class_name(int cls)
{
    if (cls < 0 || cls >= RQRCP_PROFILE_CLASSES) return "unknown";
    return kNames[cls];
}

}  // extern "C"
