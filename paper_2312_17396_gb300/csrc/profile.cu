// profile.cu -- optional per-launch timing of the library's kernels with CUDA events on
// the launch stream (used by the benchmark to measure kernel durations inside the timed
// region without a profiler).  Off by default; when off a scope costs one branch.
#include "common.cuh"

#include <mutex>
#include <vector>

namespace mpps {

namespace {
struct Rec {
    int cls;
    double work;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

ProfScope::ProfScope(int c, cudaStream_t s, double w)
    : cls(c), st(s), a(nullptr), b(nullptr), on(false), work(w) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    a = take_event();
    b = take_event();
    if (!a || !b) return;
    on = cudaEventRecord(a, st) == cudaSuccess;
}

ProfScope::~ProfScope() {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaEventRecord(b, st) == cudaSuccess) g_recs.push_back({cls, work, a, b});
}

}  // namespace mpps

using namespace mpps;

extern "C" {

void mpps_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
}

void mpps_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}

mpps_status mpps_profile_read(int kernel_class, long long* launches, double* total_ms,
                              double* total_work) {
    clear_error();
    if (!launches || !total_ms || kernel_class < 0 || kernel_class >= MPPS_PROF_NUM_CLASSES) {
        set_error("mpps_profile_read: invalid argument");
        return MPPS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    long long cnt = 0;
    double tot = 0.0, work = 0.0;
    for (auto& r : g_recs) {
        if (r.cls != kernel_class) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            set_error("mpps_profile_read: %s", cudaGetErrorString(cudaGetLastError()));
            return MPPS_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        tot += ms;
        work += r.work;
        ++cnt;
    }
    *launches = cnt;
    *total_ms = tot;
    if (total_work) *total_work = work;
    return MPPS_OK;
}

}  // extern "C"
