// autotune.cu -- schedule choices measured on the GPU instead of taken from a rule.
//
// Two product schedules have more than one valid form:
//   * the emulated FP64 product (slice counts 7..9) can give each CTA whole output tiles or
//     split the K range of tiles between CTAs (stream-K);
//   * the tensor-core low-precision product can use 128 x 64 or 128 x 128 output tiles.
// The launchers choose by a rule measured on GB300 (gemm_f64e.cu, gemm_tc.cu).  With tuning
// switched on (mpps_autotune_enable(1), or MPPS_AUTOTUNE=1 in the environment), the first
// launch of a (kind, n, batch, variant) instead times every candidate on the call's own
// operands (one untimed run, then the mean of three timed runs, CUDA events on the call's
// stream), keeps the fastest in a per-process table, and runs it once more last, so that the
// output is always the chosen schedule's.  Later launches with the same key use the table.
// Launches whose epilogue reads its own output (an in-place accumulation) are not re-run and
// keep the rule.
#include "common.cuh"

#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace mpps {

namespace {

struct Entry {
    int choice;
    float ms[kTuneMaxCandidates];
    int ncand;
};

std::mutex g_tmu;
std::map<std::tuple<int, int, int, int, int>, Entry> g_table;   // (device, kind, n, batch, variant)
int g_enabled = -1;                                               // -1: read the environment

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return dev;
}

}  // namespace

bool tune_enabled() {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_enabled < 0) {
        const char* e = std::getenv("MPPS_AUTOTUNE");
        g_enabled = (e && e[0] == '1') ? 1 : 0;
    }
    return g_enabled == 1;
}

int tune_lookup(int kind, int n, int batch, int variant) {
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_table.find(std::make_tuple(current_device(), kind, n, batch, variant));
    return it == g_table.end() ? -1 : it->second.choice;
}

mpps_status tune_run(int kind, int n, int batch, int variant, int ncand, cudaStream_t st,
                     const std::function<mpps_status(int)>& launch) {
    if (ncand < 1 || ncand > kTuneMaxCandidates) {
        set_error("autotune: %d candidates (1..%d)", ncand, kTuneMaxCandidates);
        return MPPS_EINVAL;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MPPS_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("cudaEventCreate failed: %s", cudaGetErrorString(ce));
        return MPPS_ECUDA;
    }
    Entry en;
    en.ncand = ncand;
    mpps_status rc = MPPS_OK;
    constexpr int kTimed = 3;
    for (int c = 0; c < ncand && !rc; ++c) {
        rc = launch(c);   // untimed: first-use costs (attributes, tensor-map prefetch)
        if (!rc && (ce = cudaEventRecord(e0, st)) != cudaSuccess) rc = MPPS_ECUDA;
        for (int t = 0; t < kTimed && !rc; ++t) rc = launch(c);
        if (!rc && (ce = cudaEventRecord(e1, st)) != cudaSuccess) rc = MPPS_ECUDA;
        if (!rc && (ce = cudaEventSynchronize(e1)) != cudaSuccess) rc = MPPS_ECUDA;
        float ms = 0.f;
        if (!rc && (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) rc = MPPS_ECUDA;
        en.ms[c] = ms / kTimed;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        if (rc == MPPS_ECUDA) set_error("autotune timing failed: %s", cudaGetErrorString(ce));
        return rc;
    }
    int best = 0;
    for (int c = 1; c < ncand; ++c)
        if (en.ms[c] < en.ms[best]) best = c;
    en.choice = best;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        g_table[std::make_tuple(current_device(), kind, n, batch, variant)] = en;
    }
    // the output of the call is the chosen schedule's
    return best == ncand - 1 ? MPPS_OK : launch(best);
}

}  // namespace mpps

extern "C" {

void mpps_autotune_enable(int on) {
    std::lock_guard<std::mutex> lk(mpps::g_tmu);
    mpps::g_enabled = on ? 1 : 0;
}

void mpps_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(mpps::g_tmu);
    mpps::g_table.clear();
}

int mpps_autotune_entries(int* kind, int* n, int* batch, int* variant, int* choice, float* ms,
                          int cap) {
    std::lock_guard<std::mutex> lk(mpps::g_tmu);
    int i = 0;
    for (const auto& kv : mpps::g_table) {
        if (i < cap) {
            if (kind) kind[i] = std::get<1>(kv.first);
            if (n) n[i] = std::get<2>(kv.first);
            if (batch) batch[i] = std::get<3>(kv.first);
            if (variant) variant[i] = std::get<4>(kv.first);
            if (choice) choice[i] = kv.second.choice;
            if (ms)
                for (int c = 0; c < mpps::kTuneMaxCandidates; ++c)
                    ms[(size_t)i * mpps::kTuneMaxCandidates + c] =
                        c < kv.second.ncand ? kv.second.ms[c] : 0.f;
        }
        ++i;
    }
    return i;
}

}  // extern "C"
