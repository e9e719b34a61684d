// Measurement support (no counterpart in the paper): a count of the library's
// kernel launches and, when enabled, CUDA-event timing of the SpMV chunk
// kernels, each launch tagged with its family name and algorithmic bytes.
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "b2sr_internal.cuh"

namespace b2sr {

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_timing{false};

struct TimedLaunch {
    std::string family;
    cudaEvent_t start;
    cudaEvent_t stop;
    double bytes;
};
static std::mutex g_mu;
static std::vector<TimedLaunch> g_records;

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool timing_on() { return g_timing.load(std::memory_order_relaxed); }

void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void* timing_begin(cudaStream_t s) {
    if (!timing_on()) return nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;  // launches inside a captured graph are not timed one by one
    }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    cudaEventRecord(e, s);
    return e;
}

void timing_end(void* tok, const char* family, double bytes, cudaStream_t s) {
    if (!tok) return;
    cudaEvent_t stop;
    if (cudaEventCreate(&stop) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(static_cast<cudaEvent_t>(tok));
        return;
    }
    cudaEventRecord(stop, s);
    std::lock_guard<std::mutex> lk(g_mu);
    g_records.push_back(TimedLaunch{family, static_cast<cudaEvent_t>(tok), stop, bytes});
}

}  // namespace b2sr

using namespace b2sr;

extern "C" int64_t b2sr_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" void b2sr_timing_enable(int on) { g_timing.store(on != 0); }

extern "C" b2sr_status b2sr_timing_read(const char* family, double* total_ms, int64_t* launches, double* bytes) {
    clear_error();
    if (!family || !total_ms || !launches || !bytes) return fail(B2SR_ERR_INVALID_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(g_mu);
    double ms = 0.0, by = 0.0;
    int64_t n = 0;
    for (auto& r : g_records) {
        if (r.family != family) continue;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e != cudaSuccess) return cuda_fail(e, "b2sr_timing_read");
        float t = 0.0f;
        cudaEventElapsedTime(&t, r.start, r.stop);
        ms += t;
        by += r.bytes;
        ++n;
    }
    *total_ms = ms;
    *launches = n;
    *bytes = by;
    return B2SR_OK;
}

extern "C" b2sr_status b2sr_timing_reset(void) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_records) {
        cudaEventSynchronize(r.stop);
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    g_records.clear();
    return B2SR_OK;
}
