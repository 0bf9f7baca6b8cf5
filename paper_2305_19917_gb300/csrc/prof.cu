// Launch accounting and optional per-launch CUDA-event timing.
#include <atomic>
#include <mutex>
#include <vector>
#include "common.cuh"

namespace gb {
namespace {

std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_mu;

struct Rec {
    int kind;
    cudaEvent_t e0, e1;
    double flops, bytes;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

uint64_t &capture_count()
{
    static thread_local uint64_t n = 0;
    return n;
}

LaunchScope::LaunchScope(int k, cudaStream_t s, double flops, double bytes, uint64_t nkernels)
    : kind(k), slot(-1), stream(s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        capture_count() += nkernels;
        return;
    }
    g_launches.fetch_add(nkernels, std::memory_order_relaxed);
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r;
    r.kind = k;
    r.e0 = get_event();
    r.e1 = get_event();
    r.flops = flops;
    r.bytes = bytes;
    if (!r.e0 || !r.e1) return;
    cudaEventRecord(r.e0, s);
    g_recs.push_back(r);
    slot = (int)g_recs.size() - 1;
}

LaunchScope::~LaunchScope()
{
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < (int)g_recs.size()) cudaEventRecord(g_recs[slot].e1, stream);
}

}  // namespace gb

extern "C" {

uint64_t gb_kernel_launches(void) { return gb::g_launches.load(); }

int gb_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(gb::g_mu);
    for (auto &r : gb::g_recs) {
        gb::g_pool.push_back(r.e0);
        gb::g_pool.push_back(r.e1);
    }
    gb::g_recs.clear();
    gb::g_prof_on.store(on != 0);
    return 0;
}

int gb_profile_read(int kind, int64_t *launches, double *ms, double *flops, double *bytes)
{
    if (kind < 0 || kind >= gb::KK_COUNT) return -1;
    std::lock_guard<std::mutex> lk(gb::g_mu);
    int64_t n = 0;
    double t = 0, f = 0, b = 0;
    for (auto &r : gb::g_recs) {
        if (r.kind != kind) continue;
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e != cudaSuccess) return gb::check(e);
        float x = 0;
        e = cudaEventElapsedTime(&x, r.e0, r.e1);
        if (e != cudaSuccess) return gb::check(e);
        n++;
        t += x;
        f += r.flops;
        b += r.bytes;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    return 0;
}

}  // extern "C"
