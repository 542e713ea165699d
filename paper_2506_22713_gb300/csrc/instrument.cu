// Measurement hooks: a count of every kernel the library launches and,
// when enabled, CUDA-event timing of each launch grouped by kernel kind,
// with the algorithmic flops and bytes of the launch.  Events are recorded on
// the stream the kernel is launched on.
#include "common.cuh"
#include "instrument.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace eod {
namespace {

std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};

struct Rec {
    int kind;
    double flops, bytes;
    cudaEvent_t a, b;
};

std::mutex g_mu;
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

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    constexpr int kMaxDev = 64;
    static cudaMemPool_t pools[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np;
            e = cudaMemPoolCreate(&np, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = 64ull << 30;
            e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
            pools[dev] = np;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

ProfScope::ProfScope(int kind, double flops, double bytes, cudaStream_t s) : s_(s), rec_(-1) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t a = take_event(), b = take_event();
    if (!a || !b) return;
    if (cudaEventRecord(a, s) != cudaSuccess) { cudaGetLastError(); return; }
    g_recs.push_back(Rec{kind, flops, bytes, a, b});
    rec_ = (int)g_recs.size() - 1;
}

ProfScope::~ProfScope() {
    if (rec_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (rec_ < (int)g_recs.size()) {
        if (cudaEventRecord(g_recs[rec_].b, s_) != cudaSuccess) cudaGetLastError();
    }
}

void profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_enabled.store(on ? 1 : 0);
}

long long launch_count() { return g_launches.load(); }

int profile_read(int kind, long long *launches, double *ms, double *flops, double *bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    long long n = 0;
    double t = 0, f = 0, by = 0;
    for (auto &r : g_recs) {
        if (r.kind != kind) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) { cudaGetLastError(); return 1; }
        float e = 0.f;
        if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) { cudaGetLastError(); return 1; }
        ++n;
        t += e;
        f += r.flops;
        by += r.bytes;
    }
    *launches = n;
    *ms = t;
    *flops = f;
    *bytes = by;
    return 0;
}

}  // namespace eod

extern "C" {

void eod_abe_debug_profile(int32_t enable) { eod::profile_enable(enable); }

int64_t eod_abe_debug_launch_count(void) { return (int64_t)eod::launch_count(); }

eod_status eod_abe_debug_profile_read(int32_t kind, int64_t *launches, double *total_ms, double *total_flops,
                                      double *total_bytes) {
    if (!launches || !total_ms || !total_flops || !total_bytes || kind < 0 || kind >= eod::PROF_KINDS)
        return EOD_EINVAL;
    long long n = 0;
    if (eod::profile_read(kind, &n, total_ms, total_flops, total_bytes)) return EOD_ECUDA;
    *launches = (int64_t)n;
    return EOD_OK;
}

}  // extern "C"
