// Process-wide launch counters and optional per-launch CUDA-event timing
// (cd_stats_reset / cd_stats_get).  Every kernel launch of the library goes
// through a LaunchScope, so the counters are the library's own claim of how
// many kernels it ran.
#include <atomic>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace cd {
namespace {

struct Pending {
    int kind;
    cudaEvent_t a, b;
};

std::mutex g_mu;
int64_t g_count[CD_K_COUNT] = {};
double g_ms[CD_K_COUNT] = {};
double g_flops[CD_K_COUNT] = {};
bool g_timing = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

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

void drain()
{
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            g_ms[p.kind] += ms;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

const char *const kKindRange[CD_K_COUNT] = {"colden:restrict", "colden:shell",    "colden:leaf",
                                            "colden:other",    "colden:net",      "colden:features",
                                            "colden:raymarch", "colden:learned",  "colden:heating"};

NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

static std::atomic<int64_t> g_free_gen{0};

cudaError_t lib_free(void *p)
{
    g_free_gen.fetch_add(1);
    return cudaFree(p);
}

int64_t free_generation() { return g_free_gen.load(); }

void stats_snapshot(int64_t *count, double *flops)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < CD_K_COUNT; ++k) {
        count[k] = g_count[k];
        flops[k] = g_flops[k];
    }
}

void stats_add(const int64_t *count, const double *flops, int sign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < CD_K_COUNT; ++k) {
        g_count[k] += sign * count[k];
        g_flops[k] += sign * flops[k];
    }
}

bool stats_timing()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_timing;
}

LaunchScope::LaunchScope(int kind, cudaStream_t s, double flops) : kind_(kind), s_(s)
{
    nvtxRangePushA(kKindRange[kind]);
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_count[kind];
    g_flops[kind] += flops;
    // no timing events inside a stream capture (the graph would hold them and
    // the runtime refuses timing events there)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (g_timing && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
        a_ = take_event();
        b_ = take_event();
        cudaEventRecord(a_, s_);
    }
}

LaunchScope::~LaunchScope()
{
    if (a_) {
        cudaEventRecord(b_, s_);
        std::lock_guard<std::mutex> lk(g_mu);
        g_pending.push_back({kind_, a_, b_});
    }
    nvtxRangePop();
}

}  // namespace cd

extern "C" {

void cd_stats_reset(int timing)
{
    std::lock_guard<std::mutex> lk(cd::g_mu);
    cd::drain();
    for (int k = 0; k < CD_K_COUNT; ++k) {
        cd::g_count[k] = 0;
        cd::g_ms[k] = 0.0;
        cd::g_flops[k] = 0.0;
    }
    cd::g_timing = timing != 0;
}

cd_status cd_stats_get(int kind, int64_t *launches, double *ms)
{
    if (kind < 0 || kind >= CD_K_COUNT) {
        cd::set_error("unknown kernel kind %d", kind);
        return CD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(cd::g_mu);
    cd::drain();
    if (launches) *launches = cd::g_count[kind];
    if (ms) *ms = cd::g_ms[kind];
    return CD_OK;
}

cd_status cd_stats_flops(int kind, double *flops)
{
    if (kind < 0 || kind >= CD_K_COUNT) {
        cd::set_error("unknown kernel kind %d", kind);
        return CD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(cd::g_mu);
    if (flops) *flops = cd::g_flops[kind];
    return CD_OK;
}

}  // extern "C"
