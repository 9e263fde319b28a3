// Optional region timers: CUDA event pairs recorded on the launching stream around named regions
// (one exp-apply, one tridiagonal reduction, ...). Off by default; resolved lazily on read.
#include "eda_internal.cuh"

#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace eda {

namespace {
struct Region {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double total_ms = 0.0;
    int64_t calls = 0;
    double flops = 0.0, bytes = 0.0;   // algorithmic work of the calls, as counted at entry
};
std::mutex g_mu;
bool g_on = false;
std::map<std::string, Region> g_regions;
std::vector<cudaEvent_t> g_pool;

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

int resolve(Region& r) {
    for (auto& pr : r.pending) {
        if (cudaEventSynchronize(pr.second) != cudaSuccess) return EDA_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess) return EDA_ERR_CUDA;
        r.total_ms += ms;
        r.calls += 1;
        g_pool.push_back(pr.first);
        g_pool.push_back(pr.second);
    }
    r.pending.clear();
    return EDA_OK;
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t s, double flops, double bytes) : name_(name), s_(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    Region& r = g_regions[name_];
    r.flops += flops;
    r.bytes += bytes;
    e0_ = get_event();
    if (e0_) cudaEventRecord(e0_, s_);
}

ProfScope::~ProfScope() {
    if (!e0_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e1 = get_event();
    if (!e1) return;
    cudaEventRecord(e1, s_);
    g_regions[name_].pending.emplace_back(e0_, e1);
}

}  // namespace eda

using namespace eda;

extern "C" {

int eda_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return EDA_OK;
}

int eda_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_regions) {
        resolve(kv.second);
        kv.second.total_ms = 0.0;
        kv.second.calls = 0;
        kv.second.flops = 0.0;
        kv.second.bytes = 0.0;
    }
    return EDA_OK;
}

int eda_profile_read(const char* region, double* total_ms, int64_t* calls) {
    if (!region) return EDA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_regions.find(region);
    if (it == g_regions.end()) {
        if (total_ms) *total_ms = 0.0;
        if (calls) *calls = 0;
        return EDA_OK;
    }
    int rc = resolve(it->second);
    if (total_ms) *total_ms = it->second.total_ms;
    if (calls) *calls = it->second.calls;
    return rc;
}

int eda_profile_work(const char* region, double* flops, double* bytes) {
    if (!region) return EDA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_regions.find(region);
    if (flops) *flops = it == g_regions.end() ? 0.0 : it->second.flops;
    if (bytes) *bytes = it == g_regions.end() ? 0.0 : it->second.bytes;
    return EDA_OK;
}

}  // extern "C"
