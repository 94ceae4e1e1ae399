// Optional per-kernel device timing: when enabled, the library records a pair
// of CUDA events on the launch stream around each of its main kernel launches
// and sums the elapsed times per kernel name on request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "gwe_internal.h"

namespace gwe {
namespace {

struct Entry {
    std::string name;
    std::vector<cudaEvent_t> begin, end;
    double ms = 0.0;
    int64_t launches = 0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Entry> g_entries;

int slot_of(const char *name) {
    for (size_t i = 0; i < g_entries.size(); ++i)
        if (g_entries[i].name == name) return (int)i;
    g_entries.push_back(Entry());
    g_entries.back().name = name;
    return (int)g_entries.size() - 1;
}

void drain(Entry &e) {
    for (size_t i = 0; i < e.begin.size(); ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(e.end[i]) == cudaSuccess && cudaEventElapsedTime(&ms, e.begin[i], e.end[i]) == cudaSuccess)
            e.ms += ms;
        cudaEventDestroy(e.begin[i]);
        cudaEventDestroy(e.end[i]);
    }
    e.begin.clear();
    e.end.clear();
}

std::atomic<long long> g_launches{0};
thread_local int tl_suspend = 0;    // > 0 while a stream capture is being recorded on this thread

}  // namespace

ProfSuspend::ProfSuspend() { ++tl_suspend; }
ProfSuspend::~ProfSuspend() { --tl_suspend; }

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(const char *name, cudaStream_t s) : slot(-1), st(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on || tl_suspend > 0) return;
    cudaEvent_t b, e;
    if (cudaEventCreate(&b) != cudaSuccess) return;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaEventDestroy(b);
        return;
    }
    slot = slot_of(name);
    g_entries[slot].begin.push_back(b);
    g_entries[slot].end.push_back(e);
    g_entries[slot].launches++;
    cudaEventRecord(b, st);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_entries[slot].end.back(), st);
}

}  // namespace gwe

using namespace gwe;

extern "C" {

gwe_status gwe_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &e : g_entries) drain(e);
    g_entries.clear();
    g_on = on != 0;
    return GWE_OK;
}

gwe_status gwe_profile_read(int idx, char *name, int name_cap, double *total_ms, int64_t *launches) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx < 0 || idx >= (int)g_entries.size() || !total_ms || !launches) return GWE_ERR_ARG;
    Entry &e = g_entries[idx];
    drain(e);
    if (name && name_cap > 0) {
        size_t n = std::min((size_t)(name_cap - 1), e.name.size());
        e.name.copy(name, n);
        name[n] = 0;
    }
    *total_ms = e.ms;
    *launches = e.launches;
    return GWE_OK;
}

int64_t gwe_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
