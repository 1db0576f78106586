// Kernel tracing: a launch counter that is always on, and, while enabled, a
// pair of CUDA events recorded on the launch stream around every kernel launch
// of the library, grouped by kernel name.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dn_internal.cuh"

namespace dn {

namespace {

struct Tag {
    std::string name;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    long long launches = 0;
    double ms = 0.0;
};

std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::vector<Tag> g_tags;
std::vector<cudaEvent_t> g_pool;
thread_local std::vector<const char *> t_phase;

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

int tag_index(const char *name) {
    for (size_t i = 0; i < g_tags.size(); ++i)
        if (g_tags[i].name == name) return (int)i;
    g_tags.push_back(Tag{name, {}, 0, 0.0});
    return (int)g_tags.size() - 1;
}

// Fold recorded event pairs into the totals (the events must have completed).
void drain() {
    for (Tag &t : g_tags) {
        for (auto &pr : t.ev) {
            float ms = 0.0f;
            if (pr.first && pr.second && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) t.ms += ms;
            else cudaGetLastError();
            if (pr.first) g_pool.push_back(pr.first);
            if (pr.second) g_pool.push_back(pr.second);
        }
        t.ev.clear();
    }
}

}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t st) : st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    std::string full;
    for (const char *s : t_phase) {
        full += s;
        full += '/';
    }
    full += name;
    tag_ = tag_index(full.c_str());
    start_ = take_event();
    if (start_) cudaEventRecord(start_, st_);
}

ProfPhase::ProfPhase(const char *name) { t_phase.push_back(name); }
ProfPhase::~ProfPhase() { t_phase.pop_back(); }

ProfScope::~ProfScope() {
    if (tag_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t stop = take_event();
    if (stop) cudaEventRecord(stop, st_);
    if (tag_ < (int)g_tags.size()) {
        g_tags[tag_].ev.emplace_back(start_, stop);
        g_tags[tag_].launches += 1;
    }
}

}  // namespace dn

extern "C" {

long long dn_launch_count(void) { return dn::g_launches.load(); }

dn_status dn_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(dn::g_mu);
    if (on && !dn::g_on) {
        for (auto &t : dn::g_tags) {
            t.launches = 0;
            t.ms = 0.0;
        }
    }
    dn::g_on = on != 0;
    return DN_OK;
}

int dn_profile_count(void) {
    std::lock_guard<std::mutex> lk(dn::g_mu);
    return (int)dn::g_tags.size();
}

dn_status dn_profile_get(int i, char *name, size_t name_len, long long *launches, double *total_ms) {
    if (cudaDeviceSynchronize() != cudaSuccess) return DN_ECUDA;
    std::lock_guard<std::mutex> lk(dn::g_mu);
    dn::drain();
    if (i < 0 || i >= (int)dn::g_tags.size()) return DN_EINVAL;
    const dn::Tag &t = dn::g_tags[i];
    if (name && name_len) {
        std::strncpy(name, t.name.c_str(), name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = t.launches;
    if (total_ms) *total_ms = t.ms;
    return DN_OK;
}

}  // extern "C"
