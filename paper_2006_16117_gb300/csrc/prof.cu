// Launch counter and optional per-kernel event timing (host side only).
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace sim {

int64_t& launch_counter() {
    static int64_t n = 0;
    return n;
}

namespace {
struct KRec {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    double bytes = 0.0, flops = 0.0, ms = 0.0;
    int64_t launches = 0;
    cudaEvent_t pending = nullptr;
};
bool g_on = false;
std::map<std::string, KRec>& recs() {
    static std::map<std::string, KRec> r;
    return r;
}
std::vector<cudaEvent_t>& pool() {
    static std::vector<cudaEvent_t> p;
    return p;
}
cudaEvent_t take() {
    auto& p = pool();
    if (!p.empty()) {
        cudaEvent_t e = p.back();
        p.pop_back();
        return e;
    }
    cudaEvent_t e;
    SIM_CUDA(cudaEventCreate(&e));
    return e;
}
void settle(KRec& r) {
    for (auto& pr : r.ev) {
        float ms = 0.f;
        if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
            r.ms += ms;
        pool().push_back(pr.first);
        pool().push_back(pr.second);
    }
    r.ev.clear();
}
}  // namespace

bool kprof_enabled() { return g_on; }
void kprof_enable(bool on) { g_on = on; }

void kprof_begin(const char* name, cudaStream_t st) {
    if (!g_on) return;
    KRec& r = recs()[name];
    r.pending = take();
    SIM_CUDA(cudaEventRecord(r.pending, st));
}

void kprof_end(const char* name, cudaStream_t st, double bytes, double flops) {
    if (!g_on) return;
    KRec& r = recs()[name];
    if (!r.pending) return;
    cudaEvent_t e = take();
    SIM_CUDA(cudaEventRecord(e, st));
    r.ev.push_back({r.pending, e});
    r.pending = nullptr;
    r.bytes += bytes;
    r.flops += flops;
    r.launches += 1;
    if (r.ev.size() > 4096) settle(r);
}

void kprof_reset() {
    for (auto& kv : recs()) settle(kv.second);
    recs().clear();
}

bool kprof_query(const char* name, double* ms, double* bytes, double* flops, int64_t* launches) {
    auto it = recs().find(name);
    if (it == recs().end()) return false;
    settle(it->second);
    if (ms) *ms = it->second.ms;
    if (bytes) *bytes = it->second.bytes;
    if (flops) *flops = it->second.flops;
    if (launches) *launches = it->second.launches;
    return true;
}

}  // namespace sim
