// Run-time autotuner (see autotune.h).
#include <map>
#include <vector>

#include "autotune.h"
#include "common.cuh"

namespace sim {

namespace {

constexpr int kSamples = 3;  // timed launches per candidate

struct Pending {
    int cand;
    cudaEvent_t e0, e1;
};

struct Site {
    int ncand = 0;
    int best = -1;
    int next = 0;
    std::vector<double> ms;
    std::vector<int> count;
    std::vector<Pending> pending;
    Pending open{-1, nullptr, nullptr};
};

std::map<std::string, Site>& sites() {
    static std::map<std::string, Site> s;
    return s;
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
    cudaEvent_t e = nullptr;
    SIM_CUDA(cudaEventCreate(&e));
    return e;
}

void collect(Site& s) {
    std::vector<Pending> keep;
    for (const Pending& q : s.pending) {
        if (cudaEventQuery(q.e1) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, q.e0, q.e1) == cudaSuccess) {
                s.ms[q.cand] += ms;
                s.count[q.cand] += 1;
            }
            pool().push_back(q.e0);
            pool().push_back(q.e1);
        } else {
            keep.push_back(q);
        }
    }
    s.pending.swap(keep);
    (void)cudaGetLastError();  // a not-ready query is not an error
    for (int c = 0; c < s.ncand; ++c)
        if (s.count[c] < kSamples) return;
    int b = 0;
    for (int c = 1; c < s.ncand; ++c)
        if (s.ms[c] / s.count[c] < s.ms[b] / s.count[b]) b = c;
    s.best = b;
}

}  // namespace

int autotune_begin(const std::string& key, int ncand, cudaStream_t st, bool* timing) {
    *timing = false;
    Site& s = sites()[key];
    if (s.ncand == 0) {
        s.ncand = ncand;
        s.ms.assign(ncand, 0.0);
        s.count.assign(ncand, 0);
    }
    if (s.best >= 0) return s.best;
    collect(s);
    if (s.best >= 0) return s.best;
    // the candidate with the fewest samples (issued or measured) goes next
    std::vector<int> issued(s.count);
    for (const Pending& q : s.pending) issued[q.cand] += 1;
    int c = 0;
    for (int i = 1; i < s.ncand; ++i)
        if (issued[i] < issued[c]) c = i;
    if (issued[c] >= kSamples) return c;  // all issued, results not in yet
    s.open = Pending{c, take(), take()};
    SIM_CUDA(cudaEventRecord(s.open.e0, st));
    *timing = true;
    return c;
}

void autotune_end(const std::string& key, cudaStream_t st) {
    Site& s = sites()[key];
    if (s.open.cand < 0) return;
    SIM_CUDA(cudaEventRecord(s.open.e1, st));
    s.pending.push_back(s.open);
    s.open = Pending{-1, nullptr, nullptr};
}

int autotune_choice(const std::string& key) {
    auto it = sites().find(key);
    return it == sites().end() ? -1 : it->second.best;
}

}  // namespace sim
