// profile.cu -- optional per-stage device timing.  When enabled, the library
// records a CUDA event pair around each stage on the caller's stream and adds
// the elapsed time to a process-wide table when the stage's call completes.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace ct {

std::atomic<int64_t> g_total_launches{0};

namespace {
struct Pending {
    std::string name;
    cudaEvent_t a, b;
    bool closed = false;  // its end event is recorded
    bool done = false;    // added to the table, events released
};
struct Acc {
    double ms = 0;
    int64_t calls = 0;
};
std::mutex g_mu;
std::atomic<int> g_on{0};
thread_local std::vector<Pending> t_pending;
std::map<std::string, Acc> g_acc;
std::vector<std::string> g_names;  // stable storage for returned names
}  // namespace

bool prof_on() { return g_on.load(std::memory_order_relaxed) != 0; }

ProfScope::ProfScope(const char *name, cudaStream_t s) : s_(s), active_(prof_on()) {
    if (!active_) return;
    Pending p;
    p.name = name;
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecord(p.a, s);
    t_pending.push_back(p);
    idx_ = (int)t_pending.size() - 1;
}

ProfScope::~ProfScope() {
    if (!active_) return;
    cudaEventRecord(t_pending[idx_].b, s_);
    t_pending[idx_].closed = true;
}

// Scopes may nest (a stage that calls another entry point): only closed
// scopes are added; entries stay in place (their indices are held by open
// scopes) until every scope of the thread is closed.
void prof_flush() {
    if (t_pending.empty()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    bool all_done = true;
    for (auto &p : t_pending) {
        if (p.done) continue;
        if (!p.closed) {
            all_done = false;
            continue;
        }
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Acc &a = g_acc[p.name];
            a.ms += ms;
            a.calls += 1;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
        p.done = true;
    }
    if (all_done) t_pending.clear();
}

}  // namespace ct

extern "C" {

void ct_profile_enable(int32_t on) { ct::g_on.store(on ? 1 : 0); }

void ct_profile_reset(void) {
    std::lock_guard<std::mutex> lk(ct::g_mu);
    ct::g_acc.clear();
}

int32_t ct_profile_count(void) {
    std::lock_guard<std::mutex> lk(ct::g_mu);
    ct::g_names.clear();
    for (auto &kv : ct::g_acc) ct::g_names.push_back(kv.first);
    return (int32_t)ct::g_names.size();
}

ct_status ct_profile_entry(int32_t i, const char **name, double *total_ms, int64_t *calls) {
    std::lock_guard<std::mutex> lk(ct::g_mu);
    if (i < 0 || i >= (int32_t)ct::g_names.size() || !name || !total_ms || !calls) return CT_EINVAL;
    auto it = ct::g_acc.find(ct::g_names[i]);
    if (it == ct::g_acc.end()) return CT_EINVAL;
    *name = ct::g_names[i].c_str();
    *total_ms = it->second.ms;
    *calls = it->second.calls;
    return CT_OK;
}

int64_t ct_kernel_launches(void) { return ct::g_total_launches.load(); }

}  // extern "C"
