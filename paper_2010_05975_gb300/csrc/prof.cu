// Per-launch-class CUDA-event timing and a launch counter (the C ABI's
// lu_prof_* and lu_kernel_launch_count).  Event pairs are recorded on the
// stream each kernel is launched on, so a pair measures that launch as the
// stream executed it.  Process-wide state; one profiling session at a time.
#include "common.cuh"
#include "prof.cuh"
#include <atomic>
#include <mutex>
#include <vector>

namespace lu {

namespace {
struct Rec {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<unsigned long long> g_launches{0};

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

void count_launches(int n) { g_launches.fetch_add(static_cast<unsigned long long>(n)); }

ProfScope::ProfScope(int cls, cudaStream_t s, double flops, double bytes) : cls_(cls), s_(s), flops_(flops), bytes_(bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    a_ = take_event();
    b_ = take_event();
    if (a_ && b_) cudaEventRecord(a_, s_);
}

ProfScope::~ProfScope() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on || !a_ || !b_) return;
    cudaEventRecord(b_, s_);
    g_recs.push_back(Rec{cls_, a_, b_, flops_, bytes_});
}

}  // namespace lu

using namespace lu;

extern "C" int lu_prof_begin(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_on = true;
    return 0;
}

extern "C" int lu_prof_end(lu_prof_entry* out, int max_entries, int* n_entries) {
    if (max_entries < 0) return -2;
    if (n_entries == nullptr) return -3;
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = false;
    lu_prof_entry acc[LU_PROF_NCLASS] = {};
    for (int c = 0; c < LU_PROF_NCLASS; ++c) acc[c].kernel_class = c;
    int rc = 0;
    for (auto& r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            rc = LU_ELAUNCH;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            rc = LU_ELAUNCH;
            break;
        }
        lu_prof_entry& e = acc[r.cls];
        e.launches += 1;
        e.total_ms += ms;
        e.total_flops += r.flops;
        e.total_bytes += r.bytes;
    }
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    cudaGetLastError();
    int n = 0;
    for (int c = 0; c < LU_PROF_NCLASS && n < max_entries; ++c)
        if (acc[c].launches > 0 && out) out[n++] = acc[c];
    *n_entries = n;
    return rc;
}

extern "C" unsigned long long lu_kernel_launch_count(void) { return g_launches.load(); }

// ---------------------------------------------------------------------------
// Wait deadlines and the test hook that makes a wait run out
// ---------------------------------------------------------------------------
namespace lu {
namespace {
std::atomic<unsigned long long> g_wait_ns[LU_WAIT_NSITES] = {};
std::atomic<int> g_inject[LU_WAIT_NSITES] = {};
}  // namespace

WaitCfg wait_cfg(int site) {
    WaitCfg c{kWaitDefaultNs, 0};
    if (site < 0 || site >= LU_WAIT_NSITES) return c;
    const unsigned long long ns = g_wait_ns[site].load();
    if (ns > 0) c.wait_ns = ns;
    c.inject = g_inject[site].load();
    return c;
}
}  // namespace lu

extern "C" int lu_test_wait_config(int site, long long wait_ns, int inject) {
    if (site < 0 || site >= LU_WAIT_NSITES) return -1;
    if (wait_ns < 0 || wait_ns > 600000000000ll) return -2;
    if (inject != 0 && inject != 1) return -3;
    g_wait_ns[site].store(static_cast<unsigned long long>(wait_ns));
    g_inject[site].store(inject);
    return 0;
}

extern "C" long long lu_wait_deadline_ns(int site) {
    if (site < 0 || site >= LU_WAIT_NSITES) return -1;
    return static_cast<long long>(wait_cfg(site).wait_ns);
}
