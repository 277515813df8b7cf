// Launch counting and optional per-kernel-family device timing with CUDA events recorded
// on the launch stream around each launch (used by the benchmark to report the live
// duration of the dominant kernel).
#include <atomic>
#include <mutex>
#include <vector>

#include "qm_internal.h"

namespace qm {

static std::atomic<unsigned long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::mutex g_prof_mu;

struct ProfRec {
    int family;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_recs;          // pending (not yet read) records
static std::vector<cudaEvent_t> g_pool;      // recycled events
static double g_ms[kProfFamilies];
static long long g_cnt[kProfFamilies];

static const char* kNames[kProfFamilies] = {"k_vt", "k_stick_inverse", "k_plane", "k_stick_forward",
                                            "k_gemm_cn", "k_reduce_splits", "k_gemm_tn", "other", "k_chol",
                                            "k_tridiag", "k_multisect", "k_inviter", "k_backtransf", "k_convert",
                                            "k_umma_bf16x3", "k_split", "k_batch", "k_mlp"};

static cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

ProfScope::ProfScope(int family, cudaStream_t s) : family_(family), s_(s) {
    count_launch(1);
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    a_ = get_event();
    b_ = get_event();
    cudaEventRecord(a_, s_);
    active_ = true;
}

ProfScope::~ProfScope() {
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(b_, s_);
    g_recs.push_back({family_, a_, b_});
}

static void drain_locked() {
    for (auto& r : g_recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_ms[r.family] += ms;
            g_cnt[r.family] += 1;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}

}  // namespace qm

using namespace qm;

extern "C" unsigned long long qm_launch_count(void) { return g_launches.load(); }

extern "C" qm_status qm_prof_enable(int on) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    for (int i = 0; i < kProfFamilies; ++i) {
        g_ms[i] = 0.0;
        g_cnt[i] = 0;
    }
    g_prof_on.store(on ? 1 : 0);
    return QM_OK;
}

extern "C" qm_status qm_prof_read(int family, double* ms_total, long long* launches) {
    clear_error();
    if (family < 0 || family >= kProfFamilies) return fail(QM_ERR_ARG, "qm_prof_read: family out of range");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    if (ms_total) *ms_total = g_ms[family];
    if (launches) *launches = g_cnt[family];
    return QM_OK;
}

extern "C" const char* qm_prof_name(int family) {
    if (family < 0 || family >= kProfFamilies) return "";
    return kNames[family];
}
