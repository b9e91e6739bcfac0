// Optional per-kernel timing: CUDA events on the launching stream around each
// launch, aggregated by kernel name on request.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gwn_internal.cuh"

namespace gwn {

namespace {
struct Rec {
    const char *name;
    cudaEvent_t a, b;
    int64_t kernels;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
thread_local ProfScope *t_scope = nullptr;   // innermost active scope of this thread
}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t s) : name_(name), s_(s) {
    if (!g_on) return;
    cudaEventCreate(&a_);
    cudaEventCreate(&b_);
    cudaEventRecord(a_, s_);
    active_ = true;
    parent_ = t_scope;
    t_scope = this;
}

ProfScope::~ProfScope() {
    if (!active_) return;
    t_scope = parent_;
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back(Rec{name_, a_, b_, kernels_ > 0 ? kernels_ : 1});
}

void note_launches(int k) {
    if (t_scope) t_scope->kernels_ += k;
}

}  // namespace gwn

using namespace gwn;

extern "C" {

gwn_status gwn_profile_enable(int on) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
    g_on = on != 0;
    return GWN_OK;
}

gwn_status gwn_profile_read(gwn_kernel_stat *stats, int cap, int *n_out) {
    clear_error();
    if (!n_out || (cap > 0 && !stats)) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    std::vector<Rec> recs;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        recs.swap(g_recs);
    }
    std::map<std::string, std::pair<int64_t, double>> agg;
    std::map<std::string, int64_t> kern;
    gwn_status st = GWN_OK;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess && st == GWN_OK) st = set_error(GWN_ERR_CUDA, cudaGetErrorString(e));
        auto &v = agg[r.name];
        v.first += 1;
        v.second += ms;
        kern[r.name] += r.kernels;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    int i = 0;
    for (auto &kv : agg) {
        if (i < cap) {
            std::memset(&stats[i], 0, sizeof(stats[i]));
            std::strncpy(stats[i].name, kv.first.c_str(), sizeof(stats[i].name) - 1);
            stats[i].launches = kv.second.first;
            stats[i].total_ms = kv.second.second;
            stats[i].kernels = kern[kv.first];
        }
        ++i;
    }
    *n_out = i;
    return st;
}

}  // extern "C"
