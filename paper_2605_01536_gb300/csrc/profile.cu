// Optional per-kernel timing: CUDA events on the launching stream around each
// launch, aggregated by kernel name on request.
#include <algorithm>
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

// ---------------------------------------------------------------------------
// Pipe-throughput microbenchmarks behind the ALU rooflines: the issue rate of
// scalar FP32 FMAs, of paired FP32 FMAs (FFMA2, two lanes of work per
// instruction) and of the SFU reciprocal square root and reciprocal that the
// boundary kernels use.  Each
// thread runs kChains independent dependency chains so that latency is hidden;
// the result is folded into one store so that nothing is optimised away.
// ---------------------------------------------------------------------------
namespace gwn {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_ffma2(int iters, float seed, float *out) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + c + threadIdx.x, seed - c);
    const float2 m = make_float2(0.9999f, 0.9998f), k = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c].x + a[c].y;
    if (s == 1.2345f) out[blockIdx.x] = s;   // never true in practice; keeps the chains alive
}

__global__ void __launch_bounds__(256) k_peak_ffma(int iters, float seed, float *out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + c + threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], 0.9999f, 1e-7f);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 1.2345f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_mufu(int iters, float seed, float *out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 0.01f * (c + threadIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float r;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(a[c]) : "f"(r));   // a = sqrt(a): stays in range
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 1.2345f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace gwn

extern "C" gwn_status gwn_measure_pipe_peaks(double *ffma_per_s, double *ffma2_per_s, double *mufu_per_s,
                                             int32_t *sm_count, void *stream) {
    using namespace gwn;
    clear_error();
    if (!ffma_per_s || !ffma2_per_s || !mufu_per_s || !sm_count)
        return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    GWN_CUDA_TRY(cudaGetDevice(&dev));
    GWN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    *sm_count = sms;
    float *out = nullptr;
    const int blocks = sms * 8;   // 8 x 256 threads per SM: 64 warps
    GWN_CUDA_TRY(cudaMallocAsync(&out, sizeof(float) * blocks, s));
    cudaEvent_t a, b;
    GWN_CUDA_TRY(cudaEventCreate(&a));
    GWN_CUDA_TRY(cudaEventCreate(&b));
    const int iters_f = 32768, iters_m = 4096;
    float ms = 0.f;
    double best_f = 0.0, best_m = 0.0, best_1 = 0.0;
    for (int rep = 0; rep < 4; ++rep) {   // the first of each warms up
        cudaEventRecord(a, s);
        k_peak_ffma<<<blocks, 256, 0, s>>>(iters_f, 1.0f, out);
        cudaEventRecord(b, s);
        GWN_CUDA_TRY(cudaEventSynchronize(b));
        cudaEventElapsedTime(&ms, a, b);
        const double f1 = (double)blocks * 256 * iters_f * kChains / (ms * 1e-3);   // FFMA thread-instructions / s
        if (rep > 0) best_1 = std::max(best_1, f1);
        cudaEventRecord(a, s);
        k_peak_ffma2<<<blocks, 256, 0, s>>>(iters_f, 1.0f, out);
        cudaEventRecord(b, s);
        GWN_CUDA_TRY(cudaEventSynchronize(b));
        cudaEventElapsedTime(&ms, a, b);
        const double f = (double)blocks * 256 * iters_f * kChains / (ms * 1e-3);   // FFMA2 thread-instructions / s
        if (rep > 0) best_f = std::max(best_f, f);
        cudaEventRecord(a, s);
        k_peak_mufu<<<blocks, 256, 0, s>>>(iters_m, 1.5f, out);
        cudaEventRecord(b, s);
        GWN_CUDA_TRY(cudaEventSynchronize(b));
        cudaEventElapsedTime(&ms, a, b);
        const double m = (double)blocks * 256 * iters_m * kChains * 2 / (ms * 1e-3);   // SFU thread-operations / s
        if (rep > 0) best_m = std::max(best_m, m);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(out, s);
    GWN_LAUNCH_CHECK("pipe peaks");
    *ffma_per_s = best_1;
    *ffma2_per_s = best_f;
    *mufu_per_s = best_m;
    return GWN_OK;
}
