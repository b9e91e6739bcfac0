// gwn_classify_static: gwn_classify without any device allocation.
//
// Some callers cannot allocate device memory on the call path: hosts that
// reserve their whole device-memory budget up front (a fixed pool, another
// framework's caching allocator owning the GPU), and latency-critical loops
// that must not enter the CUDA allocator, whose calls can take locks,
// synchronise or grow a memory pool.  gwn_classify obtains its scratch (the
// crossing numbers, the FP64 re-evaluation list and the boundary-sum partials)
// from the stream-ordered allocator on every call; this entry point instead
// uses one file-scope device array that every GPU loading the library holds
// until the process exits.
#include <mutex>

#include "gwn_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int64_t kMaxQueries = int64_t(1) << 21;     // 2,097,152 queries per call
constexpr size_t kHeader = 256;                       // the re-evaluation counter, padded

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device;
// a host-side reference to g_scratch names a host stand-in, not device memory).
gwn_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return gwn::set_error(GWN_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return gwn::set_error(GWN_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                                    cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return GWN_OK;
}


}  // namespace

extern "C" gwn_status gwn_classify_static(const gwn_mesh *m, const float *q, int64_t n, uint8_t *label,
                                          float *w_or_null, void *stream) {
    gwn::clear_error();
    if (!m) return gwn::set_error(GWN_ERR_INVALID_ARG, "mesh is NULL");
    if (n < 0) return gwn::set_error(GWN_ERR_INVALID_ARG, "negative query count");
    if (n > kMaxQueries)
        return gwn::set_error(GWN_ERR_INVALID_ARG,
                              "gwn_classify_static: n = " + std::to_string(n) +
                                  " exceeds the static scratch limit of 2097152 queries per call");
    if (!m->built) return gwn::set_error(GWN_ERR_NOT_BUILT, "call gwn_build_accel first");
    if (n == 0) return GWN_OK;
    if (!q || !label) return gwn::set_error(GWN_ERR_INVALID_ARG, "q or label is NULL");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != m->device) cudaSetDevice(m->device);
    gwn_status st = GWN_OK;
    const int kq = gwn::pointer_kind(q, m->device), kl = gwn::pointer_kind(label, m->device),
              kw = gwn::pointer_kind(w_or_null, m->device);
    if (kq < 0 || kl < 0 || kw < 0) {
        st = gwn::set_error(GWN_ERR_INVALID_ARG, "gwn_classify_static: a buffer is device memory of another GPU "
                                                 "than the mesh's");
    } else if (kq == 0 || kl == 0 || kw == 0) {
        st = gwn::set_error(GWN_ERR_INVALID_ARG,
                            "gwn_classify_static takes device pointers only (host buffers would need staging)");
    } else {
        unsigned char *base = nullptr;
        st = scratch_address(m->device, &base);
        if (st == GWN_OK) {
            cudaStream_t s = (cudaStream_t)stream;
            // layout: [counter | chi n x int32 | list n x int32 | w n x float | listed (n + 31) / 32 x uint32 |
            //          FP64 partials ...]
            auto *len = reinterpret_cast<unsigned long long *>(base);
            auto *chi = reinterpret_cast<int32_t *>(base + kHeader);
            auto *list = chi + n;
            float *w_tmp = reinterpret_cast<float *>(list + n);
            auto *listed = reinterpret_cast<unsigned *>(w_tmp + n);
            const size_t words = (size_t)((n + 31) / 32);
            size_t used = kHeader + size_t(12) * size_t(n) + sizeof(unsigned) * words;
            used = (used + 255) & ~size_t(255);
            double *partial = reinterpret_cast<double *>(base + used);
            const int64_t partial_cap = (int64_t)((kScratchBytes - used) / sizeof(double));
            cudaError_t e = cudaMemsetAsync(len, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(listed, 0, sizeof(unsigned) * words, s);
            if (e != cudaSuccess) st = gwn::set_error(GWN_ERR_CUDA, cudaGetErrorString(e));
            else
                st = gwn::launch_classify_on_scratch(m, q, n, label, w_or_null ? w_or_null : w_tmp, chi, list, len,
                                                     listed, partial, partial_cap, s);
        }
    }
    if (prev >= 0 && prev != m->device) cudaSetDevice(prev);
    return st;
}
