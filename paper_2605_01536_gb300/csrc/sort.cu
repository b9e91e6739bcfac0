// Device-wide exclusive scan and stable LSD radix sort (8-bit digits).
//
// Used by the acceleration build: Morton codes of triangle centroids for the
// LBVH, and undirected half-edge keys for the boundary extraction.
//
// Radix pass (per 8-bit digit), three kernels:
//   1. per-tile digit histogram, written digit-major: counts[d * ntiles + t];
//   2. exclusive scan of the counts, giving each (digit, tile) its first output
//      slot; digit-major order makes the sort stable across tiles;
//   3. scatter: each tile walks its keys in input order, 256 at a time; a key's
//      slot is its (digit, tile) base + keys of the same digit in earlier rounds
//      + same digit in earlier warps of this round + same digit in lower lanes
//      (__match_any_sync), which keeps the order of equal digits.
#include "gwn_internal.cuh"

namespace gwn {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t warp_prefix = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void k_chunk_sums(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_chunk_scan(const uint32_t *in, int64_t n, const uint32_t *__restrict__ offsets,
                             uint32_t *out, uint32_t *total_out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, &total) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) *total_out = run;
}

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_digit_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                           uint32_t *__restrict__ counts, int ntiles) {
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&hist[(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_digit_scatter(const K *__restrict__ keys_in,
                                                              const uint32_t *__restrict__ vals_in,
                                                              K *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                                                              int64_t n, int shift,
                                                              const uint32_t *__restrict__ offsets, int ntiles) {
    __shared__ uint32_t warp_cnt[RS_WARPS][256];
    __shared__ uint32_t running[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    running[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int w = 0; w < RS_WARPS; ++w) warp_cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + r * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        K key = valid ? keys_in[i] : K(0);
        uint32_t val = valid ? vals_in[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 0xffu) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) warp_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t s = running[threadIdx.x];
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = warp_cnt[w][threadIdx.x];
                warp_cnt[w][threadIdx.x] = s;
                s += c;
            }
            running[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = warp_cnt[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

template <typename K>
gwn_status radix_sort_impl(K *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return GWN_OK;
    if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "radix sort: too many keys");
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    const int64_t ncounts = (int64_t)ntiles * 256;
    K *k2 = nullptr;
    uint32_t *v2 = nullptr, *counts = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&k2, sizeof(K) * n, s));
    GWN_CUDA_TRY(cudaMallocAsync(&v2, sizeof(uint32_t) * n, s));
    GWN_CUDA_TRY(cudaMallocAsync(&counts, sizeof(uint32_t) * ncounts, s));
    K *kin = keys, *kout = k2;
    uint32_t *vin = vals, *vout = v2;
    gwn_status st = GWN_OK;
    for (int shift = 0; shift < bits; shift += 8) {
        k_digit_hist<K><<<ntiles, RS_THREADS, 0, s>>>(kin, n, shift, counts, ntiles);
        note_launches(2);   // with k_digit_scatter
        st = exclusive_scan_u32(counts, counts, ncounts, nullptr, s);
        if (st != GWN_OK) break;
        k_digit_scatter<K><<<ntiles, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, shift, counts, ntiles);
        K *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    if (st == GWN_OK && kin != keys) {
        cudaMemcpyAsync(keys, kin, sizeof(K) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    cudaFreeAsync(k2, s);
    cudaFreeAsync(v2, s);
    cudaFreeAsync(counts, s);
    if (st != GWN_OK) return st;
    GWN_LAUNCH_CHECK("radix sort");
    return GWN_OK;
}

}  // namespace

gwn_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, cudaStream_t s) {
    if (n <= 0) {
        if (total) GWN_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(uint32_t), s));
        return GWN_OK;
    }
    const int64_t nchunks = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nchunks == 1) {
        k_chunk_scan<<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out, total);
        note_launches(1);
        GWN_LAUNCH_CHECK("scan");
        return GWN_OK;
    }
    uint32_t *sums = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&sums, sizeof(uint32_t) * nchunks, s));
    k_chunk_sums<<<(unsigned)nchunks, SCAN_THREADS, 0, s>>>(in, n, sums);
    note_launches(2);   // with k_chunk_scan
    gwn_status st = exclusive_scan_u32(sums, sums, nchunks, nullptr, s);
    if (st == GWN_OK) k_chunk_scan<<<(unsigned)nchunks, SCAN_THREADS, 0, s>>>(in, n, sums, out, total);
    cudaFreeAsync(sums, s);
    if (st != GWN_OK) return st;
    GWN_LAUNCH_CHECK("scan");
    return GWN_OK;
}

gwn_status radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    return radix_sort_impl<uint32_t>(keys, vals, n, bits, s);
}

gwn_status radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    return radix_sort_impl<uint64_t>(keys, vals, n, bits, s);
}

}  // namespace gwn
