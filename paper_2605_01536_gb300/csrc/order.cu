// Spatial order of a query batch.  The crossing count walks the BVH once per
// query, and the boundary kernel decides per warp and boundary tile whether
// its cancellation test is needed; both do best when the queries of a warp lie
// close together.  Large batches are therefore evaluated in the order of the
// Morton codes of the queries in the mesh's box (the build's own radix sort),
// and the results are scattered back to the caller's order.  Each query's
// arithmetic does not depend on its neighbours, so the order changes
// no result.  Batches of many meshes are ordered the same way within each
// mesh's range of queries.
#include "gwn_internal.cuh"

namespace gwn {

namespace {

constexpr int TB = 256;

__device__ __forceinline__ uint32_t spread10q(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// The sort keys keep the top 24 bits of the codes (8 per axis, 256^3 cells of
// the box): as coherent for a warp as 30 and one radix pass fewer (measured 3%
// of the degenerate precision workload's classify step).
constexpr int kOrderBits = 24;

// 30-bit Morton code of p in box = (min x, min y, min z, max x, max y, max z);
// points outside the box are clamped onto it (NaN coordinates count as the minimum)
__device__ __forceinline__ uint32_t morton_in_box(const float *__restrict__ p, const float *__restrict__ box) {
    uint32_t c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = box[k], ext = box[3 + k] - lo;
        float u = ext > 0.f ? (p[k] - lo) / ext : 0.f;
        u = fminf(fmaxf(u, 0.f), 1.f);   // fmaxf(NaN, 0) = 0
        c[k] = min((uint32_t)(u * 1024.0f), 1023u);
    }
    return (spread10q(c[0]) << 2) | (spread10q(c[1]) << 1) | spread10q(c[2]);
}

// box: the mesh's vertex box
__global__ void k_query_morton(const float *__restrict__ q, int64_t n, const float *__restrict__ box,
                               uint32_t *__restrict__ keys, uint32_t *__restrict__ ids) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = morton_in_box(q + 3 * i, box) >> (30 - kOrderBits);
    ids[i] = (uint32_t)i;
}

// Batch key of query i: its mesh index (found in the meshes' query offsets)
// above the Morton code in that mesh's box, so that the sort keeps every mesh's
// queries together and orders each range in space.
__global__ void k_batch_keys(const float *__restrict__ q, int64_t n, const int64_t *__restrict__ mesh_off,
                             int n_mesh, const BatchMesh *__restrict__ meshes, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ ids) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_mesh - 1;   // mesh_off[lo] <= i < mesh_off[lo + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mesh_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    keys[i] = (uint64_t)lo << kOrderBits | morton_in_box(q + 3 * i, meshes[lo].box) >> (30 - kOrderBits);
    ids[i] = (uint32_t)i;
}

// keys of listed queries (list: indices into q)
__global__ void k_list_morton(const float *__restrict__ q, const int32_t *__restrict__ list, int64_t n,
                              const float *__restrict__ box, uint32_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = morton_in_box(q + 3 * (int64_t)list[i], box) >> (30 - kOrderBits);
}

__global__ void k_gather_queries(const float *__restrict__ q, const uint32_t *__restrict__ perm, int64_t n,
                                 float *__restrict__ qs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    qs[3 * i] = q[3 * j];
    qs[3 * i + 1] = q[3 * j + 1];
    qs[3 * i + 2] = q[3 * j + 2];
}

template <class T>
__global__ void k_scatter(const T *__restrict__ in, const uint32_t *__restrict__ perm, int64_t n, T *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[perm[i]] = in[i];
}

}  // namespace

gwn_status order_queries(const gwn_mesh *m, const float *q, int64_t n, uint32_t *keys, uint32_t *perm, float *qs,
                         cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    if (n > (int64_t)0xffffffffu) return set_error(GWN_ERR_INVALID_ARG, "too many queries to order");
    ProfScope prof("query_order", s);
    k_query_morton<<<grid_for(n, TB), TB, 0, s>>>(q, n, m->box, keys, perm);
    gwn_status st = radix_sort_u32(keys, perm, n, kOrderBits, s);
    if (st != GWN_OK) return st;
    k_gather_queries<<<grid_for(n, TB), TB, 0, s>>>(q, perm, n, qs);
    note_launches(2);
    GWN_LAUNCH_CHECK("query order");
    return GWN_OK;
}

gwn_status order_query_list(const gwn_mesh *m, const float *q, int32_t *list, int64_t n, cudaStream_t s) {
    if (n < kOrderMinQueries) return GWN_OK;
    if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "too many queries to order");
    ProfScope prof("query_order", s);
    uint32_t *keys = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&keys, sizeof(uint32_t) * n, s));
    k_list_morton<<<grid_for(n, TB), TB, 0, s>>>(q, list, n, m->box, keys);
    note_launches(1);
    gwn_status st = radix_sort_u32(keys, reinterpret_cast<uint32_t *>(list), n, kOrderBits, s);
    cudaFreeAsync(keys, s);
    if (st != GWN_OK) return st;
    GWN_LAUNCH_CHECK("query list order");
    return GWN_OK;
}

gwn_status order_batch_queries(const float *q, int64_t n, const int64_t *mesh_off, int n_mesh,
                               const BatchMesh *meshes, uint64_t *keys, uint32_t *perm, float *qs, cudaStream_t s) {
    if (n <= 0 || n_mesh <= 0) return GWN_OK;
    if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "too many queries to order");
    int mbits = 0;
    while ((1 << mbits) < n_mesh) ++mbits;
    k_batch_keys<<<grid_for(n, TB), TB, 0, s>>>(q, n, mesh_off, n_mesh, meshes, keys, perm);
    gwn_status st = radix_sort_u64(keys, perm, n, kOrderBits + mbits, s);
    if (st != GWN_OK) return st;
    k_gather_queries<<<grid_for(n, TB), TB, 0, s>>>(q, perm, n, qs);
    GWN_LAUNCH_CHECK("batch query order");
    return GWN_OK;
}

gwn_status scatter_f32(const float *in, const uint32_t *perm, int64_t n, float *out, cudaStream_t s) {
    if (n <= 0 || !out) return GWN_OK;
    ProfScope prof("scatter", s);
    k_scatter<float><<<grid_for(n, TB), TB, 0, s>>>(in, perm, n, out);
    GWN_LAUNCH_CHECK("scatter");
    return GWN_OK;
}

gwn_status scatter_i32(const int32_t *in, const uint32_t *perm, int64_t n, int32_t *out, cudaStream_t s) {
    if (n <= 0 || !out) return GWN_OK;
    ProfScope prof("scatter", s);
    k_scatter<int32_t><<<grid_for(n, TB), TB, 0, s>>>(in, perm, n, out);
    GWN_LAUNCH_CHECK("scatter");
    return GWN_OK;
}

gwn_status scatter_u8(const uint8_t *in, const uint32_t *perm, int64_t n, uint8_t *out, cudaStream_t s) {
    if (n <= 0 || !out) return GWN_OK;
    ProfScope prof("scatter", s);
    k_scatter<uint8_t><<<grid_for(n, TB), TB, 0, s>>>(in, perm, n, out);
    GWN_LAUNCH_CHECK("scatter");
    return GWN_OK;
}

}  // namespace gwn
