// Acceleration build: oriented boundary extraction + chaining, and the LBVH.
//
// Boundary (Sec. 4.1, Eq. 9): the auxiliary triangles of an interior edge cancel
// in pairs, so only the oriented boundary dM contributes.  Treated as a 1-chain:
// every face contributes its three directed edges; an undirected edge {u, v}
// (matched by vertex index) has net multiplicity m = #(u->v) - #(v->u) and
// appears |m| times in its net direction.  Steps: sort the 3 nt half-edge keys,
// segmented sum of the signs, compaction.  Edges are then chained into closed
// loops (the boundary of a 2-chain is a cycle: in-degree = out-degree at every
// vertex) so that consecutive edges share their common point in the query
// kernel.
//
// LBVH (replaces the paper's Embree BVH, Sec. 5): 30-bit Morton codes of the
// triangle centroids, radix sort, Karras' binary radix tree (Karras 2012),
// bottom-up box refit, and depth-first escape links for stackless traversal.
#include "gwn_internal.cuh"
#include "traverse.cuh"

namespace gwn {

namespace {

constexpr int TB = 256;

// ------------------------------------------------------------ boundary ----

__global__ void k_halfedge_keys(const int32_t *__restrict__ F, int64_t nt, int64_t nv,
                                uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * nt) return;
    int64_t t = i / 3;
    int e = (int)(i % 3);
    int64_t u = F[3 * t + e], v = F[3 * t + (e + 1) % 3];
    int64_t lo = u < v ? u : v, hi = u < v ? v : u;
    // a half-edge from a vertex to itself (repeated index in a degenerate face)
    // is a zero chain and contributes nothing: mark it with sign code 2
    keys[i] = (uint64_t)(lo * nv + hi);
    vals[i] = (u == v) ? 2u : (u < v ? 1u : 0u);
}

__global__ void k_seg_heads(const uint64_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_seg_sum(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                          const uint32_t *__restrict__ head, const uint32_t *__restrict__ head_scan,
                          int64_t n, int32_t *__restrict__ mult, uint64_t *__restrict__ seg_key) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t seg = head_scan[i] + head[i] - 1u;
    if (head[i]) seg_key[seg] = keys[i];
    uint32_t v = vals[i];
    if (v != 2u) atomicAdd(&mult[seg], v ? 1 : -1);
}

__global__ void k_abs(const int32_t *__restrict__ mult, int64_t nseg, uint32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    int32_t m = mult[i];
    cnt[i] = (uint32_t)(m < 0 ? -m : m);
}

__global__ void k_emit_edges(const int32_t *__restrict__ mult, const uint64_t *__restrict__ seg_key,
                             const uint32_t *__restrict__ off, int64_t nseg, int64_t nv,
                             int32_t *__restrict__ edges) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    int32_t m = mult[i];
    if (m == 0) return;
    int64_t key = (int64_t)seg_key[i];
    int32_t lo = (int32_t)(key / nv), hi = (int32_t)(key % nv);
    int32_t a = m > 0 ? lo : hi, b = m > 0 ? hi : lo;
    int32_t c = m < 0 ? -m : m;
    for (int32_t r = 0; r < c; ++r) {
        edges[2 * (off[i] + r)] = a;
        edges[2 * (off[i] + r) + 1] = b;
    }
}

// keys for sorting edges by start (which = 0) or end (which = 1) vertex
__global__ void k_edge_vertex_keys(const int32_t *__restrict__ edges, int64_t nb, int which,
                                   uint32_t *__restrict__ keys, uint32_t *__restrict__ ids) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    keys[i] = (uint32_t)edges[2 * i + which];
    ids[i] = (uint32_t)i;
}

// in-degree = out-degree at every vertex, so the vertex segments of the two
// sorted lists start at the same positions: pair the p-th incoming edge with
// the p-th outgoing edge.
__global__ void k_pair_succ(const uint32_t *__restrict__ in_ids, const uint32_t *__restrict__ out_ids,
                            int64_t nb, uint32_t *__restrict__ succ) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nb) return;
    succ[in_ids[p]] = out_ids[p];
}

__global__ void k_init_rep(const uint32_t *__restrict__ succ, int64_t nb, uint32_t *rep, uint32_t *nxt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    rep[e] = (uint32_t)e;
    nxt[e] = succ[e];
}

// one pointer-jumping round of the cycle minimum
__global__ void k_jump_min(const uint32_t *__restrict__ rep_in, const uint32_t *__restrict__ nxt_in, int64_t nb,
                           uint32_t *__restrict__ rep_out, uint32_t *__restrict__ nxt_out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    uint32_t n = nxt_in[e];
    rep_out[e] = min(rep_in[e], rep_in[n]);
    nxt_out[e] = nxt_in[n];
}

// list ranking: cut each cycle in front of its representative
__global__ void k_init_rank(const uint32_t *__restrict__ succ, const uint32_t *__restrict__ rep, int64_t nb,
                            uint32_t *dist, int32_t *nxt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    uint32_t s = succ[e];
    bool last = (s == rep[e]);
    nxt[e] = last ? -1 : (int32_t)s;
    dist[e] = last ? 0u : 1u;
}

__global__ void k_jump_rank(const uint32_t *__restrict__ dist_in, const int32_t *__restrict__ nxt_in, int64_t nb,
                            uint32_t *__restrict__ dist_out, int32_t *__restrict__ nxt_out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    int32_t n = nxt_in[e];
    if (n < 0) {
        dist_out[e] = dist_in[e];
        nxt_out[e] = -1;
    } else {
        dist_out[e] = dist_in[e] + dist_in[n];
        nxt_out[e] = nxt_in[n];
    }
}

// points per loop (length + 1 closing point), stored at the representative
__global__ void k_loop_sizes(const uint32_t *__restrict__ rep, const uint32_t *__restrict__ dist, int64_t nb,
                             uint32_t *__restrict__ size) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    size[e] = (rep[e] == (uint32_t)e) ? dist[e] + 2u : 0u;   // dist at the head = length - 1
}

__global__ void k_emit_chained(const int32_t *__restrict__ edges, const uint32_t *__restrict__ rep,
                               const uint32_t *__restrict__ dist, const uint32_t *__restrict__ loop_off,
                               const float4 *__restrict__ V, int64_t nb, int64_t npts,
                               float4 *__restrict__ pts) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    uint32_t r = rep[e];
    if (r >= nb) return;
    uint32_t len = dist[r] + 1u;
    uint32_t pos = len - 1u - dist[e];
    uint32_t base = loop_off[r];
    if ((int64_t)base + len >= npts || pos >= len) return;   // never write outside the point array
    float4 p = V[edges[2 * e]];
    p.w = 1.0f;
    pts[base + pos] = p;
    if (e == (int64_t)r) {   // closing point: back to the loop's first vertex
        float4 c = V[edges[2 * e]];
        c.w = 0.0f;
        pts[base + len] = c;
    }
}

__global__ void k_emit_unchained(const int32_t *__restrict__ edges, const float4 *__restrict__ V, int64_t nb,
                                 float4 *__restrict__ pts) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    float4 a = V[edges[2 * e]], b = V[edges[2 * e + 1]];
    a.w = 1.0f;
    b.w = 0.0f;
    pts[2 * e] = a;
    pts[2 * e + 1] = b;
}

// Loops are laid out in the order of the Morton code (in the box of the
// boundary's points) of their first point, so that a tile of consecutive
// points covers a compact region and the boundary kernel can skip its
// cancellation test for the many queries far from it.
__global__ void k_edge_start_bounds(const int32_t *__restrict__ edges, const float4 *__restrict__ V, int64_t nb,
                                    int *__restrict__ bounds /* 6: min xyz, max xyz (ordered ints) */);
__global__ void k_loop_keys(const uint32_t *__restrict__ rep, const int32_t *__restrict__ edges,
                            const float4 *__restrict__ V, int64_t nb, const int *__restrict__ bounds,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ ids);

__global__ void k_gather_sizes(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ size, int64_t nb,
                               uint32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    out[i] = size[ids[i]];
}

__global__ void k_scatter_offsets(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ off, int64_t nb,
                                  uint32_t *__restrict__ loop_off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    loop_off[ids[i]] = off[i];
}

__global__ void k_count_heads(const uint32_t *__restrict__ rep, int64_t nb, unsigned long long *count) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    if (rep[e] == (uint32_t)e) atomicAdd(count, 1ull);
}

// ------------------------------------------------------------------ BVH ----

__device__ __forceinline__ int ordered_key(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float from_ordered_key(int k) {
    return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

__global__ void k_centroid_bounds(const float4 *__restrict__ V, const int32_t *__restrict__ F, int64_t nt,
                                  int *__restrict__ bounds /* 6: min xyz, max xyz (ordered ints) */) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float c[3] = {0.f, 0.f, 0.f};
    bool valid = t < nt;
    if (valid) {
        float4 a = V[F[3 * t]], b = V[F[3 * t + 1]], d = V[F[3 * t + 2]];
        c[0] = (a.x + b.x + d.x) * (1.0f / 3.0f);
        c[1] = (a.y + b.y + d.y) * (1.0f / 3.0f);
        c[2] = (a.z + b.z + d.z) * (1.0f / 3.0f);
    }
    for (int k = 0; k < 3; ++k) {
        int kmin = valid ? ordered_key(c[k]) : 0x7fffffff;
        int kmax = valid ? ordered_key(c[k]) : (int)0x80000000;
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bounds[k], kmin);
            atomicMax(&bounds[3 + k], kmax);
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t morton30(float x, float y, float z, const int *__restrict__ bounds) {
    const float c[3] = {x, y, z};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        const float lo = from_ordered_key(bounds[k]), hi = from_ordered_key(bounds[3 + k]);
        const float ext = hi - lo;
        float u = ext > 0.f ? (c[k] - lo) / ext : 0.f;
        u = fminf(fmaxf(u, 0.f), 1.f);
        q[k] = min((uint32_t)(u * 1024.0f), 1023u);
    }
    return (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
}

__global__ void k_edge_start_bounds(const int32_t *__restrict__ edges, const float4 *__restrict__ V, int64_t nb,
                                    int *__restrict__ bounds) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = e < nb;
    float c[3] = {0.f, 0.f, 0.f};
    if (valid) {
        const float4 p = V[edges[2 * e]];
        c[0] = p.x; c[1] = p.y; c[2] = p.z;
    }
    for (int k = 0; k < 3; ++k) {
        int kmin = valid ? ordered_key(c[k]) : 0x7fffffff;
        int kmax = valid ? ordered_key(c[k]) : (int)0x80000000;
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bounds[k], kmin);
            atomicMax(&bounds[3 + k], kmax);
        }
    }
}

// key of a loop's representative edge: the Morton code of its start point;
// every other edge sorts after all loops (bit 30)
__global__ void k_loop_keys(const uint32_t *__restrict__ rep, const int32_t *__restrict__ edges,
                            const float4 *__restrict__ V, int64_t nb, const int *__restrict__ bounds,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ ids) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    uint32_t key = 1u << 30;
    if (rep[e] == (uint32_t)e) {
        const float4 p = V[edges[2 * e]];
        key = morton30(p.x, p.y, p.z, bounds);
    }
    keys[e] = key;
    ids[e] = (uint32_t)e;
}

__device__ __forceinline__ uint32_t spread15(uint32_t v) {
    v &= 0x7fffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// 30-bit Morton code of each triangle's centroid in the centroids' box: over x,
// y and z (dims = 3), or over x and y only (dims = 2: a tree of columns, which
// +z rays from neighbouring queries walk alike)
__global__ void k_morton(const float4 *__restrict__ V, const int32_t *__restrict__ F, int64_t nt,
                         const int *__restrict__ bounds, int dims, uint32_t *__restrict__ codes,
                         uint32_t *__restrict__ ids) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float4 a = V[F[3 * t]], b = V[F[3 * t + 1]], d = V[F[3 * t + 2]];
    float c[3] = {(a.x + b.x + d.x) * (1.0f / 3.0f), (a.y + b.y + d.y) * (1.0f / 3.0f),
                  (a.z + b.z + d.z) * (1.0f / 3.0f)};
    const float cells = dims == 2 ? 32768.0f : 1024.0f;
    const uint32_t top = dims == 2 ? 32767u : 1023u;
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        float lo = from_ordered_key(bounds[k]), hi = from_ordered_key(bounds[3 + k]);
        float ext = hi - lo;
        float u = ext > 0.f ? (c[k] - lo) / ext : 0.f;
        u = fminf(fmaxf(u, 0.f), 1.f);
        q[k] = min((uint32_t)(u * cells), top);
    }
    codes[t] = dims == 2 ? (spread15(q[0]) << 1) | spread15(q[1])
                         : (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    ids[t] = (uint32_t)t;
}

// Node tests of the +z walks from nsample points spread uniformly over the
// mesh's vertex box (a fixed hash sequence), summed into *visits: the cost the
// two candidate trees are compared by.  Their leaves are the same triangles
// (a triangle's leaf box admits the same rays in either tree), so the walks
// differ only in the internal nodes they test.
__device__ __forceinline__ float hash_unit(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return (float)(x >> 8) * (1.0f / 16777216.0f);
}

__global__ void k_tree_sample_visits(const gwn::BvhNode *__restrict__ nodes, int64_t nnodes,
                                     const float *__restrict__ box, int nsample,
                                     unsigned long long *__restrict__ counters,
                                     unsigned long long *__restrict__ visits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned nv = 0;
    if (i < nsample) {
        const float3 p = make_float3(box[0] + (box[3] - box[0]) * hash_unit(3u * i + 1u),
                                     box[1] + (box[4] - box[1]) * hash_unit(3u * i + 2u),
                                     box[2] + (box[5] - box[2]) * hash_unit(3u * i + 3u));
        bvh_walk_up<false, true>(p, nodes, nnodes, nullptr, counters, [](int, float3, float3, float3) {}, 0.f, &nv,
                                 false);
    }
    unsigned long long a = nv;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(visits, a);
}

__device__ __forceinline__ int delta(const uint32_t *codes, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    uint32_t a = codes[i], b = codes[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Karras 2012: internal node i covers leaves [min(i,j), max(i,j)]; its split
// gamma gives children gamma (left) and gamma + 1 (right), leaves when the
// child's range is a single leaf.  Node numbering: internal i -> i, leaf k ->
// (n - 1) + k.
__global__ void k_karras(const uint32_t *__restrict__ codes, int64_t n, int32_t *__restrict__ left,
                         int32_t *__restrict__ right, int32_t *__restrict__ parent, int32_t *__restrict__ first,
                         int32_t *__restrict__ last) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(codes, n, i, i - d);
    int64_t lmax = 2;
    while (delta(codes, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(codes, n, i, j);
    int64_t s = 0, div = 2, t;
    do {
        t = (l + div - 1) / div;
        if (delta(codes, n, i, i + (s + t) * d) > dnode) s += t;
        div <<= 1;
    } while (t > 1);
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int32_t lc = (lo == gamma) ? (int32_t)(n - 1 + gamma) : (int32_t)gamma;
    int32_t rc = (hi == gamma + 1) ? (int32_t)(n - 1 + gamma + 1) : (int32_t)(gamma + 1);
    left[i] = lc;
    right[i] = rc;
    parent[lc] = (int32_t)i;
    parent[rc] = (int32_t)i;
    first[i] = (int32_t)lo;
    last[i] = (int32_t)hi;
}

__global__ void k_leaves(const float4 *__restrict__ V, const int32_t *__restrict__ F, const uint32_t *__restrict__ ids,
                         int64_t n, gwn::BvhNode *__restrict__ nodes, float4 *__restrict__ leaf_tri) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t t = ids[k];
    float4 a = V[F[3 * t]], b = V[F[3 * t + 1]], c = V[F[3 * t + 2]];
    a.w = b.w = c.w = 0.f;
    leaf_tri[3 * k] = a;
    leaf_tri[3 * k + 1] = b;
    leaf_tri[3 * k + 2] = c;
    gwn::BvhNode nd;
    nd.xmin = fminf(a.x, fminf(b.x, c.x));
    nd.xmax = fmaxf(a.x, fmaxf(b.x, c.x));
    nd.ymin = fminf(a.y, fminf(b.y, c.y));
    nd.ymax = fmaxf(a.y, fmaxf(b.y, c.y));
    nd.zmax = fmaxf(a.z, fmaxf(b.z, c.z));
    nd.child = (int32_t)k;
    nd.skip = -1;
    nd.is_leaf = 1;
    nodes[n - 1 + k] = nd;
}

// bottom-up refit: the second thread to reach a node merges its children
__global__ void k_refit(int64_t n, const int32_t *__restrict__ parent, const int32_t *__restrict__ left,
                        const int32_t *__restrict__ right, gwn::BvhNode *nodes, unsigned *visits) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || n < 2) return;
    int32_t node = (int32_t)(n - 1 + k);
    for (int level = 0; level < 256; ++level) {   // Karras depth <= 63 (30-bit codes + index bits)
        int32_t p = parent[node];
        if (p < 0 || p >= n - 1) break;
        __threadfence();
        if (atomicAdd(&visits[p], 1u) == 0u) break;
        __threadfence();
        const gwn::BvhNode *L = nodes + left[p], *R = nodes + right[p];
        float lxmin = __ldcg(&L->xmin), lxmax = __ldcg(&L->xmax), lymin = __ldcg(&L->ymin),
              lymax = __ldcg(&L->ymax), lzmax = __ldcg(&L->zmax);
        float rxmin = __ldcg(&R->xmin), rxmax = __ldcg(&R->xmax), rymin = __ldcg(&R->ymin),
              rymax = __ldcg(&R->ymax), rzmax = __ldcg(&R->zmax);
        gwn::BvhNode *P = nodes + p;
        __stcg(&P->xmin, fminf(lxmin, rxmin));
        __stcg(&P->xmax, fmaxf(lxmax, rxmax));
        __stcg(&P->ymin, fminf(lymin, rymin));
        __stcg(&P->ymax, fmaxf(lymax, rymax));
        __stcg(&P->zmax, fmaxf(lzmax, rzmax));
        __stcg(&P->child, left[p]);
        __stcg(&P->is_leaf, 0);
        node = p;
    }
}

// Escape link of a node covering leaves [f, l]: the next subtree in depth-first
// order is rooted at the right sibling of the lowest ancestor-or-self that is a
// left child; its parent splits at l, so that sibling is leaf l+1 or internal
// node l+1 (the latter exactly when internal l+1 starts at l+1).
__global__ void k_skip(int64_t n, const int32_t *__restrict__ first, const int32_t *__restrict__ last,
                       gwn::BvhNode *__restrict__ nodes) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * n - 1) return;
    int64_t l = (x < n - 1) ? last[x] : x - (n - 1);
    int32_t s;
    if (l == n - 1) s = -1;
    else if (l + 1 <= n - 2 && first[l + 1] == l + 1) s = (int32_t)(l + 1);
    else s = (int32_t)(n - 1 + l + 1);
    nodes[x].skip = s;
}

__global__ void k_vertex_bounds(const float4 *__restrict__ V, int64_t nv, int *__restrict__ bounds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < nv;
    const float4 p = valid ? V[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float c[3] = {p.x, p.y, p.z};
    for (int k = 0; k < 3; ++k) {
        int kmin = valid ? ordered_key(c[k]) : 0x7fffffff;
        int kmax = valid ? ordered_key(c[k]) : (int)0x80000000;
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bounds[k], kmin);
            atomicMax(&bounds[3 + k], kmax);
        }
    }
}

__global__ void k_bounds_to_box(const int *__restrict__ bounds, float *__restrict__ box) {
    if (threadIdx.x < 6) box[threadIdx.x] = from_ordered_key(bounds[threadIdx.x]);
}

}  // namespace

gwn_status build_boundary(gwn_mesh *m, cudaStream_t s) {
    const int64_t nh = 3 * m->nt;
    m->nb = 0;
    m->npts = 0;
    m->nloops = 0;
    if (m->bedges) { cudaFree(m->bedges); m->bedges = nullptr; }
    if (m->bpts) { cudaFree(m->bpts); m->bpts = nullptr; }
    if (nh == 0) return GWN_OK;
    uint64_t *keys = nullptr, *seg_key = nullptr;
    uint32_t *vals = nullptr, *head = nullptr, *hscan = nullptr, *cnt = nullptr, *off = nullptr, *tot = nullptr;
    int32_t *mult = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&keys, sizeof(uint64_t) * nh, s));
    GWN_CUDA_TRY(cudaMallocAsync(&vals, sizeof(uint32_t) * nh, s));
    GWN_CUDA_TRY(cudaMallocAsync(&head, sizeof(uint32_t) * nh, s));
    GWN_CUDA_TRY(cudaMallocAsync(&hscan, sizeof(uint32_t) * nh, s));
    GWN_CUDA_TRY(cudaMallocAsync(&tot, sizeof(uint32_t) * 2, s));
    k_halfedge_keys<<<grid_for(nh, TB), TB, 0, s>>>(m->F, m->nt, m->nv, keys, vals);
    int bits = 1;
    while (bits < 64 && ((unsigned __int128)1 << bits) <= (unsigned __int128)m->nv * (unsigned __int128)m->nv) ++bits;
    gwn_status st = radix_sort_u64(keys, vals, nh, bits, s);
    if (st != GWN_OK) return st;
    k_seg_heads<<<grid_for(nh, TB), TB, 0, s>>>(keys, nh, head);
    if ((st = exclusive_scan_u32(head, hscan, nh, tot, s)) != GWN_OK) return st;
    uint32_t nseg_h = 0;
    GWN_CUDA_TRY(cudaMemcpyAsync(&nseg_h, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nseg = nseg_h;
    GWN_CUDA_TRY(cudaMallocAsync(&mult, sizeof(int32_t) * nseg, s));
    GWN_CUDA_TRY(cudaMallocAsync(&seg_key, sizeof(uint64_t) * nseg, s));
    GWN_CUDA_TRY(cudaMallocAsync(&cnt, sizeof(uint32_t) * nseg, s));
    GWN_CUDA_TRY(cudaMallocAsync(&off, sizeof(uint32_t) * nseg, s));
    GWN_CUDA_TRY(cudaMemsetAsync(mult, 0, sizeof(int32_t) * nseg, s));
    k_seg_sum<<<grid_for(nh, TB), TB, 0, s>>>(keys, vals, head, hscan, nh, mult, seg_key);
    k_abs<<<grid_for(nseg, TB), TB, 0, s>>>(mult, nseg, cnt);
    if ((st = exclusive_scan_u32(cnt, off, nseg, tot + 1, s)) != GWN_OK) return st;
    uint32_t nb_h = 0;
    GWN_CUDA_TRY(cudaMemcpyAsync(&nb_h, tot + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    m->nb = nb_h;
    if (m->nb > 0) {
        GWN_CUDA_TRY(cudaMalloc(&m->bedges, sizeof(int32_t) * 2 * m->nb));
        k_emit_edges<<<grid_for(nseg, TB), TB, 0, s>>>(mult, seg_key, off, nseg, m->nv, m->bedges);
    }
    cudaFreeAsync(keys, s);
    cudaFreeAsync(vals, s);
    cudaFreeAsync(head, s);
    cudaFreeAsync(hscan, s);
    cudaFreeAsync(mult, s);
    cudaFreeAsync(seg_key, s);
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(off, s);
    GWN_LAUNCH_CHECK("boundary extraction");
    if (m->nb == 0) {
        cudaFreeAsync(tot, s);
        return GWN_OK;
    }

    const int64_t nb = m->nb;
    if (m->cfg.chain_boundary < 0) {
        m->npts = 2 * nb;
        m->nloops = nb;
        GWN_CUDA_TRY(cudaMalloc(&m->bpts, sizeof(float4) * m->npts));
        k_emit_unchained<<<grid_for(nb, TB), TB, 0, s>>>(m->bedges, m->V, nb, m->bpts);
        cudaFreeAsync(tot, s);
        GWN_LAUNCH_CHECK("boundary points");
        return GWN_OK;
    }

    // ---- chaining into loops
    uint32_t *kin = nullptr, *idin = nullptr, *kout = nullptr, *idout = nullptr, *succ = nullptr;
    uint32_t *rep[2] = {nullptr, nullptr}, *nx[2] = {nullptr, nullptr}, *dist[2] = {nullptr, nullptr};
    int32_t *rnx[2] = {nullptr, nullptr};
    uint32_t *lsize = nullptr, *loff = nullptr;
    unsigned long long *nl = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&kin, sizeof(uint32_t) * nb, s));
    GWN_CUDA_TRY(cudaMallocAsync(&idin, sizeof(uint32_t) * nb, s));
    GWN_CUDA_TRY(cudaMallocAsync(&kout, sizeof(uint32_t) * nb, s));
    GWN_CUDA_TRY(cudaMallocAsync(&idout, sizeof(uint32_t) * nb, s));
    GWN_CUDA_TRY(cudaMallocAsync(&succ, sizeof(uint32_t) * nb, s));
    for (int b = 0; b < 2; ++b) {
        GWN_CUDA_TRY(cudaMallocAsync(&rep[b], sizeof(uint32_t) * nb, s));
        GWN_CUDA_TRY(cudaMallocAsync(&nx[b], sizeof(uint32_t) * nb, s));
        GWN_CUDA_TRY(cudaMallocAsync(&dist[b], sizeof(uint32_t) * nb, s));
        GWN_CUDA_TRY(cudaMallocAsync(&rnx[b], sizeof(int32_t) * nb, s));
    }
    GWN_CUDA_TRY(cudaMallocAsync(&lsize, sizeof(uint32_t) * nb, s));
    GWN_CUDA_TRY(cudaMallocAsync(&loff, sizeof(uint32_t) * nb, s));
    GWN_CUDA_TRY(cudaMallocAsync(&nl, sizeof(unsigned long long), s));
    int vbits = 1;
    while (vbits < 32 && ((int64_t)1 << vbits) <= m->nv) ++vbits;
    k_edge_vertex_keys<<<grid_for(nb, TB), TB, 0, s>>>(m->bedges, nb, 1, kin, idin);
    if ((st = radix_sort_u32(kin, idin, nb, vbits, s)) != GWN_OK) return st;
    k_edge_vertex_keys<<<grid_for(nb, TB), TB, 0, s>>>(m->bedges, nb, 0, kout, idout);
    if ((st = radix_sort_u32(kout, idout, nb, vbits, s)) != GWN_OK) return st;
    k_pair_succ<<<grid_for(nb, TB), TB, 0, s>>>(idin, idout, nb, succ);
    int rounds = 1;
    while (((int64_t)1 << rounds) < nb) ++rounds;
    rounds += 1;
    k_init_rep<<<grid_for(nb, TB), TB, 0, s>>>(succ, nb, rep[0], nx[0]);
    int cur = 0;
    for (int r = 0; r < rounds; ++r) {
        k_jump_min<<<grid_for(nb, TB), TB, 0, s>>>(rep[cur], nx[cur], nb, rep[cur ^ 1], nx[cur ^ 1]);
        cur ^= 1;
    }
    uint32_t *repf = rep[cur];
    k_init_rank<<<grid_for(nb, TB), TB, 0, s>>>(succ, repf, nb, dist[0], rnx[0]);
    int cd = 0;
    for (int r = 0; r < rounds; ++r) {
        k_jump_rank<<<grid_for(nb, TB), TB, 0, s>>>(dist[cd], rnx[cd], nb, dist[cd ^ 1], rnx[cd ^ 1]);
        cd ^= 1;
    }
    uint32_t *distf = dist[cd];
    k_loop_sizes<<<grid_for(nb, TB), TB, 0, s>>>(repf, distf, nb, lsize);
    {   // loops in the Morton order of their first points
        int *bnd = nullptr;
        const int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
        GWN_CUDA_TRY(cudaMallocAsync(&bnd, sizeof(init), s));
        GWN_CUDA_TRY(cudaMemcpyAsync(bnd, init, sizeof(init), cudaMemcpyHostToDevice, s));
        k_edge_start_bounds<<<grid_for(nb, TB), TB, 0, s>>>(m->bedges, m->V, nb, bnd);
        // kin / idin / kout are free again: loop keys, representative ids, permuted sizes
        k_loop_keys<<<grid_for(nb, TB), TB, 0, s>>>(repf, m->bedges, m->V, nb, bnd, kin, idin);
        if ((st = radix_sort_u32(kin, idin, nb, 31, s)) != GWN_OK) return st;
        k_gather_sizes<<<grid_for(nb, TB), TB, 0, s>>>(idin, lsize, nb, kout);
        if ((st = exclusive_scan_u32(kout, kout, nb, tot, s)) != GWN_OK) return st;
        k_scatter_offsets<<<grid_for(nb, TB), TB, 0, s>>>(idin, kout, nb, loff);
        cudaFreeAsync(bnd, s);
    }
    GWN_CUDA_TRY(cudaMemsetAsync(nl, 0, sizeof(unsigned long long), s));
    k_count_heads<<<grid_for(nb, TB), TB, 0, s>>>(repf, nb, nl);
    uint32_t npts_h = 0;
    unsigned long long nl_h = 0;
    GWN_CUDA_TRY(cudaMemcpyAsync(&npts_h, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GWN_CUDA_TRY(cudaMemcpyAsync(&nl_h, nl, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    m->npts = npts_h;
    m->nloops = (int64_t)nl_h;
    GWN_CUDA_TRY(cudaMalloc(&m->bpts, sizeof(float4) * m->npts));
    k_emit_chained<<<grid_for(nb, TB), TB, 0, s>>>(m->bedges, repf, distf, loff, m->V, nb, m->npts, m->bpts);
    for (void *p : {(void *)kin, (void *)idin, (void *)kout, (void *)idout, (void *)succ, (void *)lsize,
                    (void *)loff, (void *)nl, (void *)tot})
        cudaFreeAsync(p, s);
    for (int b = 0; b < 2; ++b) {
        cudaFreeAsync(rep[b], s);
        cudaFreeAsync(nx[b], s);
        cudaFreeAsync(dist[b], s);
        cudaFreeAsync(rnx[b], s);
    }
    GWN_LAUNCH_CHECK("boundary chaining");
    return GWN_OK;
}

gwn_status build_box(gwn_mesh *m, cudaStream_t s) {
    if (!m->box) GWN_CUDA_TRY(cudaMalloc(&m->box, sizeof(float) * 6));
    if (m->nv == 0) {
        GWN_CUDA_TRY(cudaMemsetAsync(m->box, 0, sizeof(float) * 6, s));
        return GWN_OK;
    }
    int *bounds = nullptr;
    const int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
    GWN_CUDA_TRY(cudaMallocAsync(&bounds, sizeof(init), s));
    GWN_CUDA_TRY(cudaMemcpyAsync(bounds, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_vertex_bounds<<<grid_for(m->nv, TB), TB, 0, s>>>(m->V, m->nv, bounds);
    k_bounds_to_box<<<1, 32, 0, s>>>(bounds, m->box);
    cudaFreeAsync(bounds, s);
    GWN_LAUNCH_CHECK("vertex box");
    return GWN_OK;
}

// One LBVH over the triangles: Morton codes over dims axes, radix sort, Karras
// hierarchy, leaves in sorted order, bottom-up refit, escape links.
static gwn_status build_tree(const gwn_mesh *m, int dims, const int *bounds, gwn::BvhNode *nodes,
                             float4 *leaf_tri, cudaStream_t s) {
    const int64_t n = m->nt;
    uint32_t *codes = nullptr, *ids = nullptr;
    int32_t *left = nullptr, *right = nullptr, *parent = nullptr, *first = nullptr, *last = nullptr;
    unsigned *visits = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&codes, sizeof(uint32_t) * n, s));
    GWN_CUDA_TRY(cudaMallocAsync(&ids, sizeof(uint32_t) * n, s));
    const int64_t ni = n > 1 ? n - 1 : 1;
    GWN_CUDA_TRY(cudaMallocAsync(&left, sizeof(int32_t) * ni, s));
    GWN_CUDA_TRY(cudaMallocAsync(&right, sizeof(int32_t) * ni, s));
    GWN_CUDA_TRY(cudaMallocAsync(&first, sizeof(int32_t) * ni, s));
    GWN_CUDA_TRY(cudaMallocAsync(&last, sizeof(int32_t) * ni, s));
    GWN_CUDA_TRY(cudaMallocAsync(&parent, sizeof(int32_t) * (2 * n - 1), s));
    GWN_CUDA_TRY(cudaMallocAsync(&visits, sizeof(unsigned) * ni, s));
    GWN_CUDA_TRY(cudaMemsetAsync(parent, 0xff, sizeof(int32_t) * (2 * n - 1), s));
    GWN_CUDA_TRY(cudaMemsetAsync(visits, 0, sizeof(unsigned) * ni, s));
    k_morton<<<grid_for(n, TB), TB, 0, s>>>(m->V, m->F, n, bounds, dims, codes, ids);
    gwn_status st = radix_sort_u32(codes, ids, n, 30, s);
    if (st == GWN_OK) {
        if (n > 1) k_karras<<<grid_for(n - 1, TB), TB, 0, s>>>(codes, n, left, right, parent, first, last);
        k_leaves<<<grid_for(n, TB), TB, 0, s>>>(m->V, m->F, ids, n, nodes, leaf_tri);
        if (n > 1) k_refit<<<grid_for(n, TB), TB, 0, s>>>(n, parent, left, right, nodes, visits);
        k_skip<<<grid_for(2 * n - 1, TB), TB, 0, s>>>(n, first, last, nodes);
    }
    for (void *p : {(void *)codes, (void *)ids, (void *)left, (void *)right, (void *)parent, (void *)first,
                    (void *)last, (void *)visits})
        cudaFreeAsync(p, s);
    if (st != GWN_OK) return st;
    GWN_LAUNCH_CHECK("bvh build");
    return GWN_OK;
}

// Both a tree over xyz Morton codes and one over xy codes (columns: the +z rays
// of neighbouring queries share their paths) are built, and the one whose
// walks from a fixed sample of points test fewer nodes (k_tree_sample_visits)
// is kept.  Measured on the soup8 mesh: 57 instead of 99 node tests per query
// for the xy tree; random soups of large overlapping triangles keep the xyz
// tree, whose zmax bounds prune better there.
constexpr int kTreeSamples = 4096;
gwn_status build_bvh(gwn_mesh *m, cudaStream_t s) {
    const int64_t n = m->nt;
    if (m->nodes) { cudaFree(m->nodes); m->nodes = nullptr; }
    if (m->leaf_tri) { cudaFree(m->leaf_tri); m->leaf_tri = nullptr; }
    m->nnodes = 0;
    if (n == 0) return GWN_OK;
    m->nnodes = 2 * n - 1;
    gwn::BvhNode *nodes[2] = {nullptr, nullptr};
    float4 *leaf[2] = {nullptr, nullptr};
    int *bounds = nullptr;
    unsigned long long *visits = nullptr;
    auto cleanup = [&]() {
        for (int t = 0; t < 2; ++t) {
            if (nodes[t]) cudaFree(nodes[t]);
            if (leaf[t]) cudaFree(leaf[t]);
        }
    };
    for (int t = 0; t < 2; ++t) {
        cudaError_t e;
        if ((e = cudaMalloc(&nodes[t], sizeof(gwn::BvhNode) * m->nnodes)) != cudaSuccess ||
            (e = cudaMalloc(&leaf[t], sizeof(float4) * 3 * n)) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return set_error(GWN_ERR_OOM, std::string("bvh: ") + cudaGetErrorString(e));
        }
    }
    GWN_CUDA_TRY(cudaMallocAsync(&bounds, sizeof(int) * 6, s));
    GWN_CUDA_TRY(cudaMallocAsync(&visits, sizeof(unsigned long long) * 2, s));
    const int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
    GWN_CUDA_TRY(cudaMemcpyAsync(bounds, init, sizeof(init), cudaMemcpyHostToDevice, s));
    GWN_CUDA_TRY(cudaMemsetAsync(visits, 0, sizeof(unsigned long long) * 2, s));
    k_centroid_bounds<<<grid_for(n, TB), TB, 0, s>>>(m->V, m->F, n, bounds);
    gwn_status st = GWN_OK;
    for (int t = 0; t < 2 && st == GWN_OK; ++t) {
        st = build_tree(m, t == 0 ? 3 : 2, bounds, nodes[t], leaf[t], s);
        if (st == GWN_OK)
            k_tree_sample_visits<<<grid_for(kTreeSamples, TB), TB, 0, s>>>(nodes[t], m->nnodes, m->box, kTreeSamples,
                                                                            m->counters, visits + t);
    }
    unsigned long long cost_h[2] = {0, 0};
    if (st == GWN_OK) {
        cudaError_t e = cudaMemcpyAsync(cost_h, visits, sizeof(cost_h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = set_error(GWN_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFreeAsync(bounds, s);
    cudaFreeAsync(visits, s);
    if (st != GWN_OK) {
        cleanup();
        return st;
    }
    const int keep = cost_h[1] < cost_h[0] ? 1 : 0;
    m->nodes = nodes[keep];
    m->leaf_tri = leaf[keep];
    m->bvh_xy = keep == 1;
    cudaFree(nodes[1 - keep]);
    cudaFree(leaf[1 - keep]);
    GWN_LAUNCH_CHECK("bvh build");
    return GWN_OK;
}

}  // namespace gwn
