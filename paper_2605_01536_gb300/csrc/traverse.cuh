// Stackless walk of the escape-linked BVH for a +z ray, shared by the
// per-query crossing count and the grid (ray-reuse) kernels.
#pragma once

#include "gwn_internal.cuh"
#include "predicates.cuh"

namespace gwn {

// Visit every leaf whose node box admits the +z ray from p (p.xy inside the
// closed xy box and p.z <= zmax), in depth-first order, calling
// on_leaf(a, b, c) with the leaf triangle.  Returns false (and sets the
// traversal error flag) if the walk leaves the node array or exceeds its node
// budget (a corrupt tree), so it never loops or reads out of range.
template <class OnLeaf>
__device__ __forceinline__ bool bvh_walk_up(float3 p, const BvhNode *__restrict__ nodes, int64_t nnodes,
                                            const float4 *__restrict__ tri, unsigned long long *__restrict__ counters,
                                            OnLeaf &&on_leaf) {
    int node = nnodes > 0 ? 0 : -1;
    int64_t budget = nnodes + 1;   // depth-first order visits each node at most once
    while (node >= 0) {
        if (--budget < 0 || node >= nnodes) {
            atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
            return false;
        }
        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
        const float4 b0 = __ldg(np);
        const float4 b1 = __ldg(np + 1);
        const int child = __float_as_int(b1.y), skip = __float_as_int(b1.z), leaf = __float_as_int(b1.w);
        const bool hit = p.x >= b0.x && p.x <= b0.y && p.y >= b0.z && p.y <= b0.w && p.z <= b1.x;
        if (hit && leaf) {
            if ((unsigned)child >= (unsigned)((nnodes + 1) / 2)) {
                atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
                return false;
            }
            const float4 a = __ldg(tri + 3 * child), bb = __ldg(tri + 3 * child + 1), cc = __ldg(tri + 3 * child + 2);
            on_leaf(make_float3(a.x, a.y, a.z), make_float3(bb.x, bb.y, bb.z), make_float3(cc.x, cc.y, cc.z));
            node = skip;
        } else {
            node = hit ? child : skip;
        }
    }
    return true;
}

// Signed +z crossing count of one query (Sec. 3.2 with the perturbed
// predicates of Supp. S2.1).  INT32_MIN on a corrupt tree.
__device__ __forceinline__ int chi_one(float3 p, const BvhNode *__restrict__ nodes, int64_t nnodes,
                                       const float4 *__restrict__ tri, unsigned long long *__restrict__ counters) {
    int c = 0;
    const bool ok = bvh_walk_up(p, nodes, nnodes, tri, counters, [&](float3 a, float3 b, float3 cc) {
        c += tri_crossing(p, a, b, cc, &counters[CNT_EXACT_EDGE], &counters[CNT_EXACT_PLANE]);
    });
    return ok ? c : INT32_MIN;
}

}  // namespace gwn
