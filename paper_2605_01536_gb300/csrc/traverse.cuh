// Stackless walk of the escape-linked BVH for a +z ray, shared by the
// per-query crossing count and the grid (ray-reuse) kernels.
#pragma once

#include "gwn_internal.cuh"
#include "predicates.cuh"
#include "quant.cuh"

namespace gwn {

// Visit every leaf whose node box admits the +z ray from p (p.xy inside the
// closed xy box and p.z <= zmax, every bound widened by pad), in depth-first
// order, calling on_leaf(slot, a, b, c) with the leaf's triangle slot and
// vertices.  Returns false (and sets the traversal error flag) if the walk
// leaves the node array or exceeds its node budget (a corrupt tree), so it
// never loops or reads out of range.  Count = true adds the nodes read to
// *visits (the instrumented walk; the timed kernels compile without it);
// read_leaves = false skips the leaves' triangles (node counting only).
template <bool Padded = false, bool Count = false, class OnLeaf>
__device__ __forceinline__ bool bvh_walk_up(float3 p, const BvhNode *__restrict__ nodes, int64_t nnodes,
                                            const float4 *__restrict__ tri, unsigned long long *__restrict__ counters,
                                            OnLeaf &&on_leaf, float pad = 0.f, unsigned *visits = nullptr,
                                            bool read_leaves = true) {
    int node = nnodes > 0 ? 0 : -1;
    int64_t budget = nnodes + 1;   // depth-first order visits each node at most once
    while (node >= 0) {
        if constexpr (Count) ++*visits;
        if (--budget < 0 || node >= nnodes) {
            atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
            return false;
        }
        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
        const float4 b0 = __ldg(np);
        const float4 b1 = __ldg(np + 1);
        const int child = __float_as_int(b1.y), skip = __float_as_int(b1.z), leaf = __float_as_int(b1.w);
        const bool hit = Padded ? (p.x >= b0.x - pad && p.x <= b0.y + pad && p.y >= b0.z - pad &&
                                   p.y <= b0.w + pad && p.z <= b1.x + pad)
                                : (p.x >= b0.x && p.x <= b0.y && p.y >= b0.z && p.y <= b0.w && p.z <= b1.x);
        if (hit && leaf) {
            if ((unsigned)child >= (unsigned)((nnodes + 1) / 2)) {
                atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
                return false;
            }
            if (read_leaves) {
                const float4 a = __ldg(tri + 3 * child), bb = __ldg(tri + 3 * child + 1),
                             cc = __ldg(tri + 3 * child + 2);
                on_leaf(child, make_float3(a.x, a.y, a.z), make_float3(bb.x, bb.y, bb.z),
                        make_float3(cc.x, cc.y, cc.z));
            }
            node = skip;
        } else {
            node = hit ? child : skip;
        }
    }
    return true;
}

// The walk of bvh_walk_up taken by the 32 lanes of a warp together, with the
// leaves postponed so that the warp tests them in step: a lane that reaches a
// hit leaf holds it and walks on; reaching a second one it stops; the warp
// tests one held leaf per lane once the lanes holding a leaf are at least twice
// as many as those still looking for their first, or when no lane can walk
// (measured against 1x, 4x and "none looking": the leaf-heavy degenerate
// precision workload gains up to 25% with later phases, the node-heavy soup8
// walk loses up to 14%; 2x keeps soup8 and takes 9% of the gain).
// Each lane visits the same leaves in the same order as bvh_walk_up (on_leaf
// gets the same calls), and its node budget counts the same visits.  Every
// lane of the warp must call it; a lane without a query passes active = false.
template <class OnLeaf>
__device__ __forceinline__ bool bvh_walk_up_warp(bool active, float3 p, const BvhNode *__restrict__ nodes,
                                                 int64_t nnodes, const float4 *__restrict__ tri,
                                                 unsigned long long *__restrict__ counters, OnLeaf &&on_leaf) {
    int node = active && nnodes > 0 ? 0 : -1;
    int held = -1, next = -1;   // the leaf to test next and the one after it
    int64_t budget = nnodes + 1;
    bool ok = true;
    const unsigned nleaves = (unsigned)((nnodes + 1) / 2);
    while (true) {
        const bool movable = node >= 0 && next < 0;
        const unsigned holders = __ballot_sync(0xffffffffu, held >= 0);
        const unsigned movers = __ballot_sync(0xffffffffu, movable);
        if (!holders && !movers) break;
        const unsigned searching = movers & ~holders;
        if (holders && (!searching || __popc(holders) >= 2 * __popc(searching))) {
            if (held >= 0) {
                const float4 a = __ldg(tri + 3 * held), bb = __ldg(tri + 3 * held + 1), cc = __ldg(tri + 3 * held + 2);
                on_leaf(held, make_float3(a.x, a.y, a.z), make_float3(bb.x, bb.y, bb.z),
                        make_float3(cc.x, cc.y, cc.z));
                held = next;
                next = -1;
            }
            continue;
        }
        if (!movable) continue;
        if (--budget < 0 || node >= nnodes) {
            atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
            ok = false;
            node = held = next = -1;
            continue;
        }
        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
        const float4 b0 = __ldg(np);
        const float4 b1 = __ldg(np + 1);
        const int child = __float_as_int(b1.y), skip = __float_as_int(b1.z), leaf = __float_as_int(b1.w);
        const bool hit = p.x >= b0.x && p.x <= b0.y && p.y >= b0.z && p.y <= b0.w && p.z <= b1.x;
        if (hit && leaf) {
            if ((unsigned)child >= nleaves) {
                atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
                ok = false;
                node = held = next = -1;
                continue;
            }
            if (held < 0) held = child;
            else next = child;
            node = skip;
        } else {
            node = hit ? child : skip;
        }
    }
    return ok;
}

// Signed +z crossing count of one query with the snapped (fixed-point)
// predicates of a mesh built with quantize_bits: the float boxes are widened by
// one quantum so that snapping never hides a crossing.
static __device__ __noinline__ int chi_one_q(float3 p, const BvhNode *__restrict__ nodes, int64_t nnodes,
                                      const float4 *__restrict__ tri, unsigned long long *__restrict__ counters,
                                      const QFrame *qf) {
    const long long qx = qcoord(p.x, qf->cx, qf->scale), qy = qcoord(p.y, qf->cy, qf->scale),
                    qz = qcoord(p.z, qf->cz, qf->scale);
    const int4 *lq = qf->leaf_q;
    int c = 0;
    const bool ok = bvh_walk_up<true>(
        p, nodes, nnodes, tri, counters,
        [&](int slot, float3, float3, float3) {
            c += tri_crossing_q(qx, qy, qz, lq[3 * slot], lq[3 * slot + 1], lq[3 * slot + 2]);
        },
        qf->pad);
    return ok ? c : INT32_MIN;
}

// Signed +z crossing count of one query with the predicates decided exactly on
// the FP32 inputs (Sec. 3.2, Supp. S2.1).  INT32_MIN on a corrupt tree.
__device__ __forceinline__ int chi_one_exact(float3 p, const BvhNode *__restrict__ nodes, int64_t nnodes,
                                             const float4 *__restrict__ tri,
                                             unsigned long long *__restrict__ counters) {
    int c = 0;
    const bool ok = bvh_walk_up(p, nodes, nnodes, tri, counters, [&](int, float3 a, float3 b, float3 cc) {
        c += tri_crossing(p, a, b, cc, &counters[CNT_EXACT_EDGE], &counters[CNT_EXACT_PLANE]);
    });
    return ok ? c : INT32_MIN;
}

// Signed +z crossing count of one query in the mesh's predicate mode (exact on
// the FP32 inputs, or fixed point), read from its status block.
__device__ __forceinline__ int chi_one(float3 p, const BvhNode *__restrict__ nodes, int64_t nnodes,
                                       const float4 *__restrict__ tri, unsigned long long *__restrict__ counters) {
    const QFrame *qf = qframe(counters);
    if (qf->bits) return chi_one_q(p, nodes, nnodes, tri, counters, qf);
    int c = 0;
    const bool ok = bvh_walk_up(p, nodes, nnodes, tri, counters, [&](int, float3 a, float3 b, float3 cc) {
        c += tri_crossing(p, a, b, cc, &counters[CNT_EXACT_EDGE], &counters[CNT_EXACT_PLANE]);
    });
    return ok ? c : INT32_MIN;
}

}  // namespace gwn
