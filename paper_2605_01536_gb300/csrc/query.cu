// Query kernels: crossing number (BVH traversal), boundary-curve sum, combine /
// classify with FP64 re-evaluation, and the direct solid-angle sum.
//
// Antipodal evaluation (Eq. 9, Algorithm 1 with x0 = +z, x1 = -z):
//   w(q) = chi(q) + (1/2pi) * sum_{(a,b) in dM} atan2(n_ab, d_ab)
// since Area(A, B, x1) = 2 atan2(n, d).  With a = p_a - q, b = p_b - q,
// l = |a|, the van Oosterom-Strackee numerator and denominator scaled by the
// positive factor l_a l_b are
//   n = x1 . (a x b) = a_y b_x - a_x b_y
//   d = l_a l_b + l_b x1.a + l_a x1.b + a.b = h_a h_b + a_x b_x + a_y b_y,
//   h = l - a_z,
// (the denominator of Supp. S4's Algorithm 3 rearranged).  h is computed as
// (a_x^2 + a_y^2) / (l + a_z) when a_z > 0, which keeps d accurate when a vertex
// lies nearly straight above the query, where the plain form cancels.
#include <algorithm>
#include <type_traits>

#include "gwn_internal.cuh"
#include "predicates.cuh"
#include "atan_poly.cuh"
#include "fp32x2.cuh"
#include "traverse.cuh"

namespace gwn {

namespace {

constexpr double kInv2Pi = 0.15915494309189533577;
constexpr float kPiF = 3.14159265358979f;

// Launched in blocks of 128 threads (compiled for up to 256): finer tails than
// 256 (measured 5.6% faster on 2M soup8 queries, bit-identical).
constexpr int kChiThreads = 128;

// Fixed selects the predicate mode at compile time (the host knows the mesh's
// quantize_bits), so the exact kernel carries none of the fixed-point code.
template <bool Fixed>
__global__ void __launch_bounds__(256) k_chi(const float *__restrict__ q, int64_t n,
                                             const BvhNode *__restrict__ nodes, int64_t nnodes,
                                             const float4 *__restrict__ tri, int32_t *__restrict__ chi,
                                             unsigned long long *__restrict__ counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (Fixed) {
        if (i >= n) return;
        const float3 p = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
        chi[i] = chi_one_q(p, nodes, nnodes, tri, counters, qframe(counters));
    } else {   // the warp walks together (bvh_walk_up_warp): every lane stays to the end
        const bool active = i < n;
        const float3 p = active ? make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]) : make_float3(0.f, 0.f, 0.f);
        int c = 0;
        const bool ok = bvh_walk_up_warp(active, p, nodes, nnodes, tri, counters,
                                         [&](int, float3 a, float3 b, float3 cc) {
                                             c += tri_crossing(p, a, b, cc, &counters[CNT_EXACT_EDGE],
                                                               &counters[CNT_EXACT_PLANE]);
                                         });
        if (active) chi[i] = ok ? c : INT32_MIN;
    }
}

// The crossing count of k_chi<false>, instrumented: the BVH nodes read and the
// triangles tested, summed over the queries into visits[0] and visits[1].
__global__ void __launch_bounds__(256) k_chi_visits(const float *__restrict__ q, int64_t n,
                                                    const BvhNode *__restrict__ nodes, int64_t nnodes,
                                                    const float4 *__restrict__ tri, int32_t *__restrict__ chi,
                                                    unsigned long long *__restrict__ counters,
                                                    unsigned long long *__restrict__ visits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned nv = 0, nt = 0;
    if (i < n) {
        const float3 p = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
        int c = 0;
        const bool ok = bvh_walk_up<false, true>(
            p, nodes, nnodes, tri, counters,
            [&](int, float3 a, float3 b, float3 cc) {
                ++nt;
                c += tri_crossing(p, a, b, cc, &counters[CNT_EXACT_EDGE], &counters[CNT_EXACT_PLANE]);
            },
            0.f, &nv);
        chi[i] = ok ? c : INT32_MIN;
    }
    unsigned long long a = nv, b = nt;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&visits[0], a);
        atomicAdd(&visits[1], b);
    }
}

// ------------------------------------------------------ boundary terms ----

// atan2 for the hot loops: octant reduction to t = min/max in [0, 1], then
// atan(t) = t P(t^2) with the minimax polynomial of atan_poly.cuh (fitted by
// fit_atan.py), then the octant is undone.  Branch-free.  Callers never pass
// (0, 0).  The larger magnitude is clamped to the smallest normal float only
// to keep the approximate reciprocal finite; every operand the kernels pass is
// a normal number (an accepted group product is at least (4.9e-5)^8 ~ 3e-35),
// so the clamp never changes a result.
constexpr float kFltMin = 1.17549435e-38f;
__device__ __forceinline__ float fast_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(fmaxf(ax, ay), kFltMin), mn = fminf(ax, ay);
    const float t = mn * sfu_rcp(mx);
    const float s = t * t;
    float r = gwn_atan_poly(s) * t;
    r = ay > ax ? 1.57079632679489662f - r : r;
    r = x < 0.f ? 3.14159265358979324f - r : r;
    return copysignf(r, y);
}

// Unit vector from the query to a boundary point, kept as (A_x, A_y, H) with
// H = 1 - A_z computed without cancellation: (A_x^2 + A_y^2) / (1 + A_z) when
// A_z > 0.  The point coincident with the query gives (0, 0, 0).  With two such
// vectors A, B the van Oosterom-Strackee numerator and denominator of
// Area(A, B, x1) / 2 for x1 = (0, 0, -1) are
//   n = A.(B x x1) = A_y B_x - A_x B_y,
//   d = 1 + A.B + A.x1 + B.x1 = H_a H_b + A_x B_x + A_y B_y.
struct PointRel {
    float ax, ay, h;
};

// Limit of atan2(n, d) for the edge (u, v) when u lies exactly on the query's
// vertical ray (u - q = (0, 0, h), h > 0): the perturbed unit vector to u is
// (-e1/h, -e2/h, 1), so n ~ e1 r_y - e2 r_x and d ~ -e1 r_x - e2 r_y with
// r = v - q; hence atan2(r_y, -r_x), and for r_y = 0 the e2 order gives -pi
// (r_x > 0) or 0 (r_x < 0).
__device__ __forceinline__ float apex_angle(float rx, float ry, bool &degenerate) {
    if (ry != 0.f) return atan2f(ry, -rx);
    if (rx > 0.f) return -kPiF;
    if (rx < 0.f) return 0.f;
    degenerate = true;
    return 0.f;
}

// Rare path of one edge term: n = d = 0 (a boundary vertex straight above the
// query, or the query on the edge), or d <= 0 with |n| within its rounding
// bound (the atan2 branch cut, where the sign of n is the exact perturbed sign
// of the 2-D edge classification, Supp. S2.1).
__device__ __noinline__ float edge_angle_slow(float4 Pa, float4 Pb, float qx, float qy, float qz, float n, float d,
                                               unsigned long long *counters) {
    if (n == 0.f && d == 0.f) {
        const float ax = Pa.x - qx, ay = Pa.y - qy, az = Pa.z - qz;
        const float bx = Pb.x - qx, by = Pb.y - qy, bz = Pb.z - qz;
        bool deg = false;
        float t;
        const bool a_up = ax == 0.f && ay == 0.f, b_up = bx == 0.f && by == 0.f;
        if (a_up && !b_up && az > 0.f) {
            t = apex_angle(bx, by, deg);
        } else if (b_up && !a_up && bz > 0.f) {
            t = -apex_angle(ax, ay, deg);
        } else {
            deg = true;
            t = 0.f;
        }
        atomicAdd(&counters[deg ? CNT_DEGENERATE : CNT_APEX], 1ull);
        return t;
    }
    atomicAdd(&counters[CNT_EXACT_BRANCH], 1ull);
    const int s = branch_sos(qx, qy, Pa.x, Pa.y, Pb.x, Pb.y, counters);   // n ~ -classification
    const float mag = fabsf(n);
    return atan2f(s > 0 ? -mag : mag, d);
}

// One edge term atan2(n, d).  |n - n_exact| <= ~4u (|A_y B_x| + |A_x B_y|) + the
// rounding of the unit vectors; 1e-6 (|A_y B_x| + |A_x B_y|) + 1e-30 covers it
// with margin, so outside that band the FP32 sign of n is the exact one.
__device__ __forceinline__ float edge_term(float n, float d, const PointRel &A, const PointRel &B, float4 Pa,
                                           float4 Pb, float qx, float qy, float qz, unsigned long long *counters) {
    if (d <= 0.f && fabsf(n) <= fmaf(1e-6f, fabsf(A.ay * B.ax) + fabsf(A.ax * B.ay), 1e-30f))
        return edge_angle_slow(Pa, Pb, qx, qy, qz, n, d, counters);
    return fast_atan2(n, d);
}

struct PointRel2 {
    float2 ax, ay, h;
};

// point_rel for two queries (nqx, nqy, nqz hold minus the query coordinates).
// H = 1 - A_z without a select: with g = 1 + |A_z|, hh = (A_x^2 + A_y^2) / g
// equals 1 - |A_z| (no cancellation), and H = hh + (|A_z| - A_z).
__device__ __forceinline__ PointRel2 point_rel2(float4 P, float2 nqx, float2 nqy, float2 nqz) {
    const float2 dx = add2(bc2(P.x), nqx), dy = add2(bc2(P.y), nqy), dz = add2(bc2(P.z), nqz);
    const float2 s = fma2(dx, dx, mul2(dy, dy));
    const float2 r2 = add2(fma2(dz, dz, s), bc2(1e-37f));    // > 0 even for a coincident point
    const float2 inv = make_float2(sfu_rsqrt(r2.x), sfu_rsqrt(r2.y));
    PointRel2 r;
    r.ax = mul2(dx, inv);
    r.ay = mul2(dy, inv);
    const float2 az = mul2(dz, inv);
    const float2 aaz = make_float2(fabsf(az.x), fabsf(az.y));
    const float2 g = add2(bc2(1.0f), aaz);
    const float2 hh = mul2(mul2(mul2(s, inv), inv), make_float2(sfu_rcp(g.x), sfu_rcp(g.y)));
    r.h = add2(hh, add2(aaz, neg2(az)));
    return r;
}


// fast_atan2 for two (y, x) pairs at once
__device__ __forceinline__ float2 fast_atan2_2(float2 y, float2 x) {
    const float axx = fabsf(x.x), axy = fabsf(x.y), ayx = fabsf(y.x), ayy = fabsf(y.y);
    const float mxx = fmaxf(fmaxf(axx, ayx), kFltMin), mxy = fmaxf(fmaxf(axy, ayy), kFltMin);
    const float2 t = mul2(make_float2(fminf(axx, ayx), fminf(axy, ayy)), make_float2(sfu_rcp(mxx), sfu_rcp(mxy)));
    const float2 s = mul2(t, t);
    float2 p = bc2(GWN_ATAN_C8);
    p = fma2(p, s, bc2(GWN_ATAN_C7));
    p = fma2(p, s, bc2(GWN_ATAN_C6));
    p = fma2(p, s, bc2(GWN_ATAN_C5));
    p = fma2(p, s, bc2(GWN_ATAN_C4));
    p = fma2(p, s, bc2(GWN_ATAN_C3));
    p = fma2(p, s, bc2(GWN_ATAN_C2));
    p = fma2(p, s, bc2(GWN_ATAN_C1));
    p = fma2(p, s, bc2(GWN_ATAN_C0));
    const float2 r = mul2(p, t);
    // undo the octant reduction: r -> A + B r with (A, B) from (|y| > |x|, x < 0)
    const bool fx1 = ayx > axx, fy1 = ayy > axy, fx2 = x.x < 0.f, fy2 = x.y < 0.f;
    const float2 A = make_float2(fx1 ? 1.57079632679489662f : (fx2 ? 3.14159265358979324f : 0.f),
                                 fy1 ? 1.57079632679489662f : (fy2 ? 3.14159265358979324f : 0.f));
    const float2 B = make_float2((fx1 != fx2) ? -1.f : 1.f, (fy1 != fy2) ? -1.f : 1.f);
    const float2 o = fma2(B, r, A);
    return make_float2(copysignf(o.x, y.x), copysignf(o.y, y.y));
}

// Terms are grouped GROUP edges at a time: each term's (d + i n) is multiplied
// into a running product, one atan2 per group.  The product's argument equals
// the sum of the accepted angles as long as it never passes +-pi, which either
// of two acceptance tests guarantees:
// - per term (the default for sparse boundaries): |n| < tan(pi/GROUP) d -
//   kAccept, each angle below pi/8 in magnitude, so 8 of them sum to less
//   than pi.  The test depends on the term alone, off the product's chain.
// - running (dense boundaries, where many terms are steep: on random soups
//   2.5% fail the per-term test, 0.35% this one): d > kMinD and the product
//   with the term keeps a positive real part.  By induction the argument
//   stays in (-pi/2, pi/2): an accepted angle is below pi/2 in magnitude
//   (d > 0), so the new argument lies in (-pi, pi), and a positive real part
//   puts it in (-pi/2, pi/2).  Rounding can only matter where the real part is
//   near zero, an argument near +-pi/2, where atan2 is continuous.  The test
//   sits on the product's chain (compare, then select), which costs 9% where
//   nearly every term passes either test.
// Both margins keep every accepted factor's modulus above 4.9e-5, so a product
// of 8 factors of modulus at most 4 neither underflows nor overflows.  A term
// that is not accepted (an edge seen steeply from the query, the atan2 branch
// cut, a vertex straight above) leaves the product unchanged and takes its own
// atan2, with the exact branch-cut sign and apex limit where they apply.
constexpr int GROUP = 8;
constexpr float kTanGroup = 0.41f;     // < tan(pi/8) = 0.41421
constexpr float kAccept = 2e-5f;
constexpr float kMinD = 5e-5f;

template <int KP>
struct BsumState {
    float2 re[KP], im[KP], part[KP], comp[KP];
};

// part + x as an unevaluated sum part + comp (Knuth's TwoSum, error folded into
// comp): keeps the FP32 running sum of group angles accurate to about one
// rounding however many groups a tile holds.
__device__ __forceinline__ void two_sum_acc2(float2 &part, float2 &comp, float2 x) {
    const float2 s = add2(part, x);
    const float2 bv = add2(s, neg2(part));
    const float2 av = add2(s, neg2(bv));
    const float2 err = add2(add2(part, neg2(av)), add2(x, neg2(bv)));
    comp = add2(comp, err);
    part = s;
}

__device__ __forceinline__ void two_sum_acc(float &part, float &comp, float x) {
    const float s = part + x;
    const float bv = s - part;
    const float av = s - bv;
    comp += (part - av) + (x - bv);
    part = s;
}

// Load the block's queries: thread t holds queries base + t + k * blockDim.x,
// k < 2 KP, as KP float2 pairs of negated coordinates (NaN past n).
template <int KP>
__device__ __forceinline__ void load_query_pairs(const float *__restrict__ q, int64_t base, int64_t n,
                                                 float2 (&nqx)[KP], float2 (&nqy)[KP], float2 (&nqz)[KP]) {
#pragma unroll
    for (int k = 0; k < 2 * KP; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        const bool ok = idx < n;
        const float nan = __int_as_float(0x7fc00000);
        const float x = ok ? -q[3 * idx] : nan, y = ok ? -q[3 * idx + 1] : nan, z = ok ? -q[3 * idx + 2] : nan;
        if (k & 1) { nqx[k >> 1].y = x; nqy[k >> 1].y = y; nqz[k >> 1].y = z; }
        else       { nqx[k >> 1].x = x; nqy[k >> 1].x = y; nqz[k >> 1].x = z; }
    }
}

// Boundary terms of the edges starting at points [e_begin, e_end) for the
// block's 2 KP queries per thread, added to the thread's FP64 accumulators in
// shared memory, s_acc[k * blockDim.x + threadIdx.x] (touched once per tile, so
// they need not occupy registers).  The
// block streams the chained points through shared memory (tile + 1 points);
// point j carries flag w = 1 when an edge runs from it to point j+1.  Every
// thread of the block must call it.
// Deferred fallback terms (the batched kernel's variant).  Where many terms
// fail the group test (dense soups: about 1 in 40), nearly every warp-edge has
// some failing lane, and computing the failing terms in place runs the scalar
// path once per query slot with most lanes idle.  Instead each warp appends its
// failing (query, edge) pairs to a queue in shared memory, entry
// j << 7 | k << 5 | lane (edge j of the tile, query slot k of that lane), and
// drains it with all 32 lanes once it holds 32 KQ entries and at the end of
// every tile.  Drained terms are added to per-query 64-bit fixed-point sums
// (units of 2^-40 rad) with integer atomics: exact, so the result does not
// depend on the order of the drain.
constexpr float kFixScale = 0x1p40f;

// Scalar twins of point_rel2 and edge_nd2: the same operations in the same
// order with explicit rounding (no contraction), so a drained term is computed
// from bit-identical n and d to the ones the group test saw.  Near n = d = 0
// (an apex seen almost head-on) atan2 is ill-conditioned enough that another
// rounding of the unit vectors moves the term by ~1e-5 rad.
__device__ __forceinline__ PointRel point_rel_twin(float4 P, float qx, float qy, float qz) {
    const float dx = __fadd_rn(P.x, -qx), dy = __fadd_rn(P.y, -qy), dz = __fadd_rn(P.z, -qz);
    const float s = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    const float r2 = __fadd_rn(__fmaf_rn(dz, dz, s), 1e-37f);
    const float inv = sfu_rsqrt(r2);
    PointRel r;
    r.ax = __fmul_rn(dx, inv);
    r.ay = __fmul_rn(dy, inv);
    const float az = __fmul_rn(dz, inv);
    const float aaz = fabsf(az);
    const float g = __fadd_rn(1.0f, aaz);
    const float hh = __fmul_rn(__fmul_rn(__fmul_rn(s, inv), inv), sfu_rcp(g));
    r.h = __fadd_rn(hh, __fadd_rn(aaz, -az));
    return r;
}

// Ill-conditioned terms: |d + i n| < 2^-6 H_a H_b.  A term's FP32 rounding
// error is a few units of rounding of the products that make up n and d,
// whose size is about H_a H_b where the term is ill-conditioned (the unit
// vectors to the edge's ends nearly opposite: the query close to the edge),
// divided by |d + i n|; below 2^-6 H_a H_b the amplification exceeds 64 and
// the term is recomputed in FP64 from the FP32 inputs, where the differences
// to the query are exact.  |d + i n|^2 = 2 (1 + A.B) H_a H_b for unit A, B, so
// this needs 1 + A.B < H_a H_b / 8192: A and B within 1/45 rad of opposite.
// The hot loop tests it (paired, the same arithmetic) only in warps near the
// boundary tile, and keeps such terms out of the group products.
constexpr float kCancel = 0x1p-6f;
__device__ __forceinline__ bool cancels(float n, float d, float ha, float hb) {
    const float t = kCancel * (ha * hb);
    return fmaf(n, n, d * d) < t * t;
}
__device__ double edge_angle64(float4 Pa, float4 Pb, float qx, float qy, float qz,
                               const unsigned long long *counters);

// The FP64 evaluation does not run inside the edge loop: its registers would
// crowd the loop's (a call to it from there cost 9% of the kernel).  A
// cancelling term found in the loop is put on a per-warp queue in shared
// memory, entry j << 7 | k << 5 | lane (edge j of the tile, query slot k of that
// lane), and the warp evaluates the queue in FP64 after the tile's edges, where
// the loop's registers are free; the results go to per-query 64-bit
// fixed-point sums (units of 2^-40 rad) with integer atomics, exact and
// independent of the order.  A queue that is full (more than kCancelCap such
// terms for one warp in one tile) lists the query for a full FP64
// re-evaluation instead (k_fp64_fix), once per query (the listed bits).
constexpr int kCancelCap = 64;
constexpr double kFixUnit = 0x1p-40;
constexpr double kFixScale64 = 0x1p40;

struct CancelQ {
    unsigned *queue;            // this warp's queue, kCancelCap entries
    int *count;                 // this warp's entry count
    long long *fix;             // fixed-point sums, fix[k blockDim.x + t]
    const float *q;             // the block's queries: slot k of thread t at q[3 (t + k blockDim.x)]
    int64_t qbase;              // caller's index of the block's query slot 0 of thread 0 (for the list)
    int32_t *list;              // queries for a full FP64 re-evaluation (NULL: count the term as
    unsigned long long *list_len;   //  an FP32 one and record it in CNT_CANCEL_OVERFLOW)
    unsigned *listed;           // one bit per query: already listed
};

// Put query idx on the FP64 re-evaluation list unless it is there already.
__device__ __forceinline__ void list_query(int64_t idx, int32_t *list, unsigned long long *list_len,
                                           unsigned *listed) {
    const unsigned bit = 1u << (idx & 31);
    if (atomicOr(&listed[idx >> 5], bit) & bit) return;
    list[atomicAdd(list_len, 1ull)] = (int32_t)idx;
}

// Queue a cancelling term; false when the queue is full and the query has been
// listed for a full FP64 re-evaluation (or there is no list).
__device__ __forceinline__ bool cancel_enqueue(const CancelQ &cq, int j, int k, int lane) {
    const int slot = atomicAdd(cq.count, 1);
    if (slot < kCancelCap) {
        cq.queue[slot] = (unsigned)j << 7 | (unsigned)k << 5 | (unsigned)lane;
        return true;
    }
    if (cq.list) list_query(cq.qbase + (threadIdx.x & ~31) + lane + (int64_t)k * blockDim.x, cq.list, cq.list_len,
                            cq.listed);
    return false;
}

// FP64 evaluation of this warp's queued terms (points of the staged tile); all
// 32 lanes of the warp call it, with the loop's registers out of use.
__device__ __noinline__ void cancel_drain(const CancelQ &cq, const float4 *s_pts, unsigned long long *counters) {
    __syncwarp();
    const int lane = threadIdx.x & 31, warp0 = threadIdx.x & ~31;
    const int count = min(*cq.count, kCancelCap);
    for (int r = lane; r < count; r += 32) {
        const unsigned e = cq.queue[r];
        const int owner = warp0 + (int)(e & 31u), k = (int)(e >> 5 & 3u), j = (int)(e >> 7);
        const int local = owner + k * (int)blockDim.x;
        const double t = edge_angle64(s_pts[j], s_pts[j + 1], cq.q[3 * local], cq.q[3 * local + 1],
                                      cq.q[3 * local + 2], counters);
        atomicAdd(reinterpret_cast<unsigned long long *>(cq.fix + (k * (int)blockDim.x + owner)),
                  (unsigned long long)__double2ll_rn(t * kFixScale64));
    }
    if (lane == 0 && count > 0) atomicAdd(&counters[CNT_CANCEL], (unsigned long long)count);
    __syncwarp();
    if (lane == 0) *cq.count = 0;
    __syncwarp();
}

// A term that failed the group test and does not cancel, from the n and d the
// test saw.  Out of line: it runs for a few terms in a thousand, and inlined its
// registers would crowd the group loop.
__device__ __noinline__ float fallback_term(float n, float d, PointRel a, PointRel b, float4 Pa, float4 Pb, float qx,
                                            float qy, float qz, unsigned long long *counters) {
    return edge_term(n, d, a, b, Pa, Pb, qx, qy, qz, counters);
}

struct BsumDefer {
    const float *q;            // the block's queries: query slot k of thread t at q[3 (t + k blockDim.x)]
    unsigned *queue;           // this warp's queue, 64 KQ entries
    long long *fix;            // fixed-point sums, fix[k blockDim.x + t]
};

// The deferred terms of the batched kernel, drained by all 32 lanes.  With
// Cond, a term whose d cancels goes on the cancellation queue (FP64 after the
// tile) instead; if that is full it is taken in FP32 and counted.
template <bool Cond>
__device__ __noinline__ void bsum_drain(const unsigned *queue, int count, const float4 *s_pts, const float *q,
                                        long long *fix, CancelQ cq, unsigned long long *counters) {
    const int lane = threadIdx.x & 31, warp0 = threadIdx.x & ~31;
    for (int r = lane; r < count; r += 32) {
        const unsigned e = queue[r];
        const int owner = warp0 + (int)(e & 31u), k = (int)(e >> 5 & 3u), j = (int)(e >> 7);
        const int local = owner + k * (int)blockDim.x;
        const float4 Pa = s_pts[j], Pb = s_pts[j + 1];
        const float qx = q[3 * local], qy = q[3 * local + 1], qz = q[3 * local + 2];
        const PointRel A = point_rel_twin(Pa, qx, qy, qz), B = point_rel_twin(Pb, qx, qy, qz);
        const float n = __fmaf_rn(A.ay, B.ax, -__fmul_rn(A.ax, B.ay));
        const float d = __fmaf_rn(A.h, B.h, __fmaf_rn(A.ax, B.ax, __fmul_rn(A.ay, B.ay)));
        if (Cond && cancels(n, d, A.h, B.h)) {
            const int slot = atomicAdd(cq.count, 1);
            if (slot < kCancelCap) {
                cq.queue[slot] = (unsigned)j << 7 | (unsigned)k << 5 | (unsigned)(e & 31u);
                continue;
            }
            if (cq.list) list_query(cq.qbase + local, cq.list, cq.list_len, cq.listed);
            else atomicAdd(&counters[CNT_CANCEL_OVERFLOW], 1ull);
        }
        const float t = edge_term(n, d, A, B, Pa, Pb, qx, qy, qz, counters);
        atomicAdd(reinterpret_cast<unsigned long long *>(fix + (k * (int)blockDim.x + owner)),
                  (unsigned long long)__float2ll_rn(t * kFixScale));
    }
    __syncwarp();
}

// Box of the staged tile's points (points 0..cnt) widened on every side by a
// tenth of its longest edge, into box[0..5] = (min x, max x, min y, max y,
// min z, max z) for every thread of the block.  An ill-conditioned term,
// |d + i n| < H_a H_b / 64, has |d + i n|^2 = 2 (1 + A.B) H_a H_b below
// (H_a H_b)^2 / 4096, so 1 + A.B < H_a H_b / 8192 <= 4.9e-4 (H_a H_b <= 4): the
// edge subtends an angle within 0.032 rad of pi, which puts the query within
// 0.032 L of the edge (L its length).  A tenth of the longest edge leaves a
// factor of three for rounding.  Contains barriers: every thread of the block
// must call it.
__device__ __noinline__ void tile_box(const float4 *s_pts, int cnt, float *box) {
    __shared__ float s_red[8][8];   // up to 8 warps x (3 minima, 3 maxima, edge length^2)
    float v[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.f};
    for (int i = threadIdx.x; i <= cnt; i += blockDim.x) {
        const float4 P = s_pts[i];
        v[0] = fminf(v[0], P.x); v[1] = fminf(v[1], P.y); v[2] = fminf(v[2], P.z);
        v[3] = fmaxf(v[3], P.x); v[4] = fmaxf(v[4], P.y); v[5] = fmaxf(v[5], P.z);
        if (i < cnt && P.w != 0.f) {
            const float4 Q = s_pts[i + 1];
            const float dx = Q.x - P.x, dy = Q.y - P.y, dz = Q.z - P.z;
            v[6] = fmaxf(v[6], dx * dx + dy * dy + dz * dz);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = fminf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
#pragma unroll
        for (int k = 3; k < 7; ++k) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    }
    const int warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 7; ++k) s_red[warp][k] = v[k];
    }
    __syncthreads();
    float r[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) r[k] = s_red[0][k];
    for (int w = 1; w < nwarps; ++w) {
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = fminf(r[k], s_red[w][k]);
#pragma unroll
        for (int k = 3; k < 7; ++k) r[k] = fmaxf(r[k], s_red[w][k]);
    }
    __syncthreads();   // s_red is reused by the next tile
    const float L = 0.1f * sqrtf(r[6]);
    box[0] = r[0] - L; box[1] = r[3] + L;
    box[2] = r[1] - L; box[3] = r[4] + L;
    box[4] = r[2] - L; box[5] = r[5] + L;
}

__device__ __forceinline__ bool in_box(const float *b, float x, float y, float z) {
    return x >= b[0] && x <= b[1] && y >= b[2] && y <= b[3] && z >= b[4] && z <= b[5];
}

template <int KP, bool Defer = false, bool Cond = false, bool Running = false>
__device__ __forceinline__ void bsum_accumulate(const float4 *__restrict__ pts, int64_t e_begin, int64_t e_end,
                                                int tile, float4 *s_pts, const float2 (&nqx)[KP],
                                                const float2 (&nqy)[KP], const float2 (&nqz)[KP],
                                                double *s_acc, unsigned long long *counters, CancelQ cq,
                                                BsumDefer dq = BsumDefer{}) {
    constexpr int KQ = 2 * KP;
    static_assert(!(Defer || Cond) || KQ <= 4, "queue entries hold a 2-bit query slot");
    BsumState<KP> st;
    int q_count = 0;   // entries in this warp's queue (warp-uniform)
    if constexpr (Defer || Cond) {
#pragma unroll
        for (int k = 0; k < KQ; ++k) cq.fix[k * blockDim.x + threadIdx.x] = 0;
        if ((threadIdx.x & 31) == 0) *cq.count = 0;
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        st.re[k] = bc2(1.f);
        st.im[k] = bc2(0.f);
        st.part[k] = bc2(0.f);
        st.comp[k] = bc2(0.f);
    }
    int g_count = 0;
    // close the current group: one atan2 of each query's product
    auto finalize = [&]() {
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            two_sum_acc2(st.part[k], st.comp[k], fast_atan2_2(st.im[k], st.re[k]));
            st.re[k] = bc2(1.f);
            st.im[k] = bc2(0.f);
        }
        g_count = 0;
    };

    // the edge point j -> j+1 with unit-vector data A (point j) and B (point j+1);
    // cond (std::true_type / std::false_type) selects the cancellation test
    auto add_edge = [&](auto cond, const PointRel2 *A, const PointRel2 *B, int j) {
        constexpr bool C = decltype(cond)::value;
        unsigned fail = 0;   // bit 2k + h: query half h of pair k takes its own atan2
        float2 en[KP], ed[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            en[k] = fma2(A[k].ay, B[k].ax, neg2(mul2(A[k].ax, B[k].ay)));
            const float2 pl = fma2(A[k].ax, B[k].ax, mul2(A[k].ay, B[k].ay));   // planar part of d
            ed[k] = fma2(A[k].h, B[k].h, pl);
            // a NaN (a padding query past n) counts as accepted: its sum is never read
            bool px, py;
            float2 nre, nim;
            if constexpr (Running) {
                nre = fma2(st.re[k], ed[k], neg2(mul2(st.im[k], en[k])));
                nim = fma2(st.re[k], en[k], mul2(st.im[k], ed[k]));
                px = !(ed[k].x <= kMinD) && !(nre.x <= 0.f);
                py = !(ed[k].y <= kMinD) && !(nre.y <= 0.f);
            } else {
                const float2 v = fma2(bc2(kTanGroup), ed[k], neg2(make_float2(fabsf(en[k].x), fabsf(en[k].y))));
                px = !(v.x <= kAccept);
                py = !(v.y <= kAccept);
            }
            if constexpr (C) {   // and the term must not be ill-conditioned (cancels(), paired)
                const float2 t = mul2(bc2(kCancel), mul2(A[k].h, B[k].h));
                const float2 m2 = fma2(en[k], en[k], mul2(ed[k], ed[k]));
                const float2 t2 = mul2(t, t);
                px = px && !(m2.x < t2.x);
                py = py && !(m2.y < t2.y);
            }
            if constexpr (Running) {
                st.re[k] = make_float2(px ? nre.x : st.re[k].x, py ? nre.y : st.re[k].y);
                st.im[k] = make_float2(px ? nim.x : st.im[k].x, py ? nim.y : st.im[k].y);
            } else {
                const float2 fd = make_float2(px ? ed[k].x : 1.f, py ? ed[k].y : 1.f);
                const float2 fn = make_float2(px ? en[k].x : 0.f, py ? en[k].y : 0.f);
                nre = fma2(st.re[k], fd, neg2(mul2(st.im[k], fn)));
                nim = fma2(st.re[k], fn, mul2(st.im[k], fd));
                st.re[k] = nre;
                st.im[k] = nim;
            }
            fail |= (px ? 0u : 1u << (2 * k)) | (py ? 0u : 2u << (2 * k));
        }
        if constexpr (Defer) {
            // every lane of the warp is here (the loop and the edge flags are block-uniform)
            if (__any_sync(0xffffffffu, fail)) {
                const unsigned lane = threadIdx.x & 31u, below = (1u << lane) - 1u;
#pragma unroll
                for (int k = 0; k < KQ; ++k) {
                    const bool mine = fail >> k & 1u;
                    const unsigned b = __ballot_sync(0xffffffffu, mine);
                    if (mine) dq.queue[q_count + __popc(b & below)] = (unsigned)j << 7 | (unsigned)k << 5 | lane;
                    q_count += __popc(b);
                }
                if (q_count >= 32 * KQ) {
                    __syncwarp();
                    bsum_drain<Cond>(dq.queue, q_count, s_pts, dq.q, dq.fix, cq, counters);
                    q_count = 0;
                }
            }
        } else if (fail) {   // rare: the failing terms one by one
            const float4 Pa = s_pts[j], Pb = s_pts[j + 1];
#pragma unroll
            for (int k = 0; k < KQ; ++k) {
                if (!(fail >> k & 1u)) continue;
                const int kp = k >> 1;
                const bool hi = k & 1;
                const PointRel a = {hi ? A[kp].ax.y : A[kp].ax.x, hi ? A[kp].ay.y : A[kp].ay.x,
                                    hi ? A[kp].h.y : A[kp].h.x};
                const PointRel b = {hi ? B[kp].ax.y : B[kp].ax.x, hi ? B[kp].ay.y : B[kp].ay.x,
                                    hi ? B[kp].h.y : B[kp].h.x};
                const float qx = -(hi ? nqx[kp].y : nqx[kp].x), qy = -(hi ? nqy[kp].y : nqy[kp].x),
                            qz = -(hi ? nqz[kp].y : nqz[kp].x);
                const float nk = hi ? en[kp].y : en[kp].x, dk = hi ? ed[kp].y : ed[kp].x;
                // a queued ill-conditioned term is added after the tile, in FP64.  Only
                // the loop for warps near the tile tests: no query outside the
                // tile's widened box has such a term, so a query's terms do not
                // depend on its warp
                float t = 0.f;
                if (!(C && cancels(nk, dk, a.h, b.h) && cancel_enqueue(cq, j, k, (int)(threadIdx.x & 31))))
                    t = fallback_term(nk, dk, a, b, Pa, Pb, qx, qy, qz, counters);
                if (hi) two_sum_acc(st.part[kp].y, st.comp[kp].y, t);
                else two_sum_acc(st.part[kp].x, st.comp[kp].x, t);
            }
        }
        if (++g_count == GROUP) finalize();
    };

    auto run_edges = [&](auto cond, int cnt) {
        PointRel2 ra[KP], rb[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) ra[k] = point_rel2(s_pts[0], nqx[k], nqy[k], nqz[k]);
        for (int j = 0; j < cnt; j += 2) {
            const float4 P0 = s_pts[j], P1 = s_pts[j + 1];
#pragma unroll
            for (int k = 0; k < KP; ++k) rb[k] = point_rel2(P1, nqx[k], nqy[k], nqz[k]);
            if (P0.w != 0.f) add_edge(cond, ra, rb, j);
            if (j + 1 < cnt) {
                const float4 P2 = s_pts[j + 2];
#pragma unroll
                for (int k = 0; k < KP; ++k) ra[k] = point_rel2(P2, nqx[k], nqy[k], nqz[k]);
                if (P1.w != 0.f) add_edge(cond, rb, ra, j + 1);
            }
        }
    };

    for (int64_t t0 = e_begin; t0 < e_end; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, e_end - t0);   // edge start points in this tile
        __syncthreads();
        for (int i = threadIdx.x; i <= cnt; i += blockDim.x) s_pts[i] = __ldg(pts + t0 + i);
        __syncthreads();
        bool near = false;
        if constexpr (Cond) {
            // A term can be ill-conditioned only if its edge subtends nearly pi at
            // the query, which needs the query within a small fraction of the
            // edge's length of the edge.  The tile's widened box (tile_box) holds
            // every such query; for a warp with no query in it no term is
            // ill-conditioned, so the loop without the test takes the same
            // decisions (bit-identical results).
            float box[6];
            tile_box(s_pts, cnt, box);
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                near |= in_box(box, -nqx[k].x, -nqy[k].x, -nqz[k].x) || in_box(box, -nqx[k].y, -nqy[k].y, -nqz[k].y);
            }
            near = __any_sync(0xffffffffu, near);
        }
        if (near) run_edges(std::true_type{}, cnt);
        else run_edges(std::false_type{}, cnt);
        if (g_count > 0) finalize();
        if constexpr (Defer) {
            if (q_count > 0) {   // the entries index this tile's points
                __syncwarp();
                bsum_drain<Cond>(dq.queue, q_count, s_pts, dq.q, dq.fix, cq, counters);
                q_count = 0;
            }
        }
        if constexpr (Cond) {   // the queued cancelling terms of this tile, in FP64
            __syncwarp();
            if (*cq.count > 0) cancel_drain(cq, s_pts, counters);
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            s_acc[(2 * k) * blockDim.x + threadIdx.x] += (double)st.part[k].x + (double)st.comp[k].x;
            s_acc[(2 * k + 1) * blockDim.x + threadIdx.x] += (double)st.part[k].y + (double)st.comp[k].y;
            st.part[k] = bc2(0.f);
            st.comp[k] = bc2(0.f);
        }
    }
    if constexpr (Defer || Cond) {   // the warp's own drains wrote these sums
        __syncwarp();
#pragma unroll
        for (int k = 0; k < KQ; ++k)
            s_acc[k * blockDim.x + threadIdx.x] += (double)cq.fix[k * blockDim.x + threadIdx.x] * kFixUnit;
    }
}

// One thread holds 2*KP queries as KP float2 pairs (strided by the block size).
// Blocks of 128 threads, 4 resident per SM (at most 128 registers): the same 16 warps
// per SM as 2 blocks of 256, but with finer-grained scheduling, measured 2%
// faster on 2M queries x 154k edges.
// Block (x, y) covers queries of tile x and the edges starting in point chunk y;
// with more than one chunk it writes FP64 partial sums [chunk][query] that
// k_boundary_combine adds, otherwise it combines with chi itself.
constexpr int kBsumThreads = 128;

template <int KP, bool Cond = false, bool Running = false>
__global__ void __launch_bounds__(kBsumThreads, 4) k_boundary_sum(const float *__restrict__ q, int64_t n,
                                                      const float4 *__restrict__ pts, int64_t npts, int tile,
                                                      int64_t chunk_len, double *__restrict__ partial,
                                                      const int32_t *__restrict__ chi, float *__restrict__ w,
                                                      uint8_t *__restrict__ label, int classify, float margin,
                                                      int32_t *__restrict__ list,
                                                      unsigned long long *__restrict__ list_len,
                                                      unsigned *__restrict__ listed,
                                                      unsigned long long *__restrict__ counters) {
    // dynamic shared memory (bsum_smem): tile + 1 points | 2 KP x blockDim FP64 sums |
    // (Cond) 2 KP x blockDim fixed-point sums, per warp kCancelCap queue entries, per warp
    // a count
    extern __shared__ float4 s_pts[];
    double *s_acc = reinterpret_cast<double *>(s_pts + tile + 1);
    constexpr int KQ = 2 * KP;
    const int64_t qblock = (int64_t)blockIdx.x * blockDim.x * KQ;
    const int64_t base = qblock + threadIdx.x;
    const int64_t e_begin = (int64_t)blockIdx.y * chunk_len;
    const int64_t e_end = min(npts - 1, e_begin + chunk_len);   // edge start points
    CancelQ cq{};
    if constexpr (Cond) {
        const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        cq.fix = reinterpret_cast<long long *>(s_acc + KQ * blockDim.x);
        unsigned *queues = reinterpret_cast<unsigned *>(cq.fix + KQ * blockDim.x);
        cq.queue = queues + warp * kCancelCap;
        cq.count = reinterpret_cast<int *>(queues + nwarps * kCancelCap) + warp;
        cq.q = q + 3 * qblock;
        cq.qbase = qblock;
        cq.list = list;
        cq.list_len = list_len;
        cq.listed = listed;
    }
    float2 nqx[KP], nqy[KP], nqz[KP];
    load_query_pairs<KP>(q, base, n, nqx, nqy, nqz);
#pragma unroll
    for (int k = 0; k < KQ; ++k) s_acc[k * blockDim.x + threadIdx.x] = 0.0;
    bsum_accumulate<KP, false, Cond, Running>(pts, e_begin, e_end, tile, s_pts, nqx, nqy, nqz, s_acc, counters, cq);
    double acc[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) acc[k] = s_acc[k * blockDim.x + threadIdx.x];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        if (idx >= n) continue;
        if (partial) {
            partial[(int64_t)blockIdx.y * n + idx] = acc[k];
            continue;
        }
        const double wv = (double)chi[idx] + acc[k] * kInv2Pi;
        w[idx] = (float)wv;
        if (classify) {
            label[idx] = wv > 0.5 ? 1 : 0;
            if (fabs(wv - 0.5) <= (double)margin) list_query(idx, list, list_len, listed);
        }
    }
}

// Bytes of k_boundary_sum's dynamic shared memory.
static size_t bsum_smem(int kp, int tile, bool cond) {
    const size_t kq = 2 * (size_t)kp, threads = kBsumThreads;
    size_t b = sizeof(float4) * (tile + 1) + sizeof(double) * kq * threads;
    if (cond) b += sizeof(long long) * kq * threads + (sizeof(unsigned) * kCancelCap + sizeof(int)) * (threads / 32);
    return b;
}

// Persistent kernel over the work queue of a batch of meshes.  Each block
// repeatedly takes the next item (items are sorted by estimated cost, largest
// first): a crossing item computes chi for its tile's queries; a boundary item
// adds the tile's boundary terms of one point chunk into the FP64 accumulators
// (atomically, so the FP64 summation order of chunks is not fixed).  The block
// that completes a tile's last item combines w = chi + acc / 2pi for that tile
// (the writers fence before counting), so no grid-wide barrier is needed.
template <int KP>
__global__ void __launch_bounds__(256, 2) k_batch(const BatchMesh *__restrict__ meshes,
                                               const BatchTile *__restrict__ tiles,
                                               const BatchItem *__restrict__ items, int64_t n_items,
                                               const float *__restrict__ q, int32_t *chi, double *acc,
                                               float *__restrict__ w, unsigned *tile_done,
                                               unsigned long long *head, int tile_pts, int32_t *list,
                                               unsigned long long *list_len, unsigned *listed) {
    extern __shared__ float4 s_pts[];
    __shared__ long long s_item;
    __shared__ int s_last;
    constexpr int KQ = 2 * KP;
    while (true) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(head, 1ull);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem wi = items[it];
        const BatchTile tl = tiles[wi.tile];
        const BatchMesh mh = meshes[tl.mesh];
        if (wi.kind == 0) {
            // the crossing numbers of the tile: in exact mode the warp walks
            // together (bvh_walk_up_warp), so every lane takes every round
            const bool fixed = qframe(mh.counters)->bits != 0;
            for (int base = 0; base < tl.q_count; base += blockDim.x) {
                const int i = base + (int)threadIdx.x;
                const bool active = i < tl.q_count;
                const int64_t g = tl.q_begin + (active ? i : 0);
                const float3 p = active ? make_float3(q[3 * g], q[3 * g + 1], q[3 * g + 2]) : make_float3(0.f, 0.f, 0.f);
                int c = 0;
                if (fixed) {
                    if (active) c = chi_one(p, mh.nodes, mh.nnodes, mh.tri, mh.counters);
                } else {
                    const bool ok = bvh_walk_up_warp(active, p, mh.nodes, mh.nnodes, mh.tri, mh.counters,
                                                     [&](int, float3 a, float3 b, float3 cc) {
                                                         c += tri_crossing(p, a, b, cc, &mh.counters[CNT_EXACT_EDGE],
                                                                           &mh.counters[CNT_EXACT_PLANE]);
                                                     });
                    if (!ok) c = INT32_MIN;
                }
                if (active) chi[g] = c;
            }
        } else {
            float2 nqx[KP], nqy[KP], nqz[KP];
            double *s_acc = reinterpret_cast<double *>(s_pts + tile_pts + 1);
            const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
            BsumDefer dq;
            dq.q = q + 3 * tl.q_begin;
            dq.fix = reinterpret_cast<long long *>(s_acc + KQ * blockDim.x);
            unsigned *queues = reinterpret_cast<unsigned *>(dq.fix + KQ * blockDim.x);
            dq.queue = queues + warp * (64 * KQ);
            CancelQ cq;
            cq.fix = dq.fix;
            cq.queue = queues + nwarps * (64 * KQ) + warp * kCancelCap;
            cq.count = reinterpret_cast<int *>(queues + nwarps * (64 * KQ + kCancelCap)) + warp;
            cq.q = dq.q;
            cq.qbase = tl.q_begin;
            cq.list = list;
            cq.list_len = list_len;
            cq.listed = listed;
            load_query_pairs<KP>(dq.q, threadIdx.x, tl.q_count, nqx, nqy, nqz);
#pragma unroll
            for (int k = 0; k < KQ; ++k) s_acc[k * blockDim.x + threadIdx.x] = 0.0;
            bsum_accumulate<KP, true, true, true>(mh.pts, wi.p_begin, wi.p_end, tile_pts, s_pts, nqx, nqy, nqz, s_acc,
                                            mh.counters, cq, dq);
#pragma unroll
            for (int k = 0; k < KQ; ++k) {
                const int local = threadIdx.x + k * blockDim.x;
                if (local < tl.q_count) atomicAdd(&acc[tl.q_begin + local], s_acc[k * blockDim.x + threadIdx.x]);
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(&tile_done[wi.tile], 1u) == (unsigned)(tl.n_items - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int i = threadIdx.x; i < tl.q_count; i += blockDim.x) {
                const int64_t g = tl.q_begin + i;
                w[g] = (float)((double)__ldcg(chi + g) + __ldcg(acc + g) * kInv2Pi);
            }
        }
    }
}

// w = chi + (sum over chunks, in chunk order) / 2pi, then the labels
__global__ void k_boundary_combine(const double *__restrict__ partial, int64_t n, int chunks,
                                   const int32_t *__restrict__ chi, float *__restrict__ w,
                                   uint8_t *__restrict__ label, int classify, float margin,
                                   int32_t *__restrict__ list, unsigned long long *__restrict__ list_len,
                                   unsigned *__restrict__ listed) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partial[(int64_t)c * n + idx];
    const double wv = (double)chi[idx] + s * kInv2Pi;
    w[idx] = (float)wv;
    if (classify) {
        label[idx] = wv > 0.5 ? 1 : 0;
        if (fabs(wv - 0.5) <= (double)margin) list_query(idx, list, list_len, listed);
    }
}

// --------------------------------------------------- FP64 re-evaluation ----

__device__ double apex_angle64(double rx, double ry, bool &degenerate) {
    if (ry != 0.0) return atan2(ry, -rx);
    if (rx > 0.0) return -3.14159265358979323846;
    if (rx < 0.0) return 0.0;
    degenerate = true;
    return 0.0;
}

__device__ double edge_angle64(float4 Pa, float4 Pb, float qx, float qy, float qz,
                               const unsigned long long *counters) {
    const double ax = (double)Pa.x - qx, ay = (double)Pa.y - qy, az = (double)Pa.z - qz;
    const double bx = (double)Pb.x - qx, by = (double)Pb.y - qy, bz = (double)Pb.z - qz;
    const double sa = ax * ax + ay * ay, sb = bx * bx + by * by;
    const double la = sqrt(sa + az * az), lb = sqrt(sb + bz * bz);
    const double ha = az > 0.0 ? sa / (la + az) : la - az;
    const double hb = bz > 0.0 ? sb / (lb + bz) : lb - bz;
    const double n = ay * bx - ax * by;
    const double d = ha * hb + ax * bx + ay * by;
    if (n == 0.0 && d == 0.0) {
        bool deg = false;
        if (ax == 0.0 && ay == 0.0 && ha == 0.0 && !(bx == 0.0 && by == 0.0)) return apex_angle64(bx, by, deg);
        if (bx == 0.0 && by == 0.0 && hb == 0.0 && !(ax == 0.0 && ay == 0.0)) return -apex_angle64(ax, ay, deg);
        return 0.0;
    }
    if (d < 0.0) {
        const int s = branch_sos(qx, qy, Pa.x, Pa.y, Pb.x, Pb.y, counters);
        return atan2(s > 0 ? -fabs(n) : fabs(n), d);
    }
    return atan2(n, d);
}


// FP64 boundary sum of one query over the edges that start at points
// [j0, j1) of a chained point stream, for the re-evaluation kernels.  FP64 runs
// at 1/64 of the FP32 rate here, so the terms are grouped like the FP32 path:
// each point's unnormalised relative vector (l, and h = l - z without
// cancellation) is formed once and shared by its two edges, and a term with
// 0 < |n| / d < 0.41 (angle below pi/8) is multiplied into a complex product,
// one atan2 per 8 edges.  1e-30 < d < 1e30 keeps a product of 8 such factors
// inside the FP64 range whatever the coordinates' scale.  Every other term
// (steep, on the branch cut, degenerate) is edge_angle64's, exactly as before.
__device__ double bsum64_range(const float4 *__restrict__ pts, int64_t j0, int64_t j1, float qx, float qy, float qz,
                               const unsigned long long *counters) {
    if (j0 >= j1) return 0.0;
    double acc = 0.0, re = 1.0, im = 0.0;
    int g = 0;
    float4 P = pts[j0];
    double ax = (double)P.x - qx, ay = (double)P.y - qy, az = (double)P.z - qz;
    double sa = ax * ax + ay * ay;
    double la = sqrt(sa + az * az);
    double ha = az > 0.0 ? sa / (la + az) : la - az;
    for (int64_t j = j0; j < j1; ++j) {
        const float4 Q = pts[j + 1];
        const double bx = (double)Q.x - qx, by = (double)Q.y - qy, bz = (double)Q.z - qz;
        const double sb = bx * bx + by * by, lb = sqrt(sb + bz * bz);
        const double hb = bz > 0.0 ? sb / (lb + bz) : lb - bz;
        if (P.w != 0.f) {
            const double n = ay * bx - ax * by, d = ha * hb + ax * bx + ay * by;
            if (d > 1e-30 && d < 1e30 && fabs(n) < 0.41 * d) {
                const double r = re * d - im * n;
                im = re * n + im * d;
                re = r;
            } else {
                acc += edge_angle64(P, Q, qx, qy, qz, counters);
            }
            if (++g == GROUP) {
                acc += atan2(im, re);
                re = 1.0;
                im = 0.0;
                g = 0;
            }
        }
        P = Q;
        ax = bx;
        ay = by;
        az = bz;
        ha = hb;
    }
    if (g > 0) acc += atan2(im, re);
    return acc;
}

// One block per listed query (grid-stride over the list): FP64 boundary sum,
// fixed-order block reduction, then w and the label are rewritten.
__global__ void __launch_bounds__(256) k_fp64_fix(const float *__restrict__ q, const float4 *__restrict__ pts,
                                                  int64_t npts, const int32_t *__restrict__ chi,
                                                  float *__restrict__ w, uint8_t *__restrict__ label,
                                                  const int32_t *__restrict__ list,
                                                  const unsigned long long *__restrict__ list_len,
                                                  unsigned long long *__restrict__ counters) {
    __shared__ double red[256];
    const unsigned long long len = *list_len;
    for (unsigned long long li = blockIdx.x; li < len; li += gridDim.x) {
        const int32_t idx = list[li];
        const float qx = q[3 * idx], qy = q[3 * idx + 1], qz = q[3 * idx + 2];
        // thread t: the edges starting at points [t c, (t + 1) c), c = ceil((npts - 1) / blockDim)
        const int64_t nstart = npts > 0 ? npts - 1 : 0, per = (nstart + blockDim.x - 1) / blockDim.x;
        const int64_t j0 = min((int64_t)threadIdx.x * per, nstart), j1 = min(j0 + per, nstart);
        red[threadIdx.x] = bsum64_range(pts, j0, j1, qx, qy, qz, counters);
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double wv = (double)chi[idx] + red[0] * kInv2Pi;
            w[idx] = (float)wv;
            if (label) label[idx] = wv > 0.5 ? 1 : 0;
            atomicAdd(&counters[CNT_FP64], 1ull);
        }
        __syncthreads();
    }
}

// The batched launch's FP64 re-evaluation: one block per listed query (its
// cancelling terms overflowed the kernel's queue); the mesh is found by binary
// search in the meshes' query offsets.
__global__ void __launch_bounds__(256) k_batch_fp64_fix(const BatchMesh *__restrict__ meshes,
                                                        const int64_t *__restrict__ mesh_off, int n_mesh,
                                                        const float *__restrict__ q, const int32_t *__restrict__ chi,
                                                        float *__restrict__ w, const int32_t *__restrict__ list,
                                                        const unsigned long long *__restrict__ list_len) {
    __shared__ double red[256];
    const unsigned long long len = *list_len;
    for (unsigned long long li = blockIdx.x; li < len; li += gridDim.x) {
        const int64_t g = list[li];
        int lo = 0, hi = n_mesh - 1;   // the mesh with mesh_off[mi] <= g < mesh_off[mi + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (mesh_off[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const BatchMesh mh = meshes[lo];
        const float qx = q[3 * g], qy = q[3 * g + 1], qz = q[3 * g + 2];
        const int64_t nstart = mh.npts > 0 ? mh.npts - 1 : 0, per = (nstart + blockDim.x - 1) / blockDim.x;
        const int64_t j0 = min((int64_t)threadIdx.x * per, nstart), j1 = min(j0 + per, nstart);
        red[threadIdx.x] = bsum64_range(mh.pts, j0, j1, qx, qy, qz, mh.counters);
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            w[g] = (float)((double)chi[g] + red[0] * kInv2Pi);
            atomicAdd(&mh.counters[CNT_FP64], 1ull);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- direct ----

// Direct sum (Eq. 2, each area by Eq. 6): per triangle 2 atan2(det[a b c], l_a l_b l_c + (a.b) l_c
// + (a.c) l_b + (b.c) l_a) with a, b, c the vertices relative to q (the
// unnormalised van Oosterom-Strackee form).  Triangles are staged through shared
// memory (9 floats each); each thread holds 2*KP queries as float2 pairs.  The
// triangle range is split into gridDim.y chunks so that any query count fills
// the GPU: with one chunk the kernel writes w, otherwise FP64 partial sums
// [chunk][query] that k_direct_reduce adds in chunk order.
template <int KP>
__global__ void __launch_bounds__(256) k_direct(const float *__restrict__ q, int64_t n, const float *__restrict__ tri9,
                                                int64_t nt, int tile, int64_t chunk_len, float *__restrict__ w,
                                                double *__restrict__ partial) {
    extern __shared__ float s_tri[];
    constexpr int KQ = 2 * KP;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * KQ + threadIdx.x;
    const int64_t t_begin = (int64_t)blockIdx.y * chunk_len;
    const int64_t t_end = min(nt, t_begin + chunk_len);
    float2 nqx[KP], nqy[KP], nqz[KP], part[KP];
    double acc[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        const bool ok = idx < n;
        const float x = ok ? -q[3 * idx] : 0.f, y = ok ? -q[3 * idx + 1] : 0.f, z = ok ? -q[3 * idx + 2] : 0.f;
        if (k & 1) { nqx[k >> 1].y = x; nqy[k >> 1].y = y; nqz[k >> 1].y = z; }
        else       { nqx[k >> 1].x = x; nqy[k >> 1].x = y; nqz[k >> 1].x = z; }
        acc[k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) part[k] = bc2(0.f);
    for (int64_t t0 = t_begin; t0 < t_end; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, t_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < 9 * cnt; i += blockDim.x) s_tri[i] = __ldg(tri9 + 9 * t0 + i);
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float *T = s_tri + 9 * j;
            const float2 X0 = bc2(T[0]), Y0 = bc2(T[1]), Z0 = bc2(T[2]);
            const float2 X1 = bc2(T[3]), Y1 = bc2(T[4]), Z1 = bc2(T[5]);
            const float2 X2 = bc2(T[6]), Y2 = bc2(T[7]), Z2 = bc2(T[8]);
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const float2 ax = add2(X0, nqx[k]), ay = add2(Y0, nqy[k]), az = add2(Z0, nqz[k]);
                const float2 bx = add2(X1, nqx[k]), by = add2(Y1, nqy[k]), bz = add2(Z1, nqz[k]);
                const float2 cx = add2(X2, nqx[k]), cy = add2(Y2, nqy[k]), cz = add2(Z2, nqz[k]);
                const float2 la2 = fma2(ax, ax, fma2(ay, ay, mul2(az, az)));
                const float2 lb2 = fma2(bx, bx, fma2(by, by, mul2(bz, bz)));
                const float2 lc2 = fma2(cx, cx, fma2(cy, cy, mul2(cz, cz)));
                const float2 la = mul2(la2, make_float2(sfu_rsqrt(fmaxf(la2.x, 1e-37f)), sfu_rsqrt(fmaxf(la2.y, 1e-37f))));
                const float2 lb = mul2(lb2, make_float2(sfu_rsqrt(fmaxf(lb2.x, 1e-37f)), sfu_rsqrt(fmaxf(lb2.y, 1e-37f))));
                const float2 lc = mul2(lc2, make_float2(sfu_rsqrt(fmaxf(lc2.x, 1e-37f)), sfu_rsqrt(fmaxf(lc2.y, 1e-37f))));
                const float2 cxx = fma2(by, cz, neg2(mul2(bz, cy)));
                const float2 cyy = fma2(bz, cx, neg2(mul2(bx, cz)));
                const float2 czz = fma2(bx, cy, neg2(mul2(by, cx)));
                const float2 det = fma2(ax, cxx, fma2(ay, cyy, mul2(az, czz)));
                const float2 ab = fma2(ax, bx, fma2(ay, by, mul2(az, bz)));
                const float2 ac = fma2(ax, cx, fma2(ay, cy, mul2(az, cz)));
                const float2 bc = fma2(bx, cx, fma2(by, cy, mul2(bz, cz)));
                const float2 den = fma2(ab, lc, fma2(ac, lb, fma2(bc, la, mul2(mul2(la, lb), lc))));
                part[k] = add2(part[k], fast_atan2_2(det, den));
            }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            acc[2 * k] += (double)part[k].x;
            acc[2 * k + 1] += (double)part[k].y;
            part[k] = bc2(0.f);
        }
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        if (idx >= n) continue;
        if (partial) partial[(int64_t)blockIdx.y * n + idx] = acc[k];
        else w[idx] = (float)(acc[k] * kInv2Pi);
    }
}

__global__ void k_direct_reduce(const double *__restrict__ partial, int64_t n, int chunks, float *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partial[(int64_t)c * n + i];
    w[i] = (float)(s * kInv2Pi);
}

}  // namespace

gwn_status launch_chi(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi, cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    ProfScope prof("chi_traversal", s);
    if (m->cfg.quantize_bits)
        k_chi<true><<<grid_for(n, kChiThreads), kChiThreads, 0, s>>>(q, n, m->nodes, m->nnodes, m->leaf_tri, chi,
                                                                        m->counters);
    else
        k_chi<false><<<grid_for(n, kChiThreads), kChiThreads, 0, s>>>(q, n, m->nodes, m->nnodes, m->leaf_tri, chi,
                                                                        m->counters);
    GWN_LAUNCH_CHECK("k_chi");
    return GWN_OK;
}

gwn_status launch_chi_visits(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi,
                             unsigned long long *visits, cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    k_chi_visits<<<grid_for(n, 256), 256, 0, s>>>(q, n, m->nodes, m->nnodes, m->leaf_tri, chi, m->counters, visits);
    GWN_LAUNCH_CHECK("k_chi_visits");
    return GWN_OK;
}

template <int KP, bool Cond = false, bool Running = false>
static gwn_status launch_bsum_kp(const gwn_mesh *m, const float *q, int64_t n, const int32_t *chi, float *w,
                                 uint8_t *label, bool classify, int32_t *list, unsigned long long *list_len,
                                 unsigned *listed, double *partial_buf, int64_t partial_cap, cudaStream_t s) {
    const int tile = m->cfg.boundary_tile > 0 ? m->cfg.boundary_tile : 512;
    const size_t smem = bsum_smem(KP, tile, Cond);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_boundary_sum<KP, Cond, Running>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    const float margin = m->cfg.classify_margin > 0.f ? m->cfg.classify_margin : 1e-4f;
    const int64_t per_block = kBsumThreads * 2 * KP;
    const int64_t qblocks = (n + per_block - 1) / per_block;
    const int64_t nedge_pts = m->npts > 0 ? m->npts - 1 : 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // split the boundary into chunks when the query tiles alone cannot fill the GPU
    int64_t chunks = (8 * (int64_t)(sms > 0 ? sms : 148) + qblocks - 1) / qblocks;
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (nedge_pts + 2 * tile - 1) / (2 * tile)));
    if (partial_cap >= 0) chunks = std::min<int64_t>(chunks, partial_cap / n);   // caller-provided room
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, 65535));
    const int64_t chunk_len = chunks > 1 ? (nedge_pts + chunks - 1) / chunks : std::max<int64_t>(nedge_pts, 1);
    double *partial = nullptr;
    bool own = false;
    if (chunks > 1) {
        if (partial_cap >= 0) {
            partial = partial_buf;
        } else {
            GWN_CUDA_TRY(cudaMallocAsync(&partial, sizeof(double) * chunks * n, s));
            own = true;
        }
    }
    dim3 grid((unsigned)qblocks, (unsigned)chunks);
    k_boundary_sum<KP, Cond, Running><<<grid, kBsumThreads, smem, s>>>(q, n, m->bpts, m->npts, tile, chunk_len,
                                                                      partial, chi, w, label, classify ? 1 : 0,
                                                                      margin, list, list_len, listed, m->counters);
    note_launches(1);
    if (partial) {
        k_boundary_combine<<<grid_for(n, 256), 256, 0, s>>>(partial, n, (int)chunks, chi, w, label,
                                                            classify ? 1 : 0, margin, list, list_len, listed);
        note_launches(1);
        if (own) cudaFreeAsync(partial, s);
    }
    GWN_LAUNCH_CHECK("k_boundary_sum");
    return GWN_OK;
}

// The group acceptance test of a mesh (gwn_config.group_test): the running
// test where the boundary is dense, at least one boundary edge per two
// triangles (random soups, 3 per triangle), else the per-term test.
static bool group_test_running(const gwn_mesh *m) {
    if (m->cfg.group_test == 1) return false;
    if (m->cfg.group_test == 2) return true;
    return 2 * m->nb >= m->nt && m->nb > 0;
}

// The boundary sum with the scratch it needs provided: list (n entries), a
// zeroed list_len and zeroed listed bits (n / 32 words, rounded up); the chunk
// partials in partial_buf (room for partial_cap doubles), or allocated as
// needed when partial_cap < 0.
static gwn_status boundary_sum_on(const gwn_mesh *m, const float *q, int64_t n, const int32_t *chi, float *w,
                                  uint8_t *label, bool classify, int32_t *list, unsigned long long *list_len,
                                  unsigned *listed, double *partial_buf, int64_t partial_cap, cudaStream_t s) {
    const int kq = m->cfg.queries_per_thread > 0 ? m->cfg.queries_per_thread : 4;
    ProfScope prof("boundary_sum", s);
    const bool running = group_test_running(m);
#define GWN_BSUM(KP, C, R) \
    launch_bsum_kp<KP, C, R>(m, q, n, chi, w, label, classify, list, list_len, listed, partial_buf, partial_cap, s)
    if (m->cfg.fp64_cancel >= 0) {   // the default: cancelling terms in FP64
        const bool small = kq == 1 || kq == 2;   // 8 queries per thread: the queue holds 2-bit slots
        if (running) return small ? GWN_BSUM(1, true, true) : GWN_BSUM(2, true, true);
        return small ? GWN_BSUM(1, true, false) : GWN_BSUM(2, true, false);
    }
    switch (kq) {
        case 1:
        case 2: return running ? GWN_BSUM(1, false, true) : GWN_BSUM(1, false, false);
        case 8: return GWN_BSUM(4, false, false);
        default: return running ? GWN_BSUM(2, false, true) : GWN_BSUM(2, false, false);
    }
#undef GWN_BSUM
}

gwn_status launch_boundary_sum_list(const gwn_mesh *m, const float *q, int64_t n, const int32_t *chi, float *w,
                                    uint8_t *label, bool classify, int32_t *list, unsigned long long *list_len,
                                    cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    const size_t words = (size_t)((n + 31) / 32);
    unsigned *listed = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&listed, sizeof(unsigned) * words, s));
    GWN_CUDA_TRY(cudaMemsetAsync(listed, 0, sizeof(unsigned) * words, s));
    // without a caller list (no labels wanted), queries whose cancelling terms
    // overflow the kernel's queue still need their FP64 re-evaluation
    const bool own_list = list == nullptr;
    if (own_list) {
        GWN_CUDA_TRY(cudaMallocAsync(&list, sizeof(int32_t) * n, s));
        GWN_CUDA_TRY(cudaMallocAsync(&list_len, sizeof(unsigned long long), s));
        GWN_CUDA_TRY(cudaMemsetAsync(list_len, 0, sizeof(unsigned long long), s));
    }
    gwn_status st = boundary_sum_on(m, q, n, chi, w, label, classify, list, list_len, listed, nullptr, -1, s);
    if (st == GWN_OK && own_list) st = launch_fp64_fix_list(m, q, chi, w, nullptr, list, list_len, s);
    cudaFreeAsync(listed, s);
    if (own_list) {
        cudaFreeAsync(list, s);
        cudaFreeAsync(list_len, s);
    }
    return st;
}

// The classify sequence on caller-provided scratch (allocates nothing): chi_tmp
// [n] int32, list [n] int32, list_len one zeroed counter, listed (n + 31) / 32
// zeroed words, partial room for partial_cap doubles (the boundary sum is split
// into at most partial_cap / n point chunks; fewer than two means no split).
gwn_status launch_classify_on_scratch(const gwn_mesh *m, const float *q, int64_t n, uint8_t *label, float *w,
                                      int32_t *chi_tmp, int32_t *list, unsigned long long *list_len,
                                      unsigned *listed, double *partial, int64_t partial_cap, cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    if (m->cfg.quantize_bits)
        k_chi<true><<<grid_for(n, kChiThreads), kChiThreads, 0, s>>>(q, n, m->nodes, m->nnodes, m->leaf_tri, chi_tmp,
                                                                        m->counters);
    else
        k_chi<false><<<grid_for(n, kChiThreads), kChiThreads, 0, s>>>(q, n, m->nodes, m->nnodes, m->leaf_tri, chi_tmp,
                                                                        m->counters);
    GWN_LAUNCH_CHECK("k_chi");
    gwn_status st = boundary_sum_on(m, q, n, chi_tmp, w, label, true, list, list_len, listed, partial,
                                    partial ? partial_cap : 0, s);
    if (st != GWN_OK) return st;
    return launch_fp64_fix_list(m, q, chi_tmp, w, label, list, list_len, s);
}

// k_batch's dynamic shared memory: tile + 1 points, then per query slot an FP64
// sum and a fixed-point sum, then per warp one deferred-term queue of 64 KQ
// entries, then per warp a cancelling-term queue and its count.
static size_t batch_smem(int kp, int tile_pts) {
    const size_t kq = 2 * (size_t)kp, threads = 256, warps = threads / 32;
    return sizeof(float4) * (tile_pts + 1) + (sizeof(double) + sizeof(long long)) * kq * threads +
           sizeof(unsigned) * (64 * kq + kCancelCap) * warps + sizeof(int) * warps;
}

template <int KP>
static gwn_status launch_batch_kp(int grid, int tile_pts, const BatchMesh *meshes, const BatchTile *tiles,
                                  const BatchItem *items, int64_t n_items, const float *q, int32_t *chi, double *acc,
                                  float *w, unsigned *tile_done, unsigned long long *head, int32_t *list,
                                  unsigned long long *list_len, unsigned *listed, cudaStream_t s) {
    const size_t smem = batch_smem(KP, tile_pts);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_batch<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch<KP><<<grid, 256, smem, s>>>(meshes, tiles, items, n_items, q, chi, acc, w, tile_done, head, tile_pts,
                                        list, list_len, listed);
    GWN_LAUNCH_CHECK("k_batch");
    return GWN_OK;
}

gwn_status launch_batch_kernel(int kp, int grid, int tile_pts, const BatchMesh *meshes, const BatchTile *tiles,
                               const BatchItem *items, int64_t n_items, const float *q, int32_t *chi, double *acc,
                               float *w, unsigned *tile_done, unsigned long long *head, int32_t *list,
                               unsigned long long *list_len, unsigned *listed, cudaStream_t s) {
    ProfScope prof("batch", s);
    if (kp == 1)
        return launch_batch_kp<1>(grid, tile_pts, meshes, tiles, items, n_items, q, chi, acc, w, tile_done, head,
                                  list, list_len, listed, s);
    return launch_batch_kp<2>(grid, tile_pts, meshes, tiles, items, n_items, q, chi, acc, w, tile_done, head, list,
                              list_len, listed, s);
}

int batch_blocks_per_sm(int kp, int tile_pts) {
    int nb = 0;
    const size_t smem = batch_smem(kp == 1 ? 1 : 2, tile_pts);
    if (kp == 1) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<1>, 256, smem);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<2>, 256, smem);
    }
    return nb > 0 ? nb : 1;
}

gwn_status launch_batch_fp64_fix(const BatchMesh *meshes, const int64_t *mesh_off, int n_mesh, const float *q,
                                 const int32_t *chi, float *w, const int32_t *list,
                                 const unsigned long long *list_len, cudaStream_t s) {
    if (n_mesh <= 0) return GWN_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_batch_fp64_fix<<<(unsigned)(sms > 0 ? 2 * sms : 128), 256, 0, s>>>(meshes, mesh_off, n_mesh, q, chi, w, list,
                                                                          list_len);
    GWN_LAUNCH_CHECK("k_batch_fp64_fix");
    return GWN_OK;
}

gwn_status launch_fp64_fix_list(const gwn_mesh *m, const float *q, const int32_t *chi, float *w, uint8_t *label,
                                const int32_t *list, const unsigned long long *list_len, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ProfScope prof("fp64_fix", s);
    k_fp64_fix<<<(unsigned)(sms > 0 ? 2 * sms : 128), 256, 0, s>>>(q, m->bpts, m->npts, chi, w, label, list,
                                                                    list_len, m->counters);
    GWN_LAUNCH_CHECK("k_fp64_fix");
    return GWN_OK;
}

gwn_status launch_direct(const gwn_mesh *m, const float *q, int64_t n, float *w, cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    if (m->nt == 0) {
        GWN_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(float) * n, s));
        return GWN_OK;
    }
    constexpr int KP = 2;
    const int tile = 256;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t qblocks = (n + 256 * 2 * KP - 1) / (256 * 2 * KP);
    // enough blocks for about four waves of two resident blocks per SM
    int64_t chunks = (8 * (int64_t)(sms > 0 ? sms : 148) + qblocks - 1) / qblocks;
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (m->nt + 4 * tile - 1) / (4 * tile)));
    chunks = std::min<int64_t>(chunks, 65535);
    const int64_t chunk_len = (m->nt + chunks - 1) / chunks;
    double *partial = nullptr;
    if (chunks > 1) GWN_CUDA_TRY(cudaMallocAsync(&partial, sizeof(double) * chunks * n, s));
    {
        ProfScope prof("direct_sum", s);
        dim3 grid((unsigned)qblocks, (unsigned)chunks);
        k_direct<KP><<<grid, 256, sizeof(float) * 9 * tile, s>>>(q, n, m->tri9, m->nt, tile, chunk_len, w, partial);
        if (partial) k_direct_reduce<<<grid_for(n, 256), 256, 0, s>>>(partial, n, (int)chunks, w);
    }
    if (partial) cudaFreeAsync(partial, s);
    GWN_LAUNCH_CHECK("k_direct");
    return GWN_OK;
}

}  // namespace gwn
