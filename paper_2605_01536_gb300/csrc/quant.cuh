// Fixed-point predicates (Supp. S2.1): the paper snaps the input to a 30-bit
// fixed-point grid and decides the perturbed predicates in integer arithmetic.
// A mesh built with gwn_config.quantize_bits = 30 does the same here:
//
//   X = rint((x - c) 2^-e)   (in FP64: (double)x - c is exact for FP32 x near
//                             the mesh, the scaling by a power of two is exact)
//
// with c the centre of the vertices' bounding box and e the smallest exponent
// that maps every vertex into [-2^29, 2^29].  Query coordinates are snapped the
// same way and clamped to [-2^62, 2^62].  The crossing test and the branch-cut
// sign of the boundary terms then take the same perturbed signs (real part,
// e1, e2, e3 coefficients) of the snapped integers: 2-D signs in 128-bit
// integers (differences below 2^63 times differences below 2^31), the 3-D
// determinant only where the query lies inside the triangle's projection and
// its z range, so that every difference is below 2^31 and every product fits.
//
// The frame lives in the mesh's device status block, right after the counter
// slots, so every kernel that receives the mesh's counters can read it.
#pragma once

#include "gwn_internal.cuh"
#include "predicates.cuh"

namespace gwn {

struct QFrame {
    int32_t bits;          // 0: predicates on the exact FP32 inputs; 30: fixed point
    float pad;             // one quantum (2^e) in FP32, padding of the float BVH boxes
    double cx, cy, cz;     // snapping centre
    double scale;          // 2^-e
    const int4 *leaf_q;    // [3 nt] snapped leaf-triangle vertices (x, y, z, 0)
};

constexpr double kQClamp = 4611686018427387904.0;   // 2^62

__host__ __device__ __forceinline__ const QFrame *qframe(const unsigned long long *counters) {
    return reinterpret_cast<const QFrame *>(counters + CNT_SLOTS);
}

__device__ __forceinline__ long long qcoord(float v, double c, double scale) {
    double t = (static_cast<double>(v) - c) * scale;
    t = fmin(fmax(t, -kQClamp), kQClamp);
    return __double2ll_rn(t);
}

__device__ __forceinline__ int sgn128(__int128 v) { return (v > 0) - (v < 0); }
__device__ __forceinline__ int sgnll(long long v) { return (v > 0) - (v < 0); }

// Perturbed 2-D classification of (x, y) against the edge i -> j (the integer
// counterpart of edge_sos): (x + e1 - x_i)(y_i - y_j) + (y + e2 - y_i)(x_j - x_i).
__device__ __forceinline__ int edge_sos_q(long long x, long long y, long long xi, long long yi, long long xj,
                                          long long yj) {
    const __int128 f = (__int128)(x - xi) * (__int128)(yi - yj) + (__int128)(y - yi) * (__int128)(xj - xi);
    int s = sgn128(f);
    if (s) return s;
    s = sgnll(yi - yj);
    if (s) return s;
    return sgnll(xj - xi);
}

// (b - a) x (c - a) components in 128-bit (coordinates below 2^30 in magnitude)
__device__ __forceinline__ __int128 orient2d_q(long long ax, long long ay, long long bx, long long by, long long cx,
                                               long long cy) {
    return (__int128)(bx - ax) * (__int128)(cy - ay) - (__int128)(by - ay) * (__int128)(cx - ax);
}

// Perturbed sign of n . (a - q_eps) for a query whose projection is inside the
// triangle (sign of n_z = s_nz): below the whole triangle the plane is above
// (sign s_nz); otherwise det[a - q, b - q, c - q], then -n_x, -n_y, -n_z.
__device__ __forceinline__ int plane_sos_q(long long qx, long long qy, long long qz, int4 a, int4 b, int4 c,
                                           int s_nz) {
    if (qz < min(a.z, min(b.z, c.z))) return s_nz;
    const __int128 ux = a.x - qx, uy = a.y - qy, uz = a.z - qz;
    const __int128 vx = b.x - qx, vy = b.y - qy, vz = b.z - qz;
    const __int128 wx = c.x - qx, wy = c.y - qy, wz = c.z - qz;
    const __int128 d = ux * (vy * wz - vz * wy) + uy * (vz * wx - vx * wz) + uz * (vx * wy - vy * wx);
    int s = sgn128(d);
    if (s) return s;
    s = sgn128(orient2d_q(a.y, a.z, b.y, b.z, c.y, c.z));   // n_x
    if (s) return -s;
    s = sgn128(orient2d_q(a.z, a.x, b.z, b.x, c.z, c.x));   // n_y
    if (s) return -s;
    return -s_nz;
}

// Signed crossing of the +z ray from the snapped query with a snapped triangle.
__device__ __forceinline__ int tri_crossing_q(long long qx, long long qy, long long qz, int4 a, int4 b, int4 c) {
    if (qz >= max(a.z, max(b.z, c.z))) return 0;
    const int s0 = edge_sos_q(qx, qy, a.x, a.y, b.x, b.y);
    const int s1 = edge_sos_q(qx, qy, b.x, b.y, c.x, c.y);
    if (s0 == 0 || s0 != s1) return 0;
    const int s2 = edge_sos_q(qx, qy, c.x, c.y, a.x, a.y);
    if (s2 != s0) return 0;
    const int side = plane_sos_q(qx, qy, qz, a, b, c, s0);
    return side == s0 ? s0 : 0;
}

// Sign of the 2-D classification of the query against the boundary edge a -> b
// that fixes the atan2 branch of a boundary term (Supp. S2.1): the same
// predicate as the crossing test, exact on the FP32 inputs or on the snapped
// integers of a fixed-point mesh, so that both discontinuities stay together.
__device__ __forceinline__ int branch_sos(float qx, float qy, float ax, float ay, float bx, float by,
                                          const unsigned long long *counters) {
    const QFrame *qf = qframe(counters);
    if (qf->bits)
        return edge_sos_q(qcoord(qx, qf->cx, qf->scale), qcoord(qy, qf->cy, qf->scale),
                          qcoord(ax, qf->cx, qf->scale), qcoord(ay, qf->cy, qf->scale),
                          qcoord(bx, qf->cx, qf->scale), qcoord(by, qf->cy, qf->scale));
    return edge_sos(qx, qy, ax, ay, bx, by, nullptr);
}

}  // namespace gwn
