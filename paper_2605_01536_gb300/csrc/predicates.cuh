// Robust predicates for the +z ray and the boundary branch cut (Supp. S2.1).
//
// The query is symbolically perturbed to q + (e1, e2, e3), e3 << e2 << e1, and
// every sign is taken in the order real part, e1 coefficient, e2 coefficient,
// e3 coefficient.  Inputs are FP32 values taken as exact reals.
//
// Precision pattern: an FP32 evaluation with a static error bound decides almost
// every call; when it cannot, the sign is computed exactly.  The exact stage
// first tries FP32 error-free transforms (Shewchuk 1997: TwoSum, FMA-based
// TwoProduct, Two-Two-Diff): when the coordinate differences are themselves
// exact in FP32 (always for inputs on a common grid, the degenerate cases that
// reach this stage) the determinant is an exact sum of a few FP32 terms.
// Otherwise it falls back to FP64 expansion arithmetic (every product of two
// FP32 values is exact in FP64; Grow-Expansion), which runs at 1/64 of the
// FP32 rate on this part.  The exact helpers are __noinline__ so their
// register and local-memory needs stay out of the hot loops that call them.
#pragma once

#include "gwn_internal.cuh"

namespace gwn {

// FP32 unit roundoff based static filter constants (u = 2^-24):
//   2-D determinant of differences:  (3 + 16u) u  <  2.0e-7   (Shewchuk's A bound)
//   3-D determinant of differences:  (7 + 56u) u  <  4.2e-7 -> 5.0e-7
constexpr float kFilter2 = 2.0e-7f;
constexpr float kFilter3 = 5.0e-7f;
constexpr float kTiny = 1e-30f;   // below this the products may have underflowed

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// Sign of the exact sum of N doubles: grow a nonoverlapping expansion term by
// term; its largest nonzero component carries the sign of the sum.
template <int N>
__device__ __forceinline__ int exact_sum_sign(const double *p) {
    double e[N];
    int m = 0;
    for (int k = 0; k < N; ++k) {
        double q = p[k];
        for (int i = 0; i < m; ++i) {
            double s, err;
            two_sum(q, e[i], s, err);
            e[i] = err;
            q = s;
        }
        e[m++] = q;
    }
    for (int i = m - 1; i >= 0; --i)
        if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
    return 0;
}

// Exact sign of (bx - ax)(cy - ay) - (by - ay)(cx - ax).  Expanded into six
// products of two FP32 values, each exact in FP64 (48-bit significands).
static __device__ __noinline__ int orient2d_exact(float ax, float ay, float bx, float by, float cx, float cy) {
    const double Ax = ax, Ay = ay, Bx = bx, By = by, Cx = cx, Cy = cy;
    double p[6];
    p[0] = __dmul_rn(Bx, Cy);
    p[1] = -__dmul_rn(Bx, Ay);
    p[2] = -__dmul_rn(Ax, Cy);
    p[3] = -__dmul_rn(By, Cx);
    p[4] = __dmul_rn(By, Ax);
    p[5] = __dmul_rn(Ay, Cx);
    return exact_sum_sign<6>(p);
}

// ---- FP32 error-free transforms (explicit rounding, no contraction)
__device__ __forceinline__ void two_sum32(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}
__device__ __forceinline__ void two_diff32(float a, float b, float &s, float &e) { two_sum32(a, -b, s, e); }
// p + e = a b exactly, provided the product neither overflows nor comes within
// 2^24 of the subnormal range (checked by the callers with prod_ok)
__device__ __forceinline__ void two_prod32(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ bool prod_ok(float p) {
    const float m = fabsf(p);
    return m <= 0x1p120f && (m >= 0x1p-96f || m == 0.f);
}

// Exact sign of (bx - ax)(cy - ay) - (by - ay)(cx - ax) in FP32, when every
// difference is exact in FP32 and no product leaves the safe range: the value
// is then (p1 + e1) - (p2 + e2) with TwoProduct pairs (each a nonoverlapping
// expansion, |e| <= ulp(p) / 2), and Shewchuk's Two-Two-Diff turns it into the
// nonoverlapping expansion x3 + x2 + x1 + x0 (x3 the most significant), whose
// sign is that of its most significant nonzero component.  A zero product
// means a zero factor, so its error term is zero as well.  Returns 2 when it
// cannot decide (the FP64 expansion then decides).
static __device__ __noinline__ int orient2d_exact32(float ax, float ay, float bx, float by, float cx, float cy) {
    float d1, d2, d3, d4, r;
    two_diff32(bx, ax, d1, r);
    bool ok = r == 0.f;
    two_diff32(cy, ay, d2, r);
    ok &= r == 0.f;
    two_diff32(by, ay, d3, r);
    ok &= r == 0.f;
    two_diff32(cx, ax, d4, r);
    ok &= r == 0.f;
    float p1, e1, p2, e2;
    two_prod32(d1, d2, p1, e1);
    two_prod32(d3, d4, p2, e2);
    ok &= prod_ok(p1) & prod_ok(p2);
    if (p1 == 0.f && d1 != 0.f && d2 != 0.f) ok = false;   // underflow to zero
    if (p2 == 0.f && d3 != 0.f && d4 != 0.f) ok = false;
    if (!ok) return 2;
    // Two-One-Diff(p1, e1, e2) = j + z0 + x0, then Two-One-Diff(j, z0, p2) = x3 + x2 + x1
    float i1, x0, j, z0, i2, x1, x3, x2;
    two_diff32(e1, e2, i1, x0);
    two_sum32(p1, i1, j, z0);
    two_diff32(z0, p2, i2, x1);
    two_sum32(j, i2, x3, x2);
    if (x3 != 0.f) return x3 > 0.f ? 1 : -1;
    if (x2 != 0.f) return x2 > 0.f ? 1 : -1;
    if (x1 != 0.f) return x1 > 0.f ? 1 : -1;
    return (x0 > 0.f) - (x0 < 0.f);
}

__device__ __forceinline__ int sgn_diff(float a, float b) { return (a > b) - (a < b); }

// Perturbed sign of the 2-D classification of q = (x, y) against the projected
// edge p_i -> p_j:  (x + e1 - x_i)(y_i - y_j) + (y + e2 - y_i)(x_j - x_i), which
// equals orient2d(p_i, p_j, q) plus the perturbation terms.  0 only when the
// edge projects to a point.
__device__ __forceinline__ int edge_sos(float x, float y, float xi, float yi, float xj, float yj,
                                        unsigned long long *cnt) {
    const float t1 = __fmul_rn(__fsub_rn(x, xi), __fsub_rn(yi, yj));
    const float t2 = __fmul_rn(__fsub_rn(y, yi), __fsub_rn(xj, xi));
    const float f = __fadd_rn(t1, t2);
    const float mag = fabsf(t1) + fabsf(t2);
    if (fabsf(f) > kFilter2 * mag && mag > kTiny) return f > 0.f ? 1 : -1;
    if (cnt) atomicAdd(cnt, 1ull);
    int s = orient2d_exact32(xi, yi, xj, yj, x, y);
    if (s == 2) s = orient2d_exact(xi, yi, xj, yj, x, y);
    if (s) return s;
    s = sgn_diff(yi, yj);
    if (s) return s;
    return sgn_diff(xj, xi);
}

__device__ __forceinline__ bool sub_exact(float a, float b, float &d) {
    d = __fsub_rn(a, b);
    // TwoSum error of a + (-b) in FP32: zero iff the difference is exact
    float bv = __fsub_rn(d, a);
    float av = __fsub_rn(d, bv);
    float err = __fadd_rn(__fsub_rn(a, av), __fsub_rn(-b, bv));
    return err == 0.0f;
}

__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e) {
    p = __dmul_rn(a, b);
    e = __fma_rn(a, b, -p);
}

// Exact sign of det[a - q, b - q, c - q].
static __device__ __noinline__ int orient3d_exact(float3 q, float3 a, float3 b, float3 c) {
    float u[3], v[3], w[3];
    bool ok = sub_exact(a.x, q.x, u[0]) & sub_exact(a.y, q.y, u[1]) & sub_exact(a.z, q.z, u[2]) &
              sub_exact(b.x, q.x, v[0]) & sub_exact(b.y, q.y, v[1]) & sub_exact(b.z, q.z, v[2]) &
              sub_exact(c.x, q.x, w[0]) & sub_exact(c.y, q.y, w[1]) & sub_exact(c.z, q.z, w[2]);
    if (ok) {
        // u . (v x w) with exact FP32 differences: 6 triple products, each an exact
        // FP64 product of two FP32 values times a third factor (TwoProduct).
        double p[12];
        int k = 0;
        for (int i = 0; i < 3; ++i) {
            int j = (i + 1) % 3, l = (i + 2) % 3;
            double P1 = __dmul_rn((double)v[j], (double)w[l]);
            double P2 = -__dmul_rn((double)v[l], (double)w[j]);
            two_prod(P1, (double)u[i], p[k], p[k + 1]);
            two_prod(P2, (double)u[i], p[k + 2], p[k + 3]);
            k += 4;
        }
        return exact_sum_sign<12>(p);
    }
    // General case: det[a-q, b-q, c-q] = det[a,b,c] - det[q,b,c] - det[a,q,c] - det[a,b,q],
    // 24 monomials x_i y_j z_k, each split exactly into two doubles.
    const float3 rows[4][3] = {{a, b, c}, {q, b, c}, {a, q, c}, {a, b, q}};
    const double sgn[4] = {1.0, -1.0, -1.0, -1.0};
    double p[48];
    int k = 0;
    for (int r = 0; r < 4; ++r) {
        const float3 A = rows[r][0], B = rows[r][1], C = rows[r][2];
        const double Ax = A.x, Ay = A.y, Az = A.z, Bx = B.x, By = B.y, Bz = B.z;
        const double Cx = C.x, Cy = C.y, Cz = C.z;
        const double m[6][3] = {{Ax, By, Cz}, {Ay, Bz, Cx}, {Az, Bx, Cy},
                                {Az, By, Cx}, {Ax, Bz, Cy}, {Ay, Bx, Cz}};
        for (int t = 0; t < 6; ++t) {
            double s = (t < 3 ? 1.0 : -1.0) * sgn[r];
            double P = __dmul_rn(m[t][0], m[t][1]);
            two_prod(s * P, m[t][2], p[k], p[k + 1]);
            k += 2;
        }
    }
    return exact_sum_sign<48>(p);
}

// det[a - q, b - q, c - q] evaluated in FP32 with every step checked to be
// exact (differences and sums by their TwoSum error, products by their FMA
// residual): the sign when all of them are, else 2 (the FP64 expansion then
// decides).  Inputs on a common grid whose coordinates span fewer than about
// 2^7 grid steps always pass.
__device__ __forceinline__ bool mul_exact32(float a, float b, float &p) {
    p = __fmul_rn(a, b);
    return __fmaf_rn(a, b, -p) == 0.f && prod_ok(p) && (p != 0.f || a == 0.f || b == 0.f);
}
__device__ __forceinline__ bool add_exact32(float a, float b, float &s) {
    float e;
    two_sum32(a, b, s, e);
    return e == 0.f;
}
static __device__ __noinline__ int orient3d_exact32(float3 q, float3 a, float3 b, float3 c) {
    float u[3], v[3], w[3];
    bool ok = sub_exact(a.x, q.x, u[0]) & sub_exact(a.y, q.y, u[1]) & sub_exact(a.z, q.z, u[2]) &
              sub_exact(b.x, q.x, v[0]) & sub_exact(b.y, q.y, v[1]) & sub_exact(b.z, q.z, v[2]) &
              sub_exact(c.x, q.x, w[0]) & sub_exact(c.y, q.y, w[1]) & sub_exact(c.z, q.z, w[2]);
    float det = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, l = (i + 2) % 3;
        float p1, p2, m, t;
        ok &= mul_exact32(v[j], w[l], p1) & mul_exact32(v[l], w[j], p2);
        ok &= add_exact32(p1, -p2, m);
        ok &= mul_exact32(u[i], m, t);
        ok &= add_exact32(det, t, det);
    }
    if (!ok) return 2;
    return (det > 0.f) - (det < 0.f);
}

// Perturbed sign of n . (a - q_eps), n = (b - a) x (c - a): the real part
// det[a-q, b-q, c-q], then the e1, e2, e3 coefficients -n_x, -n_y, -n_z.
// s_nz is the (already exact) sign of n_z.
__device__ __forceinline__ int plane_sos(float3 q, float3 a, float3 b, float3 c, int s_nz,
                                         unsigned long long *cnt) {
    const float ux = __fsub_rn(a.x, q.x), uy = __fsub_rn(a.y, q.y), uz = __fsub_rn(a.z, q.z);
    const float vx = __fsub_rn(b.x, q.x), vy = __fsub_rn(b.y, q.y), vz = __fsub_rn(b.z, q.z);
    const float wx = __fsub_rn(c.x, q.x), wy = __fsub_rn(c.y, q.y), wz = __fsub_rn(c.z, q.z);
    const float p1 = __fmul_rn(vy, wz), p2 = __fmul_rn(vz, wy);
    const float p3 = __fmul_rn(vz, wx), p4 = __fmul_rn(vx, wz);
    const float p5 = __fmul_rn(vx, wy), p6 = __fmul_rn(vy, wx);
    const float D = __fadd_rn(__fadd_rn(__fmul_rn(ux, __fsub_rn(p1, p2)), __fmul_rn(uy, __fsub_rn(p3, p4))),
                              __fmul_rn(uz, __fsub_rn(p5, p6)));
    const float perm = fabsf(ux) * (fabsf(p1) + fabsf(p2)) + fabsf(uy) * (fabsf(p3) + fabsf(p4)) +
                       fabsf(uz) * (fabsf(p5) + fabsf(p6));
    if (fabsf(D) > kFilter3 * perm && perm > kTiny) return D > 0.f ? 1 : -1;
    if (cnt) atomicAdd(cnt, 1ull);
    int s = orient3d_exact32(q, a, b, c);
    if (s == 2) s = orient3d_exact(q, a, b, c);
    if (s) return s;
    // n_x = orient2d in (y, z), n_y = orient2d in (z, x)
    s = orient2d_exact32(a.y, a.z, b.y, b.z, c.y, c.z);
    if (s == 2) s = orient2d_exact(a.y, a.z, b.y, b.z, c.y, c.z);
    if (s) return -s;
    s = orient2d_exact32(a.z, a.x, b.z, b.x, c.z, c.x);
    if (s == 2) s = orient2d_exact(a.z, a.x, b.z, b.x, c.z, c.x);
    if (s) return -s;
    return -s_nz;
}

// Signed crossing of the ray q_eps + t(0,0,1), t > 0, with triangle (a, b, c):
// the common sign of the three perturbed edge classifications (= sign of n_z)
// when the projected query is inside and the plane lies above it, else 0.
__device__ __forceinline__ int tri_crossing(float3 q, float3 a, float3 b, float3 c,
                                            unsigned long long *cnt_edge, unsigned long long *cnt_plane) {
    if (q.z >= fmaxf(a.z, fmaxf(b.z, c.z))) return 0;   // entirely at or below q_eps
    const int s0 = edge_sos(q.x, q.y, a.x, a.y, b.x, b.y, cnt_edge);
    const int s1 = edge_sos(q.x, q.y, b.x, b.y, c.x, c.y, cnt_edge);
    if (s0 == 0 || s0 != s1) return 0;
    const int s2 = edge_sos(q.x, q.y, c.x, c.y, a.x, a.y, cnt_edge);
    if (s2 != s0) return 0;
    const int side = plane_sos(q, a, b, c, s0, cnt_plane);
    return side == s0 ? s0 : 0;
}

}  // namespace gwn
