// Winding numbers of parametric surfaces (Sec. 4.4, Algorithm 2): untrimmed
// bicubic Bezier patches C[p][i][j] (i along u, j along v), oriented by
// S_u x S_v.  w = chi + sum over the boundary curves of the integral of
// f(phi, t) = (w(t) - d eta(t)) / 4pi, with x0 = +z, x1 = -z.
//
// chi: signed crossings of the ray q + s x0 with the surface (Sec. 4.4.1).
//   Each patch is subdivided into dyadic sub-patches (de Casteljau on the
//   parameter rectangle, FP32 nets relative to the patch's centre) while the
//   net's xy box contains q and the net rises above q, both tested with a
//   margin that covers the nets' rounding; down to the depth at which, by the
//   patch's second differences, every sub-patch lies within the flatness
//   tolerance of the bilinear patch through its corners.  The corners are
//   evaluated in FP64 in a fixed order (a corner shared by two sub-patches is
//   the same point), and the +z ray meets the bilinear patch in closed form
//   (a quadratic in one parameter, FP64).  Parameters a hair outside [0, 1] are
//   accepted so that no hit falls through the seam between two sub-patches or
//   two patches; such edge hits that repeat one another (same sign, heights
//   within a tolerance) count once.  One warp per query, lanes over patches,
//   hits gathered in shared memory.  For grids of queries one ray per (x, y)
//   column serves every cell of the column (ray reuse, as Sec. 4.4.1 does
//   for voxelization).
//
// f: with r = phi(t) - q, L = |r|, the definitions of Algorithm 2 reduce to
//   f dt = -(1/4pi) (r_x dr_y - r_y dr_x) (L + r_z) / (L (r_x^2 + r_y^2))
//        = -(1/4pi) (r_x dr_y - r_y dr_x) / (L (L - r_z)),
//   i.e. -(1 + cos theta) d phi / 4pi in spherical angles about q (the Dirac
//   monopole potential with its string along x0).  The first form is used for
//   r_z > 0, the second otherwise, so that no difference cancels.
//
// The integral over each curve: adaptive Gauss-Kronrod 15 (embedded Gauss 7
// for the error), dyadic panels.  Panels of depth <= 12 come from a
// per-curve tree built on the host in FP64: each node holds its centre (as a
// float pair) and its four control points relative to the centre in FP32, so
// that a panel's control points relative to q carry errors of the panel's own
// scale; its 15 integrand values are then FP32.  Deeper panels (a curve
// passing within ~2^-12 of its length of the ray or of q) are
// integrated in FP64 from the curve's control points.  A panel is accepted
// when its error estimate is below tol (b - a) or below the rounding level of
// its values (for FP32 panels only while that level is below 2^-18 / 4 pi);
// each query has a panel budget.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "fp32x2.cuh"
#include "gwn_internal.cuh"

namespace gwn {

namespace {

constexpr double kInv4PiD = 0.079577471545947667884;
constexpr int kStackPatch = 96;      // sub-patch stack: up to 3 pending rectangles per level
constexpr int kMaxDepth = 24;       // leaf depth cap (dyadic parameters exact in FP32)
constexpr int kMaxQuadDepth = 48;
constexpr int kWarps = 4;            // queries (warps) per block
constexpr int kHitCap = 128;         // gathered edge hits per ray (per warp)
constexpr float kNoiseCap = 0x1p-18f;  // largest rounding level an FP32 panel may be accepted at (x 4 pi)
constexpr double kParamSlack = 1e-9;

struct D3 {
    double x, y, z;
};
__host__ __device__ __forceinline__ D3 d3(double x, double y, double z) { return {x, y, z}; }
__host__ __device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__host__ __device__ __forceinline__ D3 lerp(D3 a, D3 b, double t) { return a + t * (b - a); }

// Control points of the piece [a, b] of the cubic with control points p.
__host__ __device__ void cubic_piece(const D3 p[4], double a, double b, D3 out[4]) {
    // split at b, keep the left part [0, b]
    D3 q01 = lerp(p[0], p[1], b), q12 = lerp(p[1], p[2], b), q23 = lerp(p[2], p[3], b);
    D3 q012 = lerp(q01, q12, b), q123 = lerp(q12, q23, b);
    D3 L[4] = {p[0], q01, q012, lerp(q012, q123, b)};
    if (a <= 0.0) {
        for (int k = 0; k < 4; ++k) out[k] = L[k];
        return;
    }
    // split [0, b] at a / b, keep the right part [a, b]
    const double s = a / b;
    q01 = lerp(L[0], L[1], s);
    q12 = lerp(L[1], L[2], s);
    q23 = lerp(L[2], L[3], s);
    q012 = lerp(q01, q12, s);
    q123 = lerp(q12, q23, s);
    out[0] = lerp(q012, q123, s);
    out[1] = q123;
    out[2] = q23;
    out[3] = L[3];
}

__device__ __forceinline__ D3 load_cp(const double *C, int i, int j) {
    const double *c = C + 3 * (4 * i + j);
    return d3(c[0], c[1], c[2]);
}

// Edge hits of one ray, gathered per warp in shared memory (height, sign):
// hits within the slack of their bilinear patch's edge, the only ones that can
// be found twice.  Interior hits go straight to the sink.
struct EdgeHits {
    double z[kHitCap];
    int sign[kHitCap];
    int n;
};

// Interior hits of a single query: summed per lane.
struct PointSink {
    EdgeHits *eh;
    int sum;
    __device__ void interior(double, int sign) { sum += sign; }
};

// Interior hits of a grid column: the hit's sign is added to the column's
// difference array (the chi output of the column) at the highest cell below
// the hit; a suffix sum over the column then gives every cell's chi.
struct ColumnSink {
    EdgeHits *eh;
    const float *gz;
    int nz;
    int32_t *col;         // chi of cell (k) of this column at col[k * stride]
    int64_t stride;
    __device__ int cells_below(double z) const {   // #{k : gz[k] < z}, gz non-decreasing
        int lo = 0, hi = nz;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((double)gz[mid] < z) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    }
    __device__ void interior(double z, int sign) {
        const int k = cells_below(z);
        if (k > 0) atomicAdd(&col[(int64_t)(k - 1) * stride], sign);
    }
};

__device__ __forceinline__ void push_edge(EdgeHits &eh, double z, int sign) {
    const int slot = atomicAdd(&eh.n, 1);
    if (slot < kHitCap) {
        eh.z[slot] = z;
        eh.sign[slot] = sign;
    }
}

// +z ray from q against the bilinear patch through the corners P00
// (s = t = 0), P10 (s = 1), P01 (t = 1), P11: every hit above q.z with s, t in
// [-slack, 1 + slack] goes to the sink (interior) or the warp's edge buffer.
template <class Sink>
__device__ void bilinear_crossings(D3 P00, D3 P10, D3 P01, D3 P11, D3 q, Sink &sink) {
    const D3 A = P00 - q, B = P10 - P00, C = P01 - P00, D = (P00 - P10) - (P01 - P11);
    // xy: A + s B + t C + s t D = 0  ->  (A + s B) x (C + s D) = 0 (2-D cross)
    auto cr = [](D3 a, D3 b) { return a.x * b.y - a.y * b.x; };
    const double qa = cr(B, D), qb = cr(A, D) + cr(B, C), qc = cr(A, C);
    double roots[2];
    int nr = 0;
    if (fabs(qa) <= 1e-300) {
        if (fabs(qb) > 1e-300) roots[nr++] = -qc / qb;
    } else {
        const double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            const double r = -0.5 * (qb + (qb >= 0.0 ? sq : -sq));   // stable pair of roots
            roots[nr++] = r / qa;
            if (r != 0.0) roots[nr++] = qc / r;
        }
    }
    for (int k = 0; k < nr; ++k) {
        const double s = roots[k];
        if (!(s >= -kParamSlack && s <= 1.0 + kParamSlack)) continue;
        const D3 e = C + s * D, f = A + s * B;
        double t;
        if (fabs(e.x) >= fabs(e.y)) {
            if (e.x == 0.0) continue;
            t = -f.x / e.x;
        } else {
            t = -f.y / e.y;
        }
        if (!(t >= -kParamSlack && t <= 1.0 + kParamSlack)) continue;
        const double z = A.z + s * B.z + t * C.z + s * t * D.z;   // hit height minus q.z
        if (!(z > 0.0)) continue;
        const D3 ds = B + t * D, dt = C + s * D;
        const double nz = ds.x * dt.y - ds.y * dt.x;
        if (nz == 0.0) continue;
        const bool edge = fmin(fmin(s, 1.0 - s), fmin(t, 1.0 - t)) <= 2.0 * kParamSlack;
        if (edge) push_edge(*sink.eh, q.z + z, nz > 0.0 ? 1 : -1);
        else sink.interior(q.z + z, nz > 0.0 ? 1 : -1);
    }
}

// Per-patch data of the subdivision: the control net relative to the patch's
// centre in FP32 (nodes are culled on FP32 nets, with a margin covering their
// rounding), the centre, that margin, and the depth at which every sub-patch
// lies within the flatness tolerance of its bilinear patch.
struct PatchInfo {
    float net[48];      // C[i][j] - centre, [i][j][xyz]
    float chi[3], clo[3];   // the centre as a float pair (hi + lo)
    float margin;       // bound on the FP32 nets' rounding error (any coordinate)
    int depth;          // leaf depth
};

// q - centre of a patch in FP32: the float pair's difference with q, exact up
// to one rounding (TwoSum of hi - q).
__device__ __forceinline__ float minus_centre(float q, float hi, float lo) {
    const float s = hi - q, bb = s - hi, e = (hi - (s - bb)) + (-q - bb);
    return -(s + (e + lo));
}

// Control net of the sub-patch [u0, u1] x [v0, v1] from an FP32 net.
__device__ void sub_patch_f32(const float *N, float u0, float u1, float v0, float v1, float S[4][4][3]) {
    auto piece = [](const float p[4], float a, float b, float out[4]) {
        float q01 = fmaf(b, p[1] - p[0], p[0]), q12 = fmaf(b, p[2] - p[1], p[1]), q23 = fmaf(b, p[3] - p[2], p[2]);
        float q012 = fmaf(b, q12 - q01, q01), q123 = fmaf(b, q23 - q12, q12);
        const float L[4] = {p[0], q01, q012, fmaf(b, q123 - q012, q012)};
        if (a <= 0.f) {
            for (int k = 0; k < 4; ++k) out[k] = L[k];
            return;
        }
        const float s = a / b;
        q01 = fmaf(s, L[1] - L[0], L[0]);
        q12 = fmaf(s, L[2] - L[1], L[1]);
        q23 = fmaf(s, L[3] - L[2], L[2]);
        q012 = fmaf(s, q12 - q01, q01);
        q123 = fmaf(s, q23 - q12, q12);
        out[0] = fmaf(s, q123 - q012, q012);
        out[1] = q123;
        out[2] = q23;
        out[3] = L[3];
    };
    for (int k = 0; k < 3; ++k) {
        float T[4][4];
        for (int j = 0; j < 4; ++j) {
            const float col[4] = {N[(0 * 4 + j) * 3 + k], N[(1 * 4 + j) * 3 + k], N[(2 * 4 + j) * 3 + k],
                                  N[(3 * 4 + j) * 3 + k]};
            float out[4];
            piece(col, u0, u1, out);
            for (int i = 0; i < 4; ++i) T[i][j] = out[i];
        }
        for (int i = 0; i < 4; ++i) {
            float out[4];
            piece(T[i], v0, v1, out);
            for (int j = 0; j < 4; ++j) S[i][j][k] = out[j];
        }
    }
}

// S(u, v) of the FP64 patch C by its Bernstein sums in a fixed order, so that a
// corner shared by two sub-patches is computed bit for bit alike.
__device__ D3 patch_point(const double *C, double u, double v) {
    const double su = 1.0 - u, sv = 1.0 - v;
    const double bu[4] = {su * su * su, 3.0 * su * su * u, 3.0 * su * u * u, u * u * u};
    const double bv[4] = {sv * sv * sv, 3.0 * sv * sv * v, 3.0 * sv * v * v, v * v * v};
    D3 r = d3(0.0, 0.0, 0.0);
    for (int i = 0; i < 4; ++i) {
        D3 row = d3(0.0, 0.0, 0.0);
        for (int j = 0; j < 4; ++j) row = row + bv[j] * load_cp(C, i, j);
        r = r + bu[i] * row;
    }
    return r;
}

// One sub-patch (depth d, indices iu, iv) against the +z ray (qx, qy, qz: the
// ray's origin relative to the patch's centre in FP32, e: the culling margin):
// 0 if the origin lies outside its FP32 net's xy box or above its top by more
// than e, 1 if it is a leaf to intersect, 2 if its four children are to be
// visited.
__device__ int visit_node(const PatchInfo &pi, float qx, float qy, float qz, float e, unsigned iu, unsigned iv,
                          int d) {
    const float h = ldexpf(1.0f, -d);
    float S[4][4][3];
    sub_patch_f32(pi.net, iu * h, (iu + 1) * h, iv * h, (iv + 1) * h, S);
    float xlo = S[0][0][0], xhi = xlo, ylo = S[0][0][1], yhi = ylo, zhi = S[0][0][2];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            xlo = fminf(xlo, S[i][j][0]);
            xhi = fmaxf(xhi, S[i][j][0]);
            ylo = fminf(ylo, S[i][j][1]);
            yhi = fmaxf(yhi, S[i][j][1]);
            zhi = fmaxf(zhi, S[i][j][2]);
        }
    if (qx < xlo - e || qx > xhi + e || qy < ylo - e || qy > yhi + e || qz >= zhi + e) return 0;
    return d < pi.depth ? 2 : 1;
}

// The +z ray from q against a leaf: the bilinear patch through its FP64
// corners.
template <class Sink>
__device__ void leaf_crossings(const double *C, D3 q, unsigned iu, unsigned iv, int d, Sink &sink) {
    const double hd = ldexp(1.0, -d), u0 = iu * hd, u1 = (iu + 1) * hd, v0 = iv * hd, v1 = (iv + 1) * hd;
    bilinear_crossings(patch_point(C, u0, v0), patch_point(C, u1, v0), patch_point(C, u0, v1), patch_point(C, u1, v1),
                       q, sink);
}

// The ray's origin relative to a patch's centre, and the culling margin.
struct LocalRay {
    float x, y, z, e;
};
__device__ __forceinline__ LocalRay local_ray(const PatchInfo &pi, float qx, float qy, float qz) {
    LocalRay r;
    r.x = minus_centre(qx, pi.chi[0], pi.clo[0]);
    r.y = minus_centre(qy, pi.chi[1], pi.clo[1]);
    r.z = minus_centre(qz, pi.chi[2], pi.clo[2]);
    r.e = pi.margin + 2.0f * 0x1p-24f * fmaxf(fabsf(r.x), fmaxf(fabsf(r.y), fabsf(r.z)));
    return r;
}

// The crossings below one sub-patch, depth first with a stack of its own (the
// fallback when a warp's node queue is full).  False if the stack or node
// budget ran out.
template <class Sink>
__device__ __noinline__ bool subtree_crossings(const double *C, const PatchInfo &pi, int max_nodes, D3 q, unsigned iu0,
                                  unsigned iv0, int d0, Sink &sink) {
    unsigned st_u[kStackPatch], st_v[kStackPatch];
    unsigned char st_d[kStackPatch];
    int top = 0, nodes = 0;
    st_u[0] = iu0;
    st_v[0] = iv0;
    st_d[top++] = (unsigned char)d0;
    const LocalRay r = local_ray(pi, (float)q.x, (float)q.y, (float)q.z);
    while (top > 0) {
        if (++nodes > max_nodes) return false;
        --top;
        const unsigned iu = st_u[top], iv = st_v[top];
        const int d = st_d[top];
        const int kind = visit_node(pi, r.x, r.y, r.z, r.e, iu, iv, d);
        if (kind == 1) leaf_crossings(C, q, iu, iv, d, sink);
        if (kind != 2) continue;
        if (top + 4 > kStackPatch) return false;
        for (int k = 0; k < 4; ++k) {
            st_u[top] = 2 * iu + (k & 1);
            st_v[top] = 2 * iv + (k >> 1);
            st_d[top++] = (unsigned char)(d + 1);
        }
    }
    return true;
}

// Sub-patches waiting in a warp's queues: nodes to test (FP32) and leaves to
// intersect (FP64), so that each round runs 32 of one kind.
constexpr int kNodeQ = 512;
constexpr int kLeafQ = 192;
struct NodeQueue {
    int patch[kNodeQ];
    unsigned iu[kNodeQ], iv[kNodeQ];
    unsigned char d[kNodeQ];
    int n;
    int lpatch[kLeafQ];
    unsigned liu[kLeafQ], liv[kLeafQ];
    unsigned char ld[kLeafQ];
    int nl;
};

// Every hit of the +z ray from q with the patches first, first + step, ...:
// the warp's lanes take 32 sub-patches per round from the shared node queue
// (root patches, after the box test, fill the lanes it leaves free) and queue
// the children of the sub-patches they split, so that the work of one deep
// patch spreads over the warp; leaves wait in the leaf queue and are
// intersected 32 per round (whenever 32 are waiting, and at the end).
// Budget: max_nodes per patch of the warp; when a queue is full a lane
// finishes the work on its own.  False on every lane if a budget ran out.
template <class Sink>
__device__ bool gather_hits(D3 q, const double *__restrict__ patches, const PatchInfo *__restrict__ pinfo, int np,
                            const double *__restrict__ pbox, int max_nodes, Sink &sink, NodeQueue &Q, int first,
                            int step) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) Q.n = Q.nl = 0;
    __syncwarp();
    const float fx = (float)q.x, fy = (float)q.y, fz = (float)q.z;
    const int mine = first < np ? (np - first + step - 1) / step : 0;
    const long long budget = (long long)max_nodes * mine;
    long long used = 0;
    int next = first;
    bool ok = true;
    while (true) {
        const int nl = Q.nl;
        const int n0 = Q.n;
        const int left = next < np ? (np - next + step - 1) / step : 0;
        if (nl >= 32 || (n0 == 0 && left == 0 && nl > 0)) {
            // a round of leaves
            const int take = min(nl, 32);
            int pk = -1, d = 0;
            unsigned iu = 0, iv = 0;
            if (lane < take) {
                const int s = nl - take + lane;
                pk = Q.lpatch[s];
                iu = Q.liu[s];
                iv = Q.liv[s];
                d = Q.ld[s];
            }
            __syncwarp();
            if (lane == 0) Q.nl = nl - take;
            __syncwarp();
            if (pk >= 0) leaf_crossings(patches + 48 * (size_t)pk, q, iu, iv, d, sink);
            __syncwarp();
            continue;
        }
        const int take = min(n0, 32);
        const int roots = min(32 - take, left);
        if (take + roots == 0) break;
        int pk = -1, d = 0;
        unsigned iu = 0, iv = 0;
        if (lane < take) {
            const int s = n0 - take + lane;
            pk = Q.patch[s];
            iu = Q.iu[s];
            iv = Q.iv[s];
            d = Q.d[s];
        } else if (lane < take + roots) {
            pk = next + (lane - take) * step;
            const double *b = pbox + 5 * pk;   // xlo, xhi, ylo, yhi, zhi of the patch's net
            if (q.x < b[0] || q.x > b[1] || q.y < b[2] || q.y > b[3] || q.z >= b[4]) pk = -1;
        }
        next += roots * step;
        __syncwarp();
        if (lane == 0) Q.n = n0 - take;
        __syncwarp();
        const bool stop = used >= budget;
        used += take + roots;
        if (pk >= 0) {
            const PatchInfo &pi = pinfo[pk];
            const LocalRay r = local_ray(pi, fx, fy, fz);
            const int kind = visit_node(pi, r.x, r.y, r.z, r.e, iu, iv, d);
            if (kind == 1) {
                const int s = atomicAdd(&Q.nl, 1);
                if (s < kLeafQ) {
                    Q.lpatch[s] = pk;
                    Q.liu[s] = iu;
                    Q.liv[s] = iv;
                    Q.ld[s] = (unsigned char)d;
                } else {
                    atomicSub(&Q.nl, 1);
                    leaf_crossings(patches + 48 * (size_t)pk, q, iu, iv, d, sink);
                }
            } else if (kind == 2) {
                if (stop) {
                    ok = false;
                } else {
                    const int s = atomicAdd(&Q.n, 4);
                    if (s + 4 <= kNodeQ) {
                        for (int k = 0; k < 4; ++k) {
                            Q.patch[s + k] = pk;
                            Q.iu[s + k] = 2 * iu + (k & 1);
                            Q.iv[s + k] = 2 * iv + (k >> 1);
                            Q.d[s + k] = (unsigned char)(d + 1);
                        }
                    } else {
                        atomicSub(&Q.n, 4);
                        const double *C = patches + 48 * (size_t)pk;
                        for (int k = 0; k < 4; ++k)
                            ok &= subtree_crossings(C, pi, max_nodes, q, 2 * iu + (k & 1), 2 * iv + (k >> 1), d + 1,
                                                    sink);
                    }
                }
            }
        }
        __syncwarp();
    }
    return __all_sync(0xffffffffu, ok);
}

// Whether edge hit h counts: unless another edge hit of the same sign lies
// within `same` below it (ties broken by slot), so that a crossing found from
// both sides of a seam counts once.
__device__ __forceinline__ bool edge_counts(const EdgeHits &eh, int cnt, int h, double same) {
    const int sh = eh.sign[h];
    const double zh = eh.z[h];
    for (int j = 0; j < cnt; ++j) {
        if (j == h || eh.sign[j] != sh) continue;
        const double zj = eh.z[j];
        if (fabs(zj - zh) <= same && (zj < zh || (zj == zh && j < h))) return false;
    }
    return true;
}

__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// chi of n queries: one warp per query.
__global__ void __launch_bounds__(32 * kWarps) k_param_chi(const float *__restrict__ q, int64_t n,
                                                           const double *__restrict__ patches,
                                                           const PatchInfo *__restrict__ pinfo, int np,
                                                           const double *__restrict__ pbox, double same,
                                                           int max_nodes, int32_t *__restrict__ chi,
                                                           unsigned long long *__restrict__ status) {
    __shared__ EdgeHits sh[kWarps];
    __shared__ NodeQueue nq[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
    if (i >= n) return;   // the whole warp leaves together
    EdgeHits &eh = sh[warp];
    if (lane == 0) eh.n = 0;
    __syncwarp();
    const D3 p = d3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    PointSink sink{&eh, 0};
    const bool ok = gather_hits(p, patches, pinfo, np, pbox, max_nodes, sink, nq[warp], 0, 1);
    const int total = eh.n, cnt = min(total, kHitCap);
    int c = sink.sum;
    for (int h = lane; h < cnt; h += 32)
        if (edge_counts(eh, cnt, h, same)) c += eh.sign[h];
    c = warp_sum(c);
    if (lane == 0) {
        chi[i] = c;
        if (!ok || total > kHitCap) atomicAdd(&status[0], 1ull);
    }
}

// chi of every cell of a grid (x fastest), z non-decreasing: one block per
// (x, y) column casts a single ray from zstart (below the surface), its warps
// sharing out the patches; each hit adds its sign to the column's difference
// array at the highest cell below it, and a suffix sum over the column gives
// each cell the hits above it.
__global__ void __launch_bounds__(32 * kWarps) k_param_grid_chi(
    const float *__restrict__ gx, int nx, const float *__restrict__ gy, int ny, const float *__restrict__ gz, int nz,
    double zstart, const double *__restrict__ patches, const PatchInfo *__restrict__ pinfo, int np,
    const double *__restrict__ pbox, double same, int max_nodes, int32_t *__restrict__ chi,
    unsigned long long *__restrict__ status) {
    __shared__ EdgeHits eh;
    __shared__ NodeQueue nq[kWarps];
    __shared__ int all_ok;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c0 = blockIdx.x;
    const int ix = (int)(c0 % nx), iy = (int)(c0 / nx);
    const int64_t stride = (int64_t)nx * ny;
    int32_t *col = chi + (int64_t)iy * nx + ix;
    if (threadIdx.x == 0) {
        eh.n = 0;
        all_ok = 1;
    }
    for (int k = threadIdx.x; k < nz; k += blockDim.x) col[k * stride] = 0;
    __syncthreads();
    const D3 p = d3(gx[ix], gy[iy], zstart);
    ColumnSink sink{&eh, gz, nz, col, stride};
    const bool ok = gather_hits(p, patches, pinfo, np, pbox, max_nodes, sink, nq[warp], warp, kWarps);
    if (!ok && lane == 0) all_ok = 0;
    __syncthreads();
    const int total = eh.n, cnt = min(total, kHitCap);
    for (int h = threadIdx.x; h < cnt; h += blockDim.x)
        if (edge_counts(eh, cnt, h, same)) sink.interior(eh.z[h], eh.sign[h]);
    __syncthreads();
    if (warp != 0) return;
    // suffix sum, 32 cells at a time from the top
    int carry = 0;
    for (int base = ((nz - 1) / 32) * 32; base >= 0; base -= 32) {
        const int k = base + lane;
        int v = k < nz ? col[k * stride] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_down_sync(0xffffffffu, v, o);
            if (lane + o < 32) v += u;
        }
        v += carry;
        if (k < nz) col[k * stride] = v;
        carry = __shfl_sync(0xffffffffu, v, 0);
    }
    if (lane == 0 && (!all_ok || total > kHitCap)) atomicAdd(&status[0], 1ull);
}

// ---------------------------------------------------------------------------
// Boundary integral
// ---------------------------------------------------------------------------

// One stored panel of a curve: control points relative to the panel's centre
// (FP32, by coordinate: dx = (d0.x, d1.x, d2.x, d3.x)) and the centre as a
// float pair (c = hi + lo).
struct PanelNode {
    float4 dx, dy, dz;
    float4 chi;   // (cx, cy, cz, R^2): high parts of the centre, squared radius of the control points about it
    float4 clo;   // low parts
};
static_assert(sizeof(PanelNode) == 80, "panel node layout");

// Gauss-Kronrod 15 on [0, 1]: Bernstein values and derivative weights of the
// cubic at the 15 nodes, Kronrod weights and the embedded Gauss 7 weights (0
// at Kronrod-only nodes), in FP32 and FP64.  Written by gwn_param_create.
struct GKTables {
    float bf[15][4], dbf[15][4], wkf[15], wgf[15];
    double bd[15][4], dbd[15][4], wkd[15], wgd[15];
    // the nodes in symmetric pairs (s_j, 1 - s_j), j < 7, for paired FP32:
    // Bernstein values, y-derivative weights, negated x-derivative weights,
    // negated Kronrod and Gauss weights, Kronrod weights
    float2 bp[7][4], dyp[7][4], ndxp[7][4], nwk[7], nwg[7], wk[7];
};
__constant__ GKTables c_gk;

// Kronrod nodes on [-1, 1] (positive half, decreasing, then 0) and weights;
// Gauss 7 nodes are entries 1, 3, 5 and 0, with weights kGauss.
constexpr double kXgk[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                            0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                            0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                            0.207784955007898467600689403773245, 0.0};
constexpr double kWgk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                            0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                            0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                            0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
constexpr double kGauss[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                              0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

GKTables make_gk_tables() {
    GKTables t{};
    for (int j = 0; j < 15; ++j) {
        // node j: j < 7 left of the centre, 7 the centre, j > 7 right
        const int m = j < 7 ? j : (j == 7 ? 7 : 14 - j);
        const double x = (j < 7 ? -kXgk[m] : kXgk[m]), s = 0.5 + 0.5 * x, r = 1.0 - s;
        const double b[4] = {r * r * r, 3 * r * r * s, 3 * r * s * s, s * s * s};
        const double db[4] = {-3 * r * r, 3 * r * r - 6 * r * s, 6 * r * s - 3 * s * s, 3 * s * s};
        const double wk = 0.5 * kWgk[m];
        const double wg = (m == 7) ? 0.5 * kGauss[3] : ((m & 1) ? 0.5 * kGauss[m >> 1] : 0.0);
        for (int k = 0; k < 4; ++k) {
            t.bd[j][k] = b[k];
            t.dbd[j][k] = db[k];
            t.bf[j][k] = (float)b[k];
            t.dbf[j][k] = (float)db[k];
        }
        t.wkd[j] = wk;
        t.wgd[j] = wg;
        t.wkf[j] = (float)wk;
        t.wgf[j] = (float)wg;
    }
    for (int j = 0; j < 7; ++j) {
        const int m = 14 - j;   // the mirror node 1 - s_j
        for (int k = 0; k < 4; ++k) {
            t.bp[j][k] = make_float2(t.bf[j][k], t.bf[m][k]);
            t.dyp[j][k] = make_float2(t.dbf[j][k], t.dbf[m][k]);
            t.ndxp[j][k] = make_float2(-t.dbf[j][k], -t.dbf[m][k]);
        }
        t.nwk[j] = make_float2(-t.wkf[j], -t.wkf[m]);
        t.nwg[j] = make_float2(-t.wgf[j], -t.wgf[m]);
        t.wk[j] = make_float2(t.wkf[j], t.wkf[m]);
    }
    return t;
}

struct PanelResult {
    // integral of f, |K15 - G7|, and the Kronrod sum of (|r_x dr_y| + |r_y dr_x|) g,
    // the scale of the rounding errors of the 15 values (all times 4 pi); whether
    // the panel is resolved (its control points' radius within its nodes'
    // distance from the ray's string and from q)
    double val, err, abs;
    bool resolved;
};

// FP32 panel from a stored node: r_k = (c - q) + d_k, with c - q taken from the
// float pair exactly up to one rounding.  The 14 nodes off the centre are
// evaluated in mirrored pairs with paired FP32 instructions; the reciprocal
// square root and the reciprocal are the SFU approximations (relative error
// below 2^-22, inside the panel's rounding scale).  Writes the integral, |K15 - G7| and the rounding scale (times 4
// pi); returns false if any is not finite (the caller redoes the panel in FP64).
__device__ __forceinline__ bool panel_f32(const PanelNode &nd, float qx, float qy, float qz, float &val, float &err,
                                          float &scale, float &near2) {
    auto diff = [](float hi, float lo, float q) {
        // (hi - q) + lo with the rounding error of hi - q kept (TwoSum)
        const float s = hi - q, bb = s - hi, e = (hi - (s - bb)) + (-q - bb);
        return s + (e + lo);
    };
    const float cx = diff(nd.chi.x, nd.clo.x, qx), cy = diff(nd.chi.y, nd.clo.y, qy), cz = diff(nd.chi.z, nd.clo.z, qz);
    const float rx[4] = {cx + nd.dx.x, cx + nd.dx.y, cx + nd.dx.z, cx + nd.dx.w};
    const float ry[4] = {cy + nd.dy.x, cy + nd.dy.y, cy + nd.dy.z, cy + nd.dy.w};
    const float rz[4] = {cz + nd.dz.x, cz + nd.dz.y, cz + nd.dz.z, cz + nd.dz.w};
    // the 14 nodes off the centre in mirrored pairs, two per paired instruction
    float2 RX[4], RY[4], RZ[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        RX[k] = bc2(rx[k]);
        RY[k] = bc2(ry[k]);
        RZ[k] = bc2(rz[k]);
    }
    float2 K2 = bc2(0.f), G2 = bc2(0.f), A2 = bc2(0.f);
    float2 N2 = bc2(3.0e38f);   // squared distance to the nearest singular point: the ray's string, or q
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const float2 *b = c_gk.bp[j], *dyw = c_gk.dyp[j], *ndxw = c_gk.ndxp[j];
        const float2 x = fma2(b[0], RX[0], fma2(b[1], RX[1], fma2(b[2], RX[2], mul2(b[3], RX[3]))));
        const float2 y = fma2(b[0], RY[0], fma2(b[1], RY[1], fma2(b[2], RY[2], mul2(b[3], RY[3]))));
        const float2 z = fma2(b[0], RZ[0], fma2(b[1], RZ[1], fma2(b[2], RZ[2], mul2(b[3], RZ[3]))));
        const float2 ndx = fma2(ndxw[0], RX[0], fma2(ndxw[1], RX[1], fma2(ndxw[2], RX[2], mul2(ndxw[3], RX[3]))));
        const float2 dy = fma2(dyw[0], RY[0], fma2(dyw[1], RY[1], fma2(dyw[2], RY[2], mul2(dyw[3], RY[3]))));
        const float2 xdy = mul2(x, dy), nydx = mul2(y, ndx);
        const float2 c = add2(xdy, nydx);
        const float2 rho2 = fma2(x, x, mul2(y, y));
        const float2 l2 = fma2(z, z, rho2);
        const float2 inv_l = make_float2(sfu_rsqrt(l2.x), sfu_rsqrt(l2.y));
        const float2 l = mul2(l2, inv_l);
        const float2 lpz = add2(l, z), lmz = fma2(z, bc2(-1.f), l);
        // g = (L + z) / (L rho^2) above q, 1 / (L (L - z)) elsewhere
        N2 = make_float2(fminf(N2.x, z.x > 0.f ? rho2.x : l2.x), fminf(N2.y, z.y > 0.f ? rho2.y : l2.y));
        const float2 num = make_float2(z.x > 0.f ? lpz.x : 1.f, z.y > 0.f ? lpz.y : 1.f);
        const float2 den = make_float2(z.x > 0.f ? rho2.x : lmz.x, z.y > 0.f ? rho2.y : lmz.y);
        const float2 g = mul2(mul2(num, inv_l), make_float2(sfu_rcp(den.x), sfu_rcp(den.y)));
        const float2 cg = mul2(c, g);   // f = -c g
        const float2 sc = make_float2(fabsf(xdy.x) + fabsf(nydx.x), fabsf(xdy.y) + fabsf(nydx.y));
        K2 = fma2(c_gk.nwk[j], cg, K2);
        G2 = fma2(c_gk.nwg[j], cg, G2);
        A2 = fma2(c_gk.wk[j], mul2(sc, g), A2);
    }
    // the centre node
    float K, G, A;
    {
        const float *b = c_gk.bf[7], *db = c_gk.dbf[7];
        const float x = fmaf(b[0], rx[0], fmaf(b[1], rx[1], fmaf(b[2], rx[2], b[3] * rx[3])));
        const float y = fmaf(b[0], ry[0], fmaf(b[1], ry[1], fmaf(b[2], ry[2], b[3] * ry[3])));
        const float z = fmaf(b[0], rz[0], fmaf(b[1], rz[1], fmaf(b[2], rz[2], b[3] * rz[3])));
        const float dx = fmaf(db[0], rx[0], fmaf(db[1], rx[1], fmaf(db[2], rx[2], db[3] * rx[3])));
        const float dy = fmaf(db[0], ry[0], fmaf(db[1], ry[1], fmaf(db[2], ry[2], db[3] * ry[3])));
        const float xdy = x * dy, ydx = y * dx;
        const float c = xdy - ydx;
        const float rho2 = fmaf(x, x, y * y);
        const float l2 = fmaf(z, z, rho2);
        const float inv_l = sfu_rsqrt(l2);
        const float l = l2 * inv_l;
        const bool up = z > 0.f;
        const float g = (up ? l + z : 1.f) * inv_l * sfu_rcp(up ? rho2 : l - z);
        const float cg = c * g;
        near2 = fminf(fminf(N2.x, N2.y), up ? rho2 : l2);
        K = fmaf(-c_gk.wkf[7], cg, K2.x + K2.y);
        G = fmaf(-c_gk.wgf[7], cg, G2.x + G2.y);
        A = fmaf(c_gk.wkf[7], (fabsf(xdy) + fabsf(ydx)) * g, A2.x + A2.y);
    }
    val = K;
    err = fabsf(K - G);
    scale = A;
    return isfinite(K) && isfinite(G) && isfinite(A);
}

// FP64 panel [a, b] of the curve P (12 doubles), control points relative to q.
__device__ void panel_f64(const double *P, D3 q, double a, double b, PanelResult &out) {
    D3 p[4], loc[4];
    for (int k = 0; k < 4; ++k) p[k] = d3(P[3 * k], P[3 * k + 1], P[3 * k + 2]);
    cubic_piece(p, a, b, loc);
    double rx[4], ry[4], rz[4];
    for (int k = 0; k < 4; ++k) {
        rx[k] = loc[k].x - q.x;
        ry[k] = loc[k].y - q.y;
        rz[k] = loc[k].z - q.z;
    }
    double K = 0.0, G = 0.0, A = 0.0, near2 = 1e300;
    for (int j = 0; j < 15; ++j) {
        const double *bb = c_gk.bd[j], *db = c_gk.dbd[j];
        const double x = bb[0] * rx[0] + bb[1] * rx[1] + bb[2] * rx[2] + bb[3] * rx[3];
        const double y = bb[0] * ry[0] + bb[1] * ry[1] + bb[2] * ry[2] + bb[3] * ry[3];
        const double z = bb[0] * rz[0] + bb[1] * rz[1] + bb[2] * rz[2] + bb[3] * rz[3];
        const double dx = db[0] * rx[0] + db[1] * rx[1] + db[2] * rx[2] + db[3] * rx[3];
        const double dy = db[0] * ry[0] + db[1] * ry[1] + db[2] * ry[2] + db[3] * ry[3];
        const double c = x * dy - y * dx;
        const double rho2 = x * x + y * y;
        const double L = sqrt(rho2 + z * z);
        const double g = z > 0.0 ? (L + z) / (L * rho2) : 1.0 / (L * (L - z));
        const double f = c == 0.0 ? 0.0 : -c * g;
        near2 = fmin(near2, z > 0.0 ? rho2 : rho2 + z * z);
        K += c_gk.wkd[j] * f;
        G += c_gk.wgd[j] * f;
        A += c_gk.wkd[j] * (fabs(x * dy) + fabs(y * dx)) * g;
    }
    out.val = K;
    out.err = fabs(K - G);
    out.abs = A;
    const double cx = 0.25 * (rx[0] + rx[1] + rx[2] + rx[3]), cy = 0.25 * (ry[0] + ry[1] + ry[2] + ry[3]),
                 cz = 0.25 * (rz[0] + rz[1] + rz[2] + rz[3]);
    double r2 = 0.0;
    for (int k = 0; k < 4; ++k) {
        const double ex = rx[k] - cx, ey = ry[k] - cy, ez = rz[k] - cz;
        r2 = fmax(r2, ex * ex + ey * ey + ez * ez);
    }
    out.resolved = r2 <= near2;
}

// Query points: an array of n points, or the cells of a grid (x fastest).
struct PointList {
    const float *q;
    __device__ void get(int64_t i, float &x, float &y, float &z) const {
        x = q[3 * i];
        y = q[3 * i + 1];
        z = q[3 * i + 2];
    }
};
struct GridPoints {
    const float *gx, *gy, *gz;
    int nx, ny;
    __device__ void get(int64_t i, float &x, float &y, float &z) const {
        x = gx[i % nx];
        y = gy[(i / nx) % ny];
        z = gz[i / ((int64_t)nx * ny)];
    }
};

// Panels waiting in a warp's queues: curve, dyadic index, depth.  FP32 panels
// (depth <= the tree's) and FP64 panels wait apart, so that each round of the
// warp evaluates 32 panels of one kind.
constexpr int kQ32 = 512;
constexpr int kQ64 = 256;
struct PanelQueues {
    int c32[kQ32];
    unsigned k32[kQ32];
    unsigned char d32[kQ32];
    int c64[kQ64];
    unsigned long long k64[kQ64];
    unsigned char d64[kQ64];
    int n32, n64;
};

// Reserve two slots of a queue; false (and the count restored) if it is full.
__device__ __forceinline__ int reserve2(int *n, int cap) {
    const int s = atomicAdd(n, 2);
    if (s + 2 <= cap) return s;
    atomicSub(n, 2);
    return -1;
}

// w = chi + (boundary integral) of n points: one warp per point.  The warp's
// lanes take 32 panels per round from a shared queue (the curves' root panels
// first come in order), so that every lane has work while any is left: a
// panel is accepted when its error estimate is below tol4pi 2^-d or below 16
// units of rounding of its rounding scale (capped at kNoiseCap for FP32
// panels), else its halves are queued.  FP32
// panels come from the panel trees; deeper panels, and any whose FP32 values
// are not finite, are done in FP64 after all FP32 work.  The point's budget is
// max_panels per curve; past it (or past the queues' capacity or the depth
// limit) panels are accepted as they are and the point is flagged.
template <class Points>
__global__ void __launch_bounds__(32 * kWarps) k_param_boundary(Points pts, int64_t n,
                                                                const PanelNode *__restrict__ tree, int tree_nodes,
                                                                int tree_depth, const double *__restrict__ curves,
                                                                int nc, double tol4pi, int max_panels, int fp64,
                                                                const int32_t *__restrict__ chi,
                                                                float *__restrict__ w,
                                                                unsigned long long *__restrict__ status) {
    __shared__ PanelQueues sq[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
    if (i >= n) return;
    PanelQueues &Q = sq[warp];
    if (lane == 0) Q.n32 = Q.n64 = 0;
    __syncwarp();
    float qx, qy, qz;
    pts.get(i, qx, qy, qz);
    const D3 p = d3(qx, qy, qz);
    const float tol_f = (float)tol4pi;
    const long long budget = (long long)max_panels * nc;
    long long used = 0;   // panels taken by the warp (the same on every lane)
    float acc_f = 0.f;
    double acc_d = 0.0;
    bool ok = true;
    int mine = 0, mine64 = 0;
    int next_root = 0;

    auto push64 = [&](int cv, unsigned long long k, int d) -> bool {
        const int s = reserve2(&Q.n64, kQ64);
        if (s < 0) return false;
        Q.c64[s] = Q.c64[s + 1] = cv;
        Q.k64[s] = 2 * k;
        Q.k64[s + 1] = 2 * k + 1;
        Q.d64[s] = Q.d64[s + 1] = (unsigned char)(d + 1);
        return true;
    };

    // FP32 rounds (the root panels too, unless every panel is FP64)
    while (!fp64) {
        const int n32 = Q.n32;
        const int take = min(n32, 32);
        const int roots = min(32 - take, nc - next_root);
        if (take + roots == 0) break;
        int cv = -1, d = 0;
        unsigned k = 0;
        if (lane < take) {
            const int s = n32 - take + lane;
            cv = Q.c32[s];
            k = Q.k32[s];
            d = Q.d32[s];
        } else if (lane < take + roots) {
            cv = next_root + lane - take;
        }
        next_root += roots;
        __syncwarp();
        if (lane == 0) Q.n32 = n32 - take;
        __syncwarp();
        const bool stop = used >= budget;
        used += take + roots;
        if (cv >= 0) {
            ++mine;
            float val, err, scale, near2;
            const PanelNode &nd = tree[(size_t)cv * tree_nodes + ((1u << d) - 1) + k];
            if (!panel_f32(nd, qx, qy, qz, val, err, scale, near2)) {
                // the same panel in FP64: queue it as the "child" of its parent slot
                const int s = atomicAdd(&Q.n64, 1);
                if (s < kQ64) {
                    Q.c64[s] = cv;
                    Q.k64[s] = k;
                    Q.d64[s] = (unsigned char)d;
                } else {
                    atomicSub(&Q.n64, 1);
                    const double h = ldexp(1.0, -d);
                    PanelResult pr;
                    panel_f64(curves + 12 * (size_t)cv, p, (double)k * h, (double)(k + 1) * h, pr);
                    acc_d += pr.val;
                    ok = false;
                }
            } else {
                // the rounding level stands in for the target only while it is small in
                // absolute terms: near the ray's string a radial stretch of curve can
                // carry a rounding scale far above its integral, and FP32 values there
                // are that noisy, so such a panel is refined (in FP64 below the tree)
                // and only once the panel is resolved: its control points' radius
                // within the distance of its nodes from the integrand's singular
                // set, the string and q (a narrower feature could lie between the
                // nodes, where neither rule sees it)
                const float noise = 16.0f * 0x1p-24f * scale;
                const bool resolved = nd.chi.w <= near2;
                const bool conv = resolved && err <= fmaxf(ldexpf(tol_f, -d), noise <= kNoiseCap ? noise : 0.f);
                bool done = conv || stop;
                if (!done) {
                    if (d + 1 <= tree_depth) {
                        const int s = reserve2(&Q.n32, kQ32);
                        if (s >= 0) {
                            Q.c32[s] = Q.c32[s + 1] = cv;
                            Q.k32[s] = 2 * k;
                            Q.k32[s + 1] = 2 * k + 1;
                            Q.d32[s] = Q.d32[s + 1] = (unsigned char)(d + 1);
                        } else {
                            done = true;
                        }
                    } else if (!push64(cv, k, d)) {
                        done = true;
                    }
                }
                if (done) {
                    acc_f += val;
                    if (!conv) ok = false;
                }
            }
        }
        __syncwarp();
    }
    // FP64 rounds (the root panels when every panel is FP64)
    while (true) {
        const int n64 = Q.n64;
        const int take = min(n64, 32);
        const int roots = fp64 ? min(32 - take, nc - next_root) : 0;
        if (take + roots == 0) break;
        int cv = -1, d = 0;
        unsigned long long k = 0;
        if (lane < take) {
            const int s = n64 - take + lane;
            cv = Q.c64[s];
            k = Q.k64[s];
            d = Q.d64[s];
        } else if (lane < take + roots) {
            cv = next_root + lane - take;
        }
        next_root += roots;
        __syncwarp();
        if (lane == 0) Q.n64 = n64 - take;
        __syncwarp();
        const bool stop = used >= budget;
        used += take + roots;
        if (cv >= 0) {
            ++mine;
            ++mine64;
            const double h = ldexp(1.0, -d);
            PanelResult pr;
            panel_f64(curves + 12 * (size_t)cv, p, (double)k * h, (double)(k + 1) * h, pr);
            const bool conv = pr.resolved && pr.err <= fmax(tol4pi * h, 16.0 * DBL_EPSILON * pr.abs);
            if (conv || stop || d >= kMaxQuadDepth || !push64(cv, k, d)) {
                acc_d += pr.val;
                if (!conv) ok = false;
            }
        }
        __syncwarp();
    }
    const double acc = warp_sum(acc_d + (double)acc_f);
    const int panels = warp_sum(mine), panels64 = warp_sum(mine64);
    const bool all_ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        w[i] = (float)((double)chi[i] + acc * kInv4PiD);
        if (!all_ok) atomicAdd(&status[1], 1ull);
        atomicAdd(&status[2], (unsigned long long)panels);
        if (panels64) atomicAdd(&status[3], (unsigned long long)panels64);
    }
}

}  // namespace

}  // namespace gwn

using namespace gwn;

// A parametric surface on the device: patches, their net boxes, the boundary
// curves of the union and their panel trees.
struct gwn_param {
    int device = 0;
    int np = 0, nc = 0;
    gwn_param_config cfg{};
    double *patches = nullptr;   // [np][4][4][3]
    PatchInfo *pinfo = nullptr;  // [np]
    double *pbox = nullptr;      // [np][5]: x range, y range, top of the net
    double *curves = nullptr;    // [nc][4][3]
    PanelNode *tree = nullptr;   // [nc][tree_nodes]
    int tree_depth = 0, tree_nodes = 0;
    unsigned long long *status = nullptr;   // [0]: subdivision budget hits, [1]: unconverged integrals,
                                            // [2]: quadrature panels evaluated, [3]: of them in FP64
    double flat = 0.0;           // bilinear tolerance (absolute)
    double same = 0.0;           // edge hits of one ray closer than this (same sign) are one crossing
    double zlo = 0.0;            // below every control point: start of the grid rays
    std::vector<float> h_curves;
    // pinned staging of host grid axes (a copy from pageable memory would wait
    // for the stream), reused once the event says its last copy has finished
    mutable std::mutex stage_mu;
    mutable float *stage = nullptr;
    mutable size_t stage_cap = 0;
    mutable cudaEvent_t stage_done = nullptr;
};

namespace {

// Oriented boundary of the union: each patch's four edge curves counter-clockwise
// about S_u x S_v (v = 0 along +u, u = 1 along +v, v = 1 along -u, u = 0 along
// -v); a curve and its exact reverse cancel (net multiplicity per curve).
std::vector<float> extract_boundary(const float *P, int np) {
    using Key = std::vector<float>;
    std::vector<Key> curves;
    auto cp = [&](int p, int i, int j, int k) { return P[((size_t)p * 16 + 4 * i + j) * 3 + k]; };
    for (int p = 0; p < np; ++p) {
        const int idx[4][4][2] = {{{0, 0}, {1, 0}, {2, 0}, {3, 0}},
                                  {{3, 0}, {3, 1}, {3, 2}, {3, 3}},
                                  {{3, 3}, {2, 3}, {1, 3}, {0, 3}},
                                  {{0, 3}, {0, 2}, {0, 1}, {0, 0}}};
        for (int e = 0; e < 4; ++e) {
            Key c(12);
            for (int m = 0; m < 4; ++m)
                for (int k = 0; k < 3; ++k) c[3 * m + k] = cp(p, idx[e][m][0], idx[e][m][1], k);
            curves.push_back(c);
        }
    }
    std::map<Key, int> count;
    for (auto &c : curves) ++count[c];
    std::map<Key, int> used;
    std::vector<float> out;
    for (auto &c : curves) {
        Key r(12);
        for (int m = 0; m < 4; ++m)
            for (int k = 0; k < 3; ++k) r[3 * m + k] = c[3 * (3 - m) + k];
        const auto it = count.find(r);
        const int net = count[c] - (it == count.end() ? 0 : it->second);
        if (net > 0 && used[c] < net) {
            out.insert(out.end(), c.begin(), c.end());
            ++used[c];
        }
    }
    return out;
}

// Panel tree of one curve (FP64 de Casteljau halving), nodes in heap order:
// node (d, k) covering [k 2^-d, (k + 1) 2^-d] at index 2^d - 1 + k.
void build_tree(const double *P, int depth, PanelNode *out) {
    std::vector<D3> level(4), next;
    for (int k = 0; k < 4; ++k) level[k] = d3(P[3 * k], P[3 * k + 1], P[3 * k + 2]);
    for (int d = 0; d <= depth; ++d) {
        const int cnt = 1 << d;
        for (int k = 0; k < cnt; ++k) {
            const D3 *p = &level[4 * k];
            const D3 c = 0.25 * (((p[0] + p[1]) + p[2]) + p[3]);
            PanelNode &nd = out[(cnt - 1) + k];
            const float hx = (float)c.x, hy = (float)c.y, hz = (float)c.z;
            double r2 = 0.0;
            for (int m = 0; m < 4; ++m) {
                const D3 e = p[m] - c;
                r2 = std::max(r2, e.x * e.x + e.y * e.y + e.z * e.z);
            }
            nd.chi = make_float4(hx, hy, hz, (float)r2);
            nd.clo = make_float4((float)(c.x - hx), (float)(c.y - hy), (float)(c.z - hz), 0.f);
            float dxs[4], dys[4], dzs[4];
            for (int m = 0; m < 4; ++m) {
                dxs[m] = (float)(p[m].x - c.x);
                dys[m] = (float)(p[m].y - c.y);
                dzs[m] = (float)(p[m].z - c.z);
            }
            nd.dx = make_float4(dxs[0], dxs[1], dxs[2], dxs[3]);
            nd.dy = make_float4(dys[0], dys[1], dys[2], dys[3]);
            nd.dz = make_float4(dzs[0], dzs[1], dzs[2], dzs[3]);
        }
        if (d == depth) break;
        next.resize((size_t)8 * cnt);
        for (int k = 0; k < cnt; ++k) {
            const D3 *p = &level[4 * k];
            const D3 a = 0.5 * (p[0] + p[1]), b = 0.5 * (p[1] + p[2]), e = 0.5 * (p[2] + p[3]);
            const D3 ab = 0.5 * (a + b), be = 0.5 * (b + e), m = 0.5 * (ab + be);
            D3 *l = &next[8 * k], *r = l + 4;
            l[0] = p[0], l[1] = a, l[2] = ab, l[3] = m;
            r[0] = m, r[1] = be, r[2] = e, r[3] = p[3];
        }
        level.swap(next);
    }
}

// The quadrature tables go to each device's constant memory once per process.
std::mutex g_tables_mu;
bool g_tables_ready[64] = {};

gwn_status upload_tables(int device) {
    std::lock_guard<std::mutex> lock(g_tables_mu);
    if (device >= 0 && device < 64 && g_tables_ready[device]) return GWN_OK;
    const GKTables t = make_gk_tables();
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_gk, &t, sizeof(t)));
    if (device >= 0 && device < 64) g_tables_ready[device] = true;
    return GWN_OK;
}

bool is_device_memory(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The three grid axes in one stream-ordered device allocation (x, then y, then
// z).  Host axes go through the surface's pinned staging buffer, so that the
// copy does not wait for the stream's earlier work; device axes are copied on
// the stream.
gwn_status stage_axes(const gwn_param *g, const float *x, int32_t nx, const float *y, int32_t ny, const float *z,
                      int32_t nz, float **d_out, cudaStream_t s) {
    const size_t total = (size_t)nx + ny + nz;
    float *d = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&d, sizeof(float) * std::max<size_t>(total, 1), s));
    *d_out = d;
    const float *src[3] = {x, y, z};
    const size_t len[3] = {(size_t)nx, (size_t)ny, (size_t)nz};
    if (is_device_memory(x) || is_device_memory(y) || is_device_memory(z)) {
        size_t off = 0;
        for (int a = 0; a < 3; ++a) {
            GWN_CUDA_TRY(cudaMemcpyAsync(d + off, src[a], sizeof(float) * len[a], cudaMemcpyDefault, s));
            off += len[a];
        }
        return GWN_OK;
    }
    std::lock_guard<std::mutex> lock(g->stage_mu);
    if (g->stage_done) GWN_CUDA_TRY(cudaEventSynchronize(g->stage_done));
    if (g->stage_cap < total) {
        if (g->stage) cudaFreeHost(g->stage);
        g->stage = nullptr;
        g->stage_cap = 0;
        GWN_CUDA_TRY(cudaHostAlloc((void **)&g->stage, sizeof(float) * total, cudaHostAllocDefault));
        g->stage_cap = total;
    }
    if (!g->stage_done) GWN_CUDA_TRY(cudaEventCreateWithFlags(&g->stage_done, cudaEventDisableTiming));
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
        std::memcpy(g->stage + off, src[a], sizeof(float) * len[a]);
        off += len[a];
    }
    GWN_CUDA_TRY(cudaMemcpyAsync(d, g->stage, sizeof(float) * total, cudaMemcpyHostToDevice, s));
    GWN_CUDA_TRY(cudaEventRecord(g->stage_done, s));
    return GWN_OK;
}

gwn_status check_device_ptrs(int device, std::initializer_list<const void *> ptrs, const char *what) {
    for (const void *p : ptrs) {
        const int kind = pointer_kind(p, device);
        if (kind < 0)
            return set_error(GWN_ERR_INVALID_ARG, std::string(what) + ": a buffer is device memory of another GPU "
                                                                      "than the surface's");
        if (kind == 0) return set_error(GWN_ERR_INVALID_ARG, std::string(what) + " takes device pointers for its outputs");
    }
    return GWN_OK;
}

}  // namespace

extern "C" {

void gwn_param_config_default(gwn_param_config *cfg) {
    if (!cfg) return;
    cfg->quad_tol = 1e-10;
    cfg->flat_tol = 1e-6;
    cfg->fp64 = 0;
    cfg->max_panels = 1024;
    cfg->max_nodes = 1 << 16;
}

gwn_status gwn_param_create(const float *patches, int32_t np, const gwn_param_config *cfg, gwn_param **out) {
    clear_error();
    if (!out) return set_error(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (np < 0 || (np > 0 && !patches)) return set_error(GWN_ERR_INVALID_ARG, "patches / np");
    if (np > (1 << 24)) return set_error(GWN_ERR_INVALID_ARG, "at most 2^24 patches");
    gwn_param_config c;
    gwn_param_config_default(&c);
    if (cfg) c = *cfg;
    if (!(c.quad_tol > 0.0) || !(c.flat_tol > 0.0) || c.max_panels < 1 || c.max_nodes < 1)
        return set_error(GWN_ERR_INVALID_ARG, "config: quad_tol, flat_tol > 0; max_panels, max_nodes >= 1");
    std::vector<float> hp;
    if (np > 0) {
        hp.resize((size_t)np * 48);
        GWN_CUDA_TRY(cudaMemcpy(hp.data(), patches, sizeof(float) * hp.size(), cudaMemcpyDefault));
        for (float v : hp)
            if (!std::isfinite(v)) return set_error(GWN_ERR_INVALID_MESH, "control point is not finite");
    }
    int device = 0;
    GWN_CUDA_TRY(cudaGetDevice(&device));
    if (gwn_status st = upload_tables(device)) return st;
    gwn_param *g = new gwn_param();
    g->device = device;
    g->cfg = c;
    g->np = np;
    g->h_curves = extract_boundary(hp.data(), np);
    g->nc = (int)(g->h_curves.size() / 12);
    std::vector<double> dp(hp.begin(), hp.end()), box((size_t)np * 5), dc(g->h_curves.begin(), g->h_curves.end());
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int p = 0; p < np; ++p) {
        double b[5] = {INFINITY, -INFINITY, INFINITY, -INFINITY, -INFINITY};
        for (int m = 0; m < 16; ++m) {
            const double *q = dp.data() + (size_t)p * 48 + 3 * m;
            b[0] = std::min(b[0], q[0]);
            b[1] = std::max(b[1], q[0]);
            b[2] = std::min(b[2], q[1]);
            b[3] = std::max(b[3], q[1]);
            b[4] = std::max(b[4], q[2]);
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], q[k]);
                hi[k] = std::max(hi[k], q[k]);
            }
        }
        for (int k = 0; k < 5; ++k) box[(size_t)p * 5 + k] = b[k];
    }
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, np > 0 ? hi[k] - lo[k] : 0.0);
    ext = std::max(ext, 1e-30);
    g->flat = c.flat_tol * ext;
    g->same = 4.0 * g->flat;
    std::vector<PatchInfo> info(np);
    for (int p = 0; p < np; ++p) {
        const double *P = dp.data() + (size_t)p * 48;
        PatchInfo &pi = info[p];
        double ctr[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < 16; ++m)
            for (int k = 0; k < 3; ++k) ctr[k] += P[3 * m + k] / 16.0;
        double R = 0.0, Au = 0.0, Av = 0.0;
        for (int m = 0; m < 16; ++m)
            for (int k = 0; k < 3; ++k) {
                pi.net[3 * m + k] = (float)(P[3 * m + k] - ctr[k]);
                R = std::max(R, std::fabs(P[3 * m + k] - ctr[k]));
            }
        auto cp = [&](int i, int j, int k) { return P[(4 * i + j) * 3 + k]; };
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 4; ++b)
                for (int k = 0; k < 3; ++k) {
                    Au = std::max(Au, std::fabs(cp(a + 2, b, k) - 2.0 * cp(a + 1, b, k) + cp(a, b, k)));
                    Av = std::max(Av, std::fabs(cp(b, a + 2, k) - 2.0 * cp(b, a + 1, k) + cp(b, a, k)));
                }
        for (int k = 0; k < 3; ++k) {
            pi.chi[k] = (float)ctr[k];
            pi.clo[k] = (float)(ctr[k] - (double)pi.chi[k]);
        }
        // FP32 nets: the root's rounding, 12 lerp levels and the rounded split
        // factors stay below 40 units of R; 64 units leave room
        pi.margin = (float)(64.0 * 0x1p-24 * R) + 1e-30f;
        // |S - bilinear| <= h^2 / 8 (max|S_uu| + max|S_vv|), |S_uu| <= 6 max|second difference|
        const double dev0 = 0.75 * (Au + Av);
        int depth = 0;
        while (depth < kMaxDepth && dev0 * std::ldexp(1.0, -2 * depth) > g->flat) ++depth;
        pi.depth = depth;
    }
    g->zlo = np > 0 ? lo[2] - 1.0 - ext : 0.0;
    // panel trees: depth <= 12, at most 1 GiB in all
    int depth = 12;
    while (depth > 0 && (double)g->nc * (double)((2 << depth) - 1) * sizeof(PanelNode) > (double)(1ull << 30)) --depth;
    g->tree_depth = depth;
    g->tree_nodes = (2 << depth) - 1;
    std::vector<PanelNode> tree((size_t)g->nc * g->tree_nodes);
    for (int k = 0; k < g->nc; ++k) build_tree(dc.data() + 12 * (size_t)k, depth, tree.data() + (size_t)k * g->tree_nodes);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&g->status, sizeof(unsigned long long) * 4)) != cudaSuccess ||
        (np > 0 && ((e = cudaMalloc(&g->patches, sizeof(double) * dp.size())) != cudaSuccess ||
                    (e = cudaMalloc(&g->pinfo, sizeof(PatchInfo) * info.size())) != cudaSuccess ||
                    (e = cudaMalloc(&g->pbox, sizeof(double) * box.size())) != cudaSuccess)) ||
        (g->nc > 0 && ((e = cudaMalloc(&g->curves, sizeof(double) * dc.size())) != cudaSuccess ||
                       (e = cudaMalloc(&g->tree, sizeof(PanelNode) * tree.size())) != cudaSuccess))) {
        gwn_param_destroy(g);
        return set_error(GWN_ERR_OOM, cudaGetErrorString(e));
    }
    cudaMemset(g->status, 0, sizeof(unsigned long long) * 4);
    if (np > 0) {
        cudaMemcpy(g->patches, dp.data(), sizeof(double) * dp.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(g->pinfo, info.data(), sizeof(PatchInfo) * info.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(g->pbox, box.data(), sizeof(double) * box.size(), cudaMemcpyHostToDevice);
    }
    if (g->nc > 0) {
        cudaMemcpy(g->curves, dc.data(), sizeof(double) * dc.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(g->tree, tree.data(), sizeof(PanelNode) * tree.size(), cudaMemcpyHostToDevice);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        gwn_param_destroy(g);
        return set_error(GWN_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = g;
    return GWN_OK;
}

gwn_status gwn_param_destroy(gwn_param *g) {
    clear_error();
    if (!g) return GWN_OK;
    for (void *p : {(void *)g->patches, (void *)g->pinfo, (void *)g->pbox, (void *)g->curves, (void *)g->tree,
                    (void *)g->status})
        if (p) cudaFree(p);
    if (g->stage_done) {
        cudaEventSynchronize(g->stage_done);
        cudaEventDestroy(g->stage_done);
    }
    if (g->stage) cudaFreeHost(g->stage);
    delete g;
    return GWN_OK;
}

gwn_status gwn_param_get_boundary(const gwn_param *g, float *curves, int32_t cap, int32_t *n_out) {
    clear_error();
    if (!g || !n_out) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    *n_out = g->nc;
    if (curves && cap > 0) std::memcpy(curves, g->h_curves.data(), sizeof(float) * 12 * std::min(cap, g->nc));
    return GWN_OK;
}

}  // extern "C"

namespace {

// The boundary integral of n points (an array or a grid) after chi.
template <class Points>
void launch_boundary(const gwn_param *g, Points pts, int64_t n, const int32_t *chi, float *w, cudaStream_t s) {
    ProfScope prof("param_boundary", s);
    k_param_boundary<<<grid_for(n, kWarps), 32 * kWarps, 0, s>>>(
        pts, n, g->tree, g->tree_nodes, g->tree_depth, g->curves, g->nc, g->cfg.quad_tol * 4.0 * M_PI,
        g->cfg.max_panels, g->cfg.fp64, chi, w, g->status);
}

}  // namespace

extern "C" {

gwn_status gwn_param_query(const gwn_param *g, const float *q, int64_t n, float *w, int32_t *chi_or_null,
                           void *stream) {
    clear_error();
    if (!g) return set_error(GWN_ERR_INVALID_ARG, "surface is NULL");
    if (n < 0 || n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "0 <= n < 2^31");
    if (n == 0) return GWN_OK;
    if (!q || !w) return set_error(GWN_ERR_INVALID_ARG, "q / w is NULL");
    if (gwn_status st = check_device_ptrs(g->device, {q, w, chi_or_null}, "gwn_param_query")) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *chi = chi_or_null;
    if (!chi) GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, s));
    {
        ProfScope prof("param_chi", s);
        k_param_chi<<<grid_for(n, kWarps), 32 * kWarps, 0, s>>>(q, n, g->patches, g->pinfo, g->np, g->pbox, g->same,
                                                                 g->cfg.max_nodes, chi, g->status);
    }
    launch_boundary(g, PointList{q}, n, chi, w, s);
    if (!chi_or_null) cudaFreeAsync(chi, s);
    GWN_LAUNCH_CHECK("parametric query");
    return GWN_OK;
}

gwn_status gwn_param_query_grid(const gwn_param *g, const float *x, int32_t nx, const float *y, int32_t ny,
                                const float *z, int32_t nz, float *w, int32_t *chi_or_null, void *stream) {
    clear_error();
    if (!g) return set_error(GWN_ERR_INVALID_ARG, "surface is NULL");
    if (nx < 0 || ny < 0 || nz < 0) return set_error(GWN_ERR_INVALID_ARG, "negative grid size");
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "nx * ny * nz < 2^31");
    if (n == 0) return GWN_OK;
    if (!x || !y || !z || !w) return set_error(GWN_ERR_INVALID_ARG, "x / y / z / w is NULL");
    if (gwn_status st = check_device_ptrs(g->device, {w, chi_or_null}, "gwn_param_query_grid")) return st;
    {
        // z is read where it lies: in place in host memory, else copied back
        std::vector<float> hz;
        const float *zh = z;
        if (is_device_memory(z)) {
            hz.resize(nz);
            GWN_CUDA_TRY(cudaMemcpy(hz.data(), z, sizeof(float) * nz, cudaMemcpyDeviceToHost));
            zh = hz.data();
        }
        for (int k = 0; k < nz; ++k)
            if (!std::isfinite(zh[k]) || (k > 0 && zh[k] < zh[k - 1]))
                return set_error(GWN_ERR_INVALID_ARG, "z must be finite and non-decreasing");
    }
    cudaStream_t s = (cudaStream_t)stream;
    float *axes = nullptr;
    int32_t *chi = chi_or_null;
    if (gwn_status st = stage_axes(g, x, nx, y, ny, z, nz, &axes, s)) return st;
    const float *dx = axes, *dy = axes + nx, *dz = axes + nx + ny;
    if (!chi) GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, s));
    {
        ProfScope prof("param_grid_chi", s);
        const int64_t cols = (int64_t)nx * ny;
        k_param_grid_chi<<<(unsigned)cols, 32 * kWarps, 0, s>>>(dx, nx, dy, ny, dz, nz, g->zlo, g->patches,
                                                                        g->pinfo, g->np, g->pbox, g->same,
                                                                        g->cfg.max_nodes, chi, g->status);
    }
    launch_boundary(g, GridPoints{dx, dy, dz, nx, ny}, n, chi, w, s);
    if (!chi_or_null) cudaFreeAsync(chi, s);
    cudaFreeAsync(axes, s);
    GWN_LAUNCH_CHECK("parametric grid query");
    return GWN_OK;
}

gwn_status gwn_param_status(const gwn_param *g, uint64_t *budget_hits, uint64_t *unconverged, uint64_t *panels,
                            uint64_t *panels_fp64, int reset) {
    clear_error();
    if (!g) return set_error(GWN_ERR_INVALID_ARG, "surface is NULL");
    unsigned long long h[4];
    GWN_CUDA_TRY(cudaMemcpy(h, g->status, sizeof(h), cudaMemcpyDeviceToHost));
    if (reset) GWN_CUDA_TRY(cudaMemset(g->status, 0, sizeof(h)));
    if (budget_hits) *budget_hits = h[0];
    if (unconverged) *unconverged = h[1];
    if (panels) *panels = h[2];
    if (panels_fp64) *panels_fp64 = h[3];
    return GWN_OK;
}

}  // extern "C"
