// Winding numbers of parametric surfaces (Sec. 4.4, Algorithm 2): untrimmed
// bicubic Bezier patches C[p][i][j] (i along u, j along v), oriented by
// S_u x S_v.  w = chi + sum over the boundary curves of the integral of
// f(phi, t) = (w(t) - d eta(t)) / 4pi, with x0 = +z, x1 = -z.
//
// chi: signed crossings of the ray q + s x0 with the surface (Sec. 4.4.1).
//   Each patch is subdivided (de Casteljau on the parameter rectangle, FP64)
//   while its control net's xy hull contains q and the net rises above q,
//   until the net lies within the flatness tolerance of the bilinear patch
//   through its corners; the +z ray then meets that bilinear patch in closed
//   form (a quadratic in one parameter).  Parameters a hair outside [0, 1] are
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
// for the error), dyadic panels.  Panels of depth <= 10 come from a
// per-curve tree built on the host in FP64: each node holds its centre (as a
// float pair) and its four control points relative to the centre in FP32, so
// that a panel's control points relative to q carry errors of the panel's own
// scale; its 15 integrand values are then FP32.  Deeper panels (a curve
// passing within ~2^-10 of its length of the ray or of q) are
// integrated in FP64 from the curve's control points.  A panel is accepted
// when its error estimate is below tol (b - a) or below the rounding level of
// its own integral of |f|; each (query, curve) pair has a panel budget.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "gwn_internal.cuh"

namespace gwn {

namespace {

constexpr double kInv4PiD = 0.079577471545947667884;
constexpr int kStackPatch = 96;      // sub-patch stack: up to 3 pending rectangles per level
constexpr int kMaxDepth = 30;
constexpr int kStackQuad = 64;       // quadrature panel stack
constexpr int kMaxQuadDepth = 48;
constexpr int kWarps = 4;            // queries (warps) per block
constexpr int kHitCap = 128;         // gathered edge hits per ray (per warp)
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

// Control net of the sub-patch [u0, u1] x [v0, v1] of patch C (48 doubles).
__device__ void sub_patch(const double *C, double u0, double u1, double v0, double v1, D3 S[4][4]) {
    D3 T[4][4];
    for (int j = 0; j < 4; ++j) {
        D3 col[4] = {load_cp(C, 0, j), load_cp(C, 1, j), load_cp(C, 2, j), load_cp(C, 3, j)}, out[4];
        cubic_piece(col, u0, u1, out);
        for (int i = 0; i < 4; ++i) T[i][j] = out[i];
    }
    for (int i = 0; i < 4; ++i) {
        D3 out[4];
        cubic_piece(T[i], v0, v1, out);
        for (int j = 0; j < 4; ++j) S[i][j] = out[j];
    }
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

struct Rect {
    double u0, u1, v0, v1;
};

// Crossings of the +z ray from q with one patch: subdivision while the net's
// xy hull holds q and the net rises above it, bilinear intersection once the
// net is flat.  Returns false if the depth, stack or node budget ran out.
template <class Sink>
__device__ bool patch_crossings(const double *C, double flat, int max_nodes, D3 q, Sink &sink) {
    Rect st[kStackPatch];
    unsigned char dep[kStackPatch];
    int top = 0, nodes = 0;
    st[top] = {0.0, 1.0, 0.0, 1.0};
    dep[top++] = 0;
    bool ok = true;
    while (top > 0) {
        if (++nodes > max_nodes) return false;
        const Rect r = st[--top];
        const int d = dep[top];
        D3 S[4][4];
        sub_patch(C, r.u0, r.u1, r.v0, r.v1, S);
        double xlo = S[0][0].x, xhi = xlo, ylo = S[0][0].y, yhi = ylo, zhi = S[0][0].z;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                xlo = fmin(xlo, S[i][j].x);
                xhi = fmax(xhi, S[i][j].x);
                ylo = fmin(ylo, S[i][j].y);
                yhi = fmax(yhi, S[i][j].y);
                zhi = fmax(zhi, S[i][j].z);
            }
        if (q.x < xlo || q.x > xhi || q.y < ylo || q.y > yhi || q.z >= zhi) continue;
        // flatness: distance of the net from the bilinear interpolation of its
        // corners (bounds the patch's distance from the bilinear patch)
        double dev = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                const double s = i / 3.0, t = j / 3.0;
                const D3 b = (1 - s) * ((1 - t) * S[0][0] + t * S[0][3]) + s * ((1 - t) * S[3][0] + t * S[3][3]);
                const D3 e = S[i][j] - b;
                dev = fmax(dev, fmax(fabs(e.x), fmax(fabs(e.y), fabs(e.z))));
            }
        if (dev <= flat || d >= kMaxDepth) {
            if (d >= kMaxDepth && dev > flat) ok = false;
            bilinear_crossings(S[0][0], S[3][0], S[0][3], S[3][3], q, sink);
            continue;
        }
        if (top + 4 > kStackPatch) {
            ok = false;
            continue;
        }
        const double um = 0.5 * (r.u0 + r.u1), vm = 0.5 * (r.v0 + r.v1);
        const Rect kids[4] = {{r.u0, um, r.v0, vm}, {um, r.u1, r.v0, vm}, {r.u0, um, vm, r.v1}, {um, r.u1, vm, r.v1}};
        for (int k = 0; k < 4; ++k) {
            st[top] = kids[k];
            dep[top++] = (unsigned char)(d + 1);
        }
    }
    return ok;
}

// Every hit of the +z ray from q over all patches (lanes over patches).  False
// on every lane if any budget ran out.
template <class Sink>
__device__ bool gather_hits(D3 q, const double *__restrict__ patches, int np, const double *__restrict__ pbox,
                            double flat, int max_nodes, Sink &sink) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int k = lane; k < np; k += 32) {
        const double *b = pbox + 5 * k;   // xlo, xhi, ylo, yhi, zhi of the patch's net
        if (q.x < b[0] || q.x > b[1] || q.y < b[2] || q.y > b[3] || q.z >= b[4]) continue;
        ok &= patch_crossings(patches + 48 * k, flat, max_nodes, q, sink);
    }
    __syncwarp();
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
                                                           const double *__restrict__ patches, int np,
                                                           const double *__restrict__ pbox, double flat, double same,
                                                           int max_nodes, int32_t *__restrict__ chi,
                                                           unsigned long long *__restrict__ status) {
    __shared__ EdgeHits sh[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
    if (i >= n) return;   // the whole warp leaves together
    EdgeHits &eh = sh[warp];
    if (lane == 0) eh.n = 0;
    __syncwarp();
    const D3 p = d3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    PointSink sink{&eh, 0};
    const bool ok = gather_hits(p, patches, np, pbox, flat, max_nodes, sink);
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

// chi of every cell of a grid (x fastest), z non-decreasing: one warp per
// (x, y) column casts a single ray from zstart (below the surface); each hit
// adds its sign to the column's difference array at the highest cell below
// it, and a suffix sum over the column gives each cell the hits above it.
__global__ void __launch_bounds__(32 * kWarps) k_param_grid_chi(
    const float *__restrict__ gx, int nx, const float *__restrict__ gy, int ny, const float *__restrict__ gz, int nz,
    double zstart, const double *__restrict__ patches, int np, const double *__restrict__ pbox, double flat,
    double same, int max_nodes, int32_t *__restrict__ chi, unsigned long long *__restrict__ status) {
    __shared__ EdgeHits sh[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c0 = (int64_t)blockIdx.x * kWarps + warp;
    if (c0 >= (int64_t)nx * ny) return;
    const int ix = (int)(c0 % nx), iy = (int)(c0 / nx);
    const int64_t stride = (int64_t)nx * ny;
    int32_t *col = chi + (int64_t)iy * nx + ix;
    EdgeHits &eh = sh[warp];
    if (lane == 0) eh.n = 0;
    for (int k = lane; k < nz; k += 32) col[k * stride] = 0;
    __syncwarp();
    const D3 p = d3(gx[ix], gy[iy], zstart);
    ColumnSink sink{&eh, gz, nz, col, stride};
    const bool ok = gather_hits(p, patches, np, pbox, flat, max_nodes, sink);
    const int total = eh.n, cnt = min(total, kHitCap);
    for (int h = lane; h < cnt; h += 32)
        if (edge_counts(eh, cnt, h, same)) sink.interior(eh.z[h], eh.sign[h]);
    __syncwarp();
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
    if (lane == 0 && (!ok || total > kHitCap)) atomicAdd(&status[0], 1ull);
}

// ---------------------------------------------------------------------------
// Boundary integral
// ---------------------------------------------------------------------------

// One stored panel of a curve: control points relative to the panel's centre
// (FP32, by coordinate: dx = (d0.x, d1.x, d2.x, d3.x)) and the centre as a
// float pair (c = hi + lo).
struct PanelNode {
    float4 dx, dy, dz;
    float4 chi;   // (cx, cy, cz, 0) high parts
    float4 clo;   // low parts
};
static_assert(sizeof(PanelNode) == 80, "panel node layout");

// Gauss-Kronrod 15 on [0, 1]: Bernstein values and derivative weights of the
// cubic at the 15 nodes, Kronrod weights and the embedded Gauss 7 weights (0
// at Kronrod-only nodes), in FP32 and FP64.  Written by gwn_param_create.
struct GKTables {
    float bf[15][4], dbf[15][4], wkf[15], wgf[15];
    double bd[15][4], dbd[15][4], wkd[15], wgd[15];
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
    return t;
}

struct PanelResult {
    // integral of f, |K15 - G7|, and the Kronrod sum of (|r_x dr_y| + |r_y dr_x|) g,
    // the scale of the rounding errors of the 15 values (all times 4 pi)
    double val, err, abs;
};

// FP32 panel from a stored node: r_k = (c - q) + d_k, with c - q taken from the
// float pair exactly up to one rounding; returns false if any value is not
// finite (the caller redoes the panel in FP64).
__device__ bool panel_f32(const PanelNode &nd, float qx, float qy, float qz, PanelResult &out) {
    auto diff = [](float hi, float lo, float q) {
        // (hi - q) + lo with the rounding error of hi - q kept (TwoSum)
        const float s = hi - q, bb = s - hi, e = (hi - (s - bb)) + (-q - bb);
        return s + (e + lo);
    };
    const float cx = diff(nd.chi.x, nd.clo.x, qx), cy = diff(nd.chi.y, nd.clo.y, qy), cz = diff(nd.chi.z, nd.clo.z, qz);
    const float rx[4] = {cx + nd.dx.x, cx + nd.dx.y, cx + nd.dx.z, cx + nd.dx.w};
    const float ry[4] = {cy + nd.dy.x, cy + nd.dy.y, cy + nd.dy.z, cy + nd.dy.w};
    const float rz[4] = {cz + nd.dz.x, cz + nd.dz.y, cz + nd.dz.z, cz + nd.dz.w};
    float K = 0.f, G = 0.f, A = 0.f;
#pragma unroll
    for (int j = 0; j < 15; ++j) {
        const float *b = c_gk.bf[j], *db = c_gk.dbf[j];
        const float x = fmaf(b[0], rx[0], fmaf(b[1], rx[1], fmaf(b[2], rx[2], b[3] * rx[3])));
        const float y = fmaf(b[0], ry[0], fmaf(b[1], ry[1], fmaf(b[2], ry[2], b[3] * ry[3])));
        const float z = fmaf(b[0], rz[0], fmaf(b[1], rz[1], fmaf(b[2], rz[2], b[3] * rz[3])));
        const float dx = fmaf(db[0], rx[0], fmaf(db[1], rx[1], fmaf(db[2], rx[2], db[3] * rx[3])));
        const float dy = fmaf(db[0], ry[0], fmaf(db[1], ry[1], fmaf(db[2], ry[2], db[3] * ry[3])));
        const float c = fmaf(x, dy, -y * dx);
        const float rho2 = fmaf(x, x, y * y);
        const float L = __fsqrt_rn(fmaf(z, z, rho2));
        const float g = z > 0.f ? (L + z) * __frcp_rn(L * rho2) : __frcp_rn(L * (L - z));
        const float f = c == 0.f ? 0.f : -c * g;
        K = fmaf(c_gk.wkf[j], f, K);
        G = fmaf(c_gk.wgf[j], f, G);
        A = fmaf(c_gk.wkf[j], (fabsf(x * dy) + fabsf(y * dx)) * g, A);
    }
    out.val = K;
    out.err = fabs((double)K - (double)G);
    out.abs = A;
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
    double K = 0.0, G = 0.0, A = 0.0;
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
        K += c_gk.wkd[j] * f;
        G += c_gk.wgd[j] * f;
        A += c_gk.wkd[j] * (fabs(x * dy) + fabs(y * dx)) * g;
    }
    out.val = K;
    out.err = fabs(K - G);
    out.abs = A;
}

// Adaptive integral of curve c (times 4 pi): dyadic panels (depth d, index k);
// a panel is accepted when its error estimate is below tol4pi * 2^-d or below
// 16 units of rounding of its rounding scale, else halved, within the depth,
// stack and panel budgets (exceeding one clears ok).  Adds the panels
// evaluated to *count.
__device__ double curve_integral(const PanelNode *__restrict__ tree, int tree_depth, const double *__restrict__ P,
                                 D3 q, float qx, float qy, float qz, double tol4pi, int max_panels, bool fp64,
                                 bool &ok, unsigned &count) {
    unsigned long long sk[kStackQuad];
    unsigned char sd[kStackQuad];
    int top = 0, panels = 0;
    sk[0] = 0;
    sd[top++] = 0;
    double total = 0.0;
    while (top > 0) {
        --top;
        const unsigned long long k = sk[top];
        const int d = sd[top];
        ++panels;
        const double h = ldexp(1.0, -d);
        PanelResult pr;
        double eps;
        if (!fp64 && d <= tree_depth && panel_f32(tree[((1ull << d) - 1) + k], qx, qy, qz, pr)) {
            eps = 16.0 * 0x1p-24;
        } else {
            panel_f64(P, q, (double)k * h, (double)(k + 1) * h, pr);
            eps = 16.0 * DBL_EPSILON;
        }
        const bool conv = pr.err <= fmax(tol4pi * h, eps * pr.abs);
        if (conv || d >= kMaxQuadDepth || top + 2 > kStackQuad || panels >= max_panels) {
            if (!conv) ok = false;
            total += pr.val;
            continue;
        }
        sk[top] = 2 * k + 1;
        sd[top++] = (unsigned char)(d + 1);
        sk[top] = 2 * k;
        sd[top++] = (unsigned char)(d + 1);
    }
    count += panels;
    return total;
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

// w = chi + (boundary integral) of n points: one warp per point, lanes over
// the boundary curves.
template <class Points>
__global__ void __launch_bounds__(32 * kWarps) k_param_boundary(Points pts, int64_t n,
                                                                const PanelNode *__restrict__ tree, int tree_nodes,
                                                                int tree_depth, const double *__restrict__ curves,
                                                                int nc,
                                                                double tol4pi, int max_panels, int fp64,
                                                                const int32_t *__restrict__ chi,
                                                                float *__restrict__ w,
                                                                unsigned long long *__restrict__ status) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
    if (i >= n) return;
    float qx, qy, qz;
    pts.get(i, qx, qy, qz);
    const D3 p = d3(qx, qy, qz);
    double acc = 0.0;
    bool ok = true;
    unsigned count = 0;
    for (int k = lane; k < nc; k += 32)
        acc += curve_integral(tree + (size_t)k * tree_nodes, tree_depth, curves + 12 * k, p, qx, qy, qz, tol4pi,
                              max_panels, fp64 != 0, ok, count);
    acc = warp_sum(acc);
    const int panels = warp_sum((int)count);
    const bool all_ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        w[i] = (float)((double)chi[i] + acc * kInv4PiD);
        if (!all_ok) atomicAdd(&status[1], 1ull);
        atomicAdd(&status[2], (unsigned long long)panels);
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
    double *pbox = nullptr;      // [np][5]: x range, y range, top of the net
    double *curves = nullptr;    // [nc][4][3]
    PanelNode *tree = nullptr;   // [nc][tree_nodes]
    int tree_depth = 0, tree_nodes = 0;
    unsigned long long *status = nullptr;   // [0]: subdivision budget hits, [1]: unconverged integrals,
                                            // [2]: quadrature panels evaluated
    double flat = 0.0;           // bilinear tolerance (absolute)
    double same = 0.0;           // edge hits of one ray closer than this (same sign) are one crossing
    double zlo = 0.0;            // below every control point: start of the grid rays
    std::vector<float> h_curves;
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
            nd.chi = make_float4(hx, hy, hz, 0.f);
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

bool g_tables_ready[64] = {};

gwn_status upload_tables(int device) {
    if (device >= 0 && device < 64 && g_tables_ready[device]) return GWN_OK;
    const GKTables t = make_gk_tables();
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_gk, &t, sizeof(t)));
    if (device >= 0 && device < 64) g_tables_ready[device] = true;
    return GWN_OK;
}

// Device copy of n host-or-device floats (stream-ordered scratch).
gwn_status copy_coords(const float *src, int32_t n, float **dst, cudaStream_t s) {
    GWN_CUDA_TRY(cudaMallocAsync(dst, sizeof(float) * (size_t)std::max(n, 1), s));
    GWN_CUDA_TRY(cudaMemcpyAsync(*dst, src, sizeof(float) * (size_t)n, cudaMemcpyDefault, s));
    return GWN_OK;
}

gwn_status check_device_ptrs(std::initializer_list<const void *> ptrs, const char *what) {
    for (const void *p : ptrs) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return set_error(GWN_ERR_INVALID_ARG, std::string(what) + " takes device pointers for its outputs");
        }
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
    g->zlo = np > 0 ? lo[2] - 1.0 - ext : 0.0;
    // panel trees: depth <= 10, at most 1 GiB in all
    int depth = 10;
    while (depth > 0 && (double)g->nc * (double)((2 << depth) - 1) * sizeof(PanelNode) > (double)(1ull << 30)) --depth;
    g->tree_depth = depth;
    g->tree_nodes = (2 << depth) - 1;
    std::vector<PanelNode> tree((size_t)g->nc * g->tree_nodes);
    for (int k = 0; k < g->nc; ++k) build_tree(dc.data() + 12 * (size_t)k, depth, tree.data() + (size_t)k * g->tree_nodes);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&g->status, sizeof(unsigned long long) * 3)) != cudaSuccess ||
        (np > 0 && ((e = cudaMalloc(&g->patches, sizeof(double) * dp.size())) != cudaSuccess ||
                    (e = cudaMalloc(&g->pbox, sizeof(double) * box.size())) != cudaSuccess)) ||
        (g->nc > 0 && ((e = cudaMalloc(&g->curves, sizeof(double) * dc.size())) != cudaSuccess ||
                       (e = cudaMalloc(&g->tree, sizeof(PanelNode) * tree.size())) != cudaSuccess))) {
        gwn_param_destroy(g);
        return set_error(GWN_ERR_OOM, cudaGetErrorString(e));
    }
    cudaMemset(g->status, 0, sizeof(unsigned long long) * 3);
    if (np > 0) {
        cudaMemcpy(g->patches, dp.data(), sizeof(double) * dp.size(), cudaMemcpyHostToDevice);
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
    for (void *p : {(void *)g->patches, (void *)g->pbox, (void *)g->curves, (void *)g->tree, (void *)g->status})
        if (p) cudaFree(p);
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
    if (gwn_status st = check_device_ptrs({q, w, chi_or_null}, "gwn_param_query")) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *chi = chi_or_null;
    if (!chi) GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, s));
    {
        ProfScope prof("param_chi", s);
        k_param_chi<<<grid_for(n, kWarps), 32 * kWarps, 0, s>>>(q, n, g->patches, g->np, g->pbox, g->flat, g->same,
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
    if (gwn_status st = check_device_ptrs({w, chi_or_null}, "gwn_param_query_grid")) return st;
    {
        std::vector<float> hz(nz);
        GWN_CUDA_TRY(cudaMemcpy(hz.data(), z, sizeof(float) * nz, cudaMemcpyDefault));
        for (int k = 0; k < nz; ++k)
            if (!std::isfinite(hz[k]) || (k > 0 && hz[k] < hz[k - 1]))
                return set_error(GWN_ERR_INVALID_ARG, "z must be finite and non-decreasing");
    }
    cudaStream_t s = (cudaStream_t)stream;
    float *dx = nullptr, *dy = nullptr, *dz = nullptr;
    int32_t *chi = chi_or_null;
    gwn_status st = GWN_OK;
    if ((st = copy_coords(x, nx, &dx, s)) || (st = copy_coords(y, ny, &dy, s)) || (st = copy_coords(z, nz, &dz, s)))
        return st;
    if (!chi) GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, s));
    {
        ProfScope prof("param_grid_chi", s);
        const int64_t cols = (int64_t)nx * ny;
        k_param_grid_chi<<<grid_for(cols, kWarps), 32 * kWarps, 0, s>>>(dx, nx, dy, ny, dz, nz, g->zlo, g->patches,
                                                                        g->np, g->pbox, g->flat, g->same,
                                                                        g->cfg.max_nodes, chi, g->status);
    }
    launch_boundary(g, GridPoints{dx, dy, dz, nx, ny}, n, chi, w, s);
    if (!chi_or_null) cudaFreeAsync(chi, s);
    cudaFreeAsync(dx, s);
    cudaFreeAsync(dy, s);
    cudaFreeAsync(dz, s);
    GWN_LAUNCH_CHECK("parametric grid query");
    return GWN_OK;
}

gwn_status gwn_param_status(const gwn_param *g, uint64_t *budget_hits, uint64_t *unconverged, uint64_t *panels,
                            int reset) {
    clear_error();
    if (!g) return set_error(GWN_ERR_INVALID_ARG, "surface is NULL");
    unsigned long long h[3];
    GWN_CUDA_TRY(cudaMemcpy(h, g->status, sizeof(h), cudaMemcpyDeviceToHost));
    if (reset) GWN_CUDA_TRY(cudaMemset(g->status, 0, sizeof(h)));
    if (budget_hits) *budget_hits = h[0];
    if (unconverged) *unconverged = h[1];
    if (panels) *panels = h[2];
    return GWN_OK;
}

}  // extern "C"
