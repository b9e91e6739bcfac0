// Query kernels: crossing number (BVH traversal), boundary-curve sum, combine /
// classify with FP64 re-evaluation, and the direct solid-angle sum.
//
// Antipodal evaluation (Eq. 4, Algorithm 1 with x0 = +z, x1 = -z):
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
#include "gwn_internal.cuh"
#include "predicates.cuh"
#include "atan_poly.cuh"

namespace gwn {

namespace {

constexpr double kInv2Pi = 0.15915494309189533577;
constexpr float kPiF = 3.14159265358979f;

// ----------------------------------------------------------- traversal ----

__global__ void __launch_bounds__(256) k_chi(const float *__restrict__ q, int64_t n,
                                             const BvhNode *__restrict__ nodes, int64_t nnodes,
                                             const float4 *__restrict__ tri, int32_t *__restrict__ chi,
                                             unsigned long long *__restrict__ counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float3 p = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    int c = 0;
    int node = nnodes > 0 ? 0 : -1;
    int64_t budget = nnodes + 1;   // depth-first order visits each node at most once
    while (node >= 0) {
        if (--budget < 0 || node >= nnodes) {   // corrupt tree: report, never loop or read out of range
            atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
            c = INT32_MIN;
            break;
        }
        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
        const float4 b0 = __ldg(np);
        const float4 b1 = __ldg(np + 1);
        const int child = __float_as_int(b1.y), skip = __float_as_int(b1.z), leaf = __float_as_int(b1.w);
        const bool hit = p.x >= b0.x && p.x <= b0.y && p.y >= b0.z && p.y <= b0.w && p.z <= b1.x;
        if (hit && leaf) {
            if ((unsigned)child >= (unsigned)((nnodes + 1) / 2)) {
                atomicOr(&counters[CNT_ERROR], (unsigned long long)ERR_TRAVERSAL_LIMIT);
                c = INT32_MIN;
                break;
            }
            const float4 a = __ldg(tri + 3 * child), bb = __ldg(tri + 3 * child + 1), cc = __ldg(tri + 3 * child + 2);
            c += tri_crossing(p, make_float3(a.x, a.y, a.z), make_float3(bb.x, bb.y, bb.z),
                              make_float3(cc.x, cc.y, cc.z), &counters[CNT_EXACT_EDGE], &counters[CNT_EXACT_PLANE]);
            node = skip;
        } else {
            node = hit ? child : skip;
        }
    }
    chi[i] = c;
}

// ------------------------------------------------------ boundary terms ----

// atan2 for the hot loops: octant reduction to t = min/max in [0, 1], then
// atan(t) = t P(t^2) with the minimax polynomial of atan_poly.cuh (fitted by
// fit_atan.py), then the octant is undone.  Branch-free.  Callers never pass
// (0, 0).
__device__ __forceinline__ float fast_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = __fdividef(mn, mx);
    const float s = t * t;
    float r = gwn_atan_poly(s) * t;
    r = ay > ax ? 1.57079632679489662f - r : r;
    r = x < 0.f ? 3.14159265358979324f - r : r;
    return copysignf(r, y);
}

// Unit vector from the query to a boundary point, kept as (A_x, A_y, H) with
// H = 1 - A_z computed without cancellation: (A_x^2 + A_y^2) / (1 + A_z) when
// A_z > 0.  The point coincident with the query gives (0, 0, 0).
struct PointRel {
    float ax, ay, h;
};

__device__ __forceinline__ PointRel point_rel(float4 P, float qx, float qy, float qz) {
    const float dx = P.x - qx, dy = P.y - qy, dz = P.z - qz;
    const float s = fmaf(dx, dx, dy * dy);
    const float r2 = fmaf(dz, dz, s);
    const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    PointRel r;
    r.ax = dx * inv;
    r.ay = dy * inv;
    const float az = dz * inv;
    const float g = 1.0f + fabsf(az);
    r.h = az > 0.f ? __fdividef(s * inv * inv, g) : g;
    return r;
}

// Van Oosterom-Strackee numerator and denominator of Area(A, B, x1) / 2 with
// x1 = (0, 0, -1):  n = A.(B x x1) = A_y B_x - A_x B_y,
//                   d = 1 + A.B + A.x1 + B.x1 = H_a H_b + A_x B_x + A_y B_y.
__device__ __forceinline__ void edge_nd(const PointRel &A, const PointRel &B, float &n, float &d) {
    n = fmaf(A.ay, B.ax, -(A.ax * B.ay));
    d = fmaf(A.h, B.h, fmaf(A.ax, B.ax, A.ay * B.ay));
}

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
    const int s = edge_sos(qx, qy, Pa.x, Pa.y, Pb.x, Pb.y, nullptr);   // n ~ -classification
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

__device__ __forceinline__ float edge_term_nd(float n, float d, float4 Pa, float4 Pb, float qx, float qy, float qz,
                                              unsigned long long *counters) {
    const PointRel A = point_rel(Pa, qx, qy, qz), B = point_rel(Pb, qx, qy, qz);
    return edge_term(n, d, A, B, Pa, Pb, qx, qy, qz, counters);
}

// One thread holds KQ queries (strided by the block size); the block streams the
// chained boundary points through shared memory.  Point j carries flag w = 1
// when an edge runs from it to point j+1.  Consecutive edges are taken in pairs:
// when both denominators are positive each angle lies in (-pi/2, pi/2), so the
// pair's sum lies in (-pi, pi) and equals the argument of the product
// (d1 + i n1)(d2 + i n2), one atan2 for two edges.  Otherwise both terms are
// taken one by one.  Terms are summed in FP32 per tile and folded into an FP64
// accumulator per query once per tile.
template <int KQ>
__global__ void __launch_bounds__(256) k_boundary_sum(const float *__restrict__ q, int64_t n,
                                                      const float4 *__restrict__ pts, int64_t npts, int tile,
                                                      const int32_t *__restrict__ chi, float *__restrict__ w,
                                                      uint8_t *__restrict__ label, int classify, float margin,
                                                      int32_t *__restrict__ list,
                                                      unsigned long long *__restrict__ list_len,
                                                      unsigned long long *__restrict__ counters) {
    extern __shared__ float4 s_pts[];
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * KQ + threadIdx.x;
    float qx[KQ], qy[KQ], qz[KQ];
    PointRel prev[KQ];
    float pn[KQ], pd[KQ];
    float part[KQ];
    double acc[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        const bool ok = idx < n;
        qx[k] = ok ? q[3 * idx] : __int_as_float(0x7fc00000);
        qy[k] = ok ? q[3 * idx + 1] : __int_as_float(0x7fc00000);
        qz[k] = ok ? q[3 * idx + 2] : __int_as_float(0x7fc00000);
        prev[k] = PointRel{0.f, 0.f, 0.f};
        pn[k] = 0.f;
        pd[k] = 0.f;
        part[k] = 0.f;
        acc[k] = 0.0;
    }
    bool prev_edge = false, pending = false;
    float4 prevP = make_float4(0.f, 0.f, 0.f, 0.f), pendA = prevP, pendB = prevP;
    for (int64_t t0 = 0; t0 < npts; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, npts - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) s_pts[i] = __ldg(pts + t0 + i);
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float4 P = s_pts[j];
            if (prev_edge) {
                if (pending) {
#pragma unroll
                    for (int k = 0; k < KQ; ++k) {
                        const PointRel cur = point_rel(P, qx[k], qy[k], qz[k]);
                        float n1, d1;
                        edge_nd(prev[k], cur, n1, d1);
                        if (pd[k] > 0.f && d1 > 0.f) {
                            part[k] += fast_atan2(fmaf(pn[k], d1, n1 * pd[k]), fmaf(pd[k], d1, -(pn[k] * n1)));
                        } else {
                            part[k] += edge_term_nd(pn[k], pd[k], pendA, pendB, qx[k], qy[k], qz[k], counters) +
                                       edge_term(n1, d1, prev[k], cur, prevP, P, qx[k], qy[k], qz[k], counters);
                        }
                        prev[k] = cur;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < KQ; ++k) {
                        const PointRel cur = point_rel(P, qx[k], qy[k], qz[k]);
                        edge_nd(prev[k], cur, pn[k], pd[k]);
                        prev[k] = cur;
                    }
                    pendA = prevP;
                    pendB = P;
                }
                pending = !pending;
            } else {
#pragma unroll
                for (int k = 0; k < KQ; ++k) prev[k] = point_rel(P, qx[k], qy[k], qz[k]);
            }
            prev_edge = P.w != 0.f;
            prevP = P;
        }
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
            acc[k] += (double)part[k];
            part[k] = 0.f;
        }
    }
    if (pending) {
#pragma unroll
        for (int k = 0; k < KQ; ++k)
            acc[k] += (double)edge_term_nd(pn[k], pd[k], pendA, pendB, qx[k], qy[k], qz[k], counters);
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        if (idx >= n) continue;
        const double wv = (double)chi[idx] + acc[k] * kInv2Pi;
        w[idx] = (float)wv;
        if (classify) {
            label[idx] = wv > 0.5 ? 1 : 0;
            if (fabs(wv - 0.5) <= (double)margin) {
                unsigned long long slot = atomicAdd(list_len, 1ull);
                list[slot] = (int32_t)idx;
            }
        }
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

__device__ double edge_angle64(float4 Pa, float4 Pb, float qx, float qy, float qz) {
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
        const int s = edge_sos(qx, qy, Pa.x, Pa.y, Pb.x, Pb.y, nullptr);
        return atan2(s > 0 ? -fabs(n) : fabs(n), d);
    }
    return atan2(n, d);
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
        double acc = 0.0;
        for (int64_t j = threadIdx.x; j + 1 < npts; j += blockDim.x) {
            const float4 P = pts[j];
            if (P.w != 0.f) acc += edge_angle64(P, pts[j + 1], qx, qy, qz);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double wv = (double)chi[idx] + red[0] * kInv2Pi;
            w[idx] = (float)wv;
            label[idx] = wv > 0.5 ? 1 : 0;
            atomicAdd(&counters[CNT_FP64], 1ull);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- direct ----

// Direct sum (Eq. 2): per triangle 2 atan2(det[a b c], l_a l_b l_c + (a.b) l_c
// + (a.c) l_b + (b.c) l_a) with a, b, c the vertices relative to q.  Triangles
// are staged through shared memory (9 floats each); each thread holds KQ queries.
template <int KQ>
__global__ void __launch_bounds__(256) k_direct(const float *__restrict__ q, int64_t n, const float *__restrict__ tri9,
                                                int64_t nt, int tile, float *__restrict__ w) {
    extern __shared__ float s_tri[];
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * KQ + threadIdx.x;
    float qx[KQ], qy[KQ], qz[KQ], part[KQ];
    double acc[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        const bool ok = idx < n;
        qx[k] = ok ? q[3 * idx] : 0.f;
        qy[k] = ok ? q[3 * idx + 1] : 0.f;
        qz[k] = ok ? q[3 * idx + 2] : 0.f;
        part[k] = 0.f;
        acc[k] = 0.0;
    }
    for (int64_t t0 = 0; t0 < nt; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, nt - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < 9 * cnt; i += blockDim.x) s_tri[i] = __ldg(tri9 + 9 * t0 + i);
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float *T = s_tri + 9 * j;
            const float x0 = T[0], y0 = T[1], z0 = T[2], x1 = T[3], y1 = T[4], z1 = T[5];
            const float x2 = T[6], y2 = T[7], z2 = T[8];
#pragma unroll
            for (int k = 0; k < KQ; ++k) {
                const float ax = x0 - qx[k], ay = y0 - qy[k], az = z0 - qz[k];
                const float bx = x1 - qx[k], by = y1 - qy[k], bz = z1 - qz[k];
                const float cx = x2 - qx[k], cy = y2 - qy[k], cz = z2 - qz[k];
                const float la2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                const float lb2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
                const float lc2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                const float la = la2 * rsqrtf(la2), lb = lb2 * rsqrtf(lb2), lc = lc2 * rsqrtf(lc2);
                const float det = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
                const float ab = fmaf(ax, bx, fmaf(ay, by, az * bz));
                const float ac = fmaf(ax, cx, fmaf(ay, cy, az * cz));
                const float bc = fmaf(bx, cx, fmaf(by, cy, bz * cz));
                const float den = fmaf(ab, lc, fmaf(ac, lb, fmaf(bc, la, la * lb * lc)));
                part[k] += fast_atan2(det, den);
            }
        }
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
            acc[k] += (double)part[k];
            part[k] = 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        if (idx < n) w[idx] = (float)(acc[k] * kInv2Pi);
    }
}

}  // namespace

gwn_status launch_chi(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi, cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    ProfScope prof("chi_traversal", s);
    k_chi<<<grid_for(n, 256), 256, 0, s>>>(q, n, m->nodes, m->nnodes, m->leaf_tri, chi, m->counters);
    GWN_LAUNCH_CHECK("k_chi");
    return GWN_OK;
}

template <int KQ>
static void launch_bsum_kq(const gwn_mesh *m, const float *q, int64_t n, const int32_t *chi, float *w,
                           uint8_t *label, bool classify, int32_t *list, unsigned long long *list_len,
                           cudaStream_t s) {
    const int tile = m->cfg.boundary_tile > 0 ? m->cfg.boundary_tile : 512;
    const size_t smem = sizeof(float4) * tile;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_boundary_sum<KQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t per_block = 256 * KQ;
    k_boundary_sum<KQ><<<grid_for(n, (int)per_block), 256, smem, s>>>(
        q, n, m->bpts, m->npts, tile, chi, w, label, classify ? 1 : 0,
        m->cfg.classify_margin > 0.f ? m->cfg.classify_margin : 1e-4f, list, list_len, m->counters);
}

gwn_status launch_boundary_sum_list(const gwn_mesh *m, const float *q, int64_t n, const int32_t *chi, float *w,
                                    uint8_t *label, bool classify, int32_t *list, unsigned long long *list_len,
                                    cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    const int kq = m->cfg.queries_per_thread > 0 ? m->cfg.queries_per_thread : 4;
    ProfScope prof("boundary_sum", s);
    switch (kq) {
        case 1: launch_bsum_kq<1>(m, q, n, chi, w, label, classify, list, list_len, s); break;
        case 2: launch_bsum_kq<2>(m, q, n, chi, w, label, classify, list, list_len, s); break;
        case 8: launch_bsum_kq<8>(m, q, n, chi, w, label, classify, list, list_len, s); break;
        default: launch_bsum_kq<4>(m, q, n, chi, w, label, classify, list, list_len, s); break;
    }
    GWN_LAUNCH_CHECK("k_boundary_sum");
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
    constexpr int KQ = 4;
    const int tile = 256;
    ProfScope prof("direct_sum", s);
    k_direct<KQ><<<grid_for(n, 256 * KQ), 256, sizeof(float) * 9 * tile, s>>>(q, n, m->tri9, m->nt, tile, w);
    GWN_LAUNCH_CHECK("k_direct");
    return GWN_OK;
}

}  // namespace gwn
