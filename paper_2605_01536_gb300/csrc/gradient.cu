// Gradient of the winding number with respect to the query point (Supp. S4,
// Algorithm 3).  The crossing count is piecewise constant, so only the boundary
// terms carry a gradient:
//   grad w = (1/4pi) sum_{(a,b) in dM} (c_n g_n + c_d g_d),
//   c_n = 2 d / (n^2 + d^2),  c_d = -2 n / (n^2 + d^2),
// with n, d the (unnormalised) van Oosterom-Strackee pair of the edge seen from
// the query and g_n = dn/dp, g_d = dd/dp.  With x1 = -z and r0 = a - p,
// r1 = b - p, l = |r|, v = r / l, h = l - r_z (= l (1 + x1.v)):
//   n   = r0_y r1_x - r0_x r1_y
//   d   = h0 h1 + r0_x r1_x + r0_y r1_y
//   g_n = (b_y - a_y, a_x - b_x, 0)                 (-(r1 x x1 + x1 x r0))
//   g_d = (l0 + l1) z - (r0 + r1 + h1 v0 + h0 v1)    (-(t1 + t2) of Algorithm 3)
// h is computed as (r_x^2 + r_y^2) / (l + |r_z|) + (|r_z| - r_z), which avoids the
// cancellation of l - r_z for a point nearly straight above the query.  A term
// whose n^2 + d^2 underflows (the query on the boundary curve, or a boundary
// point exactly straight above or below it, where the term is singular) is
// skipped and counted.
//
// Layout and schedule follow the boundary-sum kernel: each thread holds 2 KP
// queries as float2 pairs (one Blackwell paired instruction per step for two
// queries), the chained boundary points stream through shared memory in tiles,
// FP32 partial sums are flushed into FP64 accumulators (shared memory) every
// 64 edges, and small query batches split the boundary into chunks whose FP64
// partials are added in chunk order.
#include <algorithm>

#include "gwn_internal.cuh"
#include "fp32x2.cuh"

namespace gwn {

namespace {

constexpr double kInv4Pi = 0.079577471545947667884;
constexpr int kGradThreads = 128;
constexpr int kFlushEdges = 64;
constexpr float kMinModulus2 = 1e-30f;

// Per-point data of two queries: r = P - q, l = |r|, v = r / l, h = l - r_z.
struct GradPoint2 {
    float2 rx, ry, rz, l, h, vx, vy, vz;
};

__device__ __forceinline__ GradPoint2 grad_point2(float4 P, float2 nqx, float2 nqy, float2 nqz) {
    GradPoint2 g;
    g.rx = add2(bc2(P.x), nqx);
    g.ry = add2(bc2(P.y), nqy);
    g.rz = add2(bc2(P.z), nqz);
    const float2 s = fma2(g.rx, g.rx, mul2(g.ry, g.ry));
    const float2 r2 = add2(fma2(g.rz, g.rz, s), bc2(1e-37f));   // > 0 for a coincident point
    const float2 il = make_float2(sfu_rsqrt(r2.x), sfu_rsqrt(r2.y));
    g.l = mul2(r2, il);
    g.vx = mul2(g.rx, il);
    g.vy = mul2(g.ry, il);
    g.vz = mul2(g.rz, il);
    const float2 az = make_float2(fabsf(g.rz.x), fabsf(g.rz.y));
    const float2 den = add2(g.l, az);
    g.h = fma2(s, make_float2(sfu_rcp(den.x), sfu_rcp(den.y)), add2(az, neg2(g.rz)));
    return g;
}

// Adds the edge term (point A -> point B) of two queries to (gx, gy, gz).
// ex, ey: the query-independent edge vector a - b.  skipped counts lanes whose
// term was dropped as singular.
__device__ __forceinline__ void grad_edge2(const GradPoint2 &A, const GradPoint2 &B, float ex, float ey, float2 &gx,
                                           float2 &gy, float2 &gz, unsigned &skipped) {
    const float2 n = fma2(A.ry, B.rx, neg2(mul2(A.rx, B.ry)));
    const float2 d = fma2(A.h, B.h, fma2(A.rx, B.rx, mul2(A.ry, B.ry)));
    const float2 m2 = fma2(n, n, mul2(d, d));
    const bool okx = m2.x > kMinModulus2, oky = m2.y > kMinModulus2;
    skipped += (okx ? 0u : 1u) + (oky ? 0u : 1u);
    const float2 t = make_float2(okx ? 2.f * sfu_rcp(m2.x) : 0.f, oky ? 2.f * sfu_rcp(m2.y) : 0.f);
    const float2 cn = mul2(d, t);
    const float2 cd = neg2(mul2(n, t));
    // u = r0 + r1 + h1 v0 + h0 v1, so that g_d = (l0 + l1) z - u
    const float2 ux = fma2(A.h, B.vx, fma2(B.h, A.vx, add2(A.rx, B.rx)));
    const float2 uy = fma2(A.h, B.vy, fma2(B.h, A.vy, add2(A.ry, B.ry)));
    const float2 uz = fma2(A.h, B.vz, fma2(B.h, A.vz, add2(A.rz, B.rz)));
    // c_n g_n + c_d g_d with g_n = (-e_y, e_x, 0)
    gx = add2(gx, neg2(fma2(cn, bc2(ey), mul2(cd, ux))));
    gy = fma2(cn, bc2(ex), add2(gy, neg2(mul2(cd, uy))));
    gz = fma2(cd, add2(add2(A.l, B.l), neg2(uz)), gz);
}

template <int KP>
__global__ void __launch_bounds__(kGradThreads) k_gradient(const float *__restrict__ q, int64_t n,
                                                           const float4 *__restrict__ pts, int64_t npts, int tile,
                                                           int64_t chunk_len, double *__restrict__ partial,
                                                           float *__restrict__ grad,
                                                           unsigned long long *__restrict__ counters) {
    extern __shared__ float4 s_pts[];   // tile + 1 points, then 3 x 2 KP x blockDim doubles
    double *s_acc = reinterpret_cast<double *>(s_pts + tile + 1);
    constexpr int KQ = 2 * KP;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * KQ + threadIdx.x;
    const int64_t e_begin = (int64_t)blockIdx.y * chunk_len;
    const int64_t e_end = min(npts - 1, e_begin + chunk_len);   // edge start points
    float2 nqx[KP], nqy[KP], nqz[KP];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        const bool ok = idx < n;
        // queries past n sit far away (their n^2 + d^2 overflows to +inf, so they are
        // never counted as singular); their results are discarded
        const float x = ok ? -q[3 * idx] : 1e15f, y = ok ? -q[3 * idx + 1] : 1e15f, z = ok ? -q[3 * idx + 2] : 1e15f;
        if (k & 1) { nqx[k >> 1].y = x; nqy[k >> 1].y = y; nqz[k >> 1].y = z; }
        else       { nqx[k >> 1].x = x; nqy[k >> 1].x = y; nqz[k >> 1].x = z; }
    }
#pragma unroll
    for (int k = 0; k < 3 * KQ; ++k) s_acc[k * blockDim.x + threadIdx.x] = 0.0;
    float2 gx[KP], gy[KP], gz[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) gx[k] = gy[k] = gz[k] = bc2(0.f);
    unsigned skipped = 0;
    int since_flush = 0;
    auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            double *a = s_acc + (6 * k) * blockDim.x + threadIdx.x;
            a[0 * blockDim.x] += (double)gx[k].x;
            a[1 * blockDim.x] += (double)gy[k].x;
            a[2 * blockDim.x] += (double)gz[k].x;
            a[3 * blockDim.x] += (double)gx[k].y;
            a[4 * blockDim.x] += (double)gy[k].y;
            a[5 * blockDim.x] += (double)gz[k].y;
            gx[k] = gy[k] = gz[k] = bc2(0.f);
        }
        since_flush = 0;
    };
    for (int64_t t0 = e_begin; t0 < e_end; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, e_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i <= cnt; i += blockDim.x) s_pts[i] = __ldg(pts + t0 + i);
        __syncthreads();
        GradPoint2 ga[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) ga[k] = grad_point2(s_pts[0], nqx[k], nqy[k], nqz[k]);
        for (int j = 0; j < cnt; ++j) {
            const float4 Pa = s_pts[j], Pb = s_pts[j + 1];
            GradPoint2 gb[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) gb[k] = grad_point2(Pb, nqx[k], nqy[k], nqz[k]);
            if (Pa.w != 0.f) {
                const float ex = Pa.x - Pb.x, ey = Pa.y - Pb.y;
#pragma unroll
                for (int k = 0; k < KP; ++k) grad_edge2(ga[k], gb[k], ex, ey, gx[k], gy[k], gz[k], skipped);
                if (++since_flush == kFlushEdges) flush();
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) ga[k] = gb[k];
        }
    }
    flush();
    if (skipped) atomicAdd(&counters[CNT_GRAD_SKIPPED], (unsigned long long)skipped);
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int64_t idx = base + (int64_t)k * blockDim.x;
        if (idx >= n) continue;
        const int kp = k >> 1, lane = k & 1;
        const double *a = s_acc + (6 * kp + 3 * lane) * blockDim.x + threadIdx.x;
        for (int c = 0; c < 3; ++c) {
            const double v = a[c * blockDim.x];
            if (partial) partial[((int64_t)blockIdx.y * n + idx) * 3 + c] = v;
            else grad[3 * idx + c] = (float)(v * kInv4Pi);
        }
    }
}

__global__ void k_gradient_combine(const double *__restrict__ partial, int64_t n, int chunks, float *__restrict__ grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partial[(int64_t)c * 3 * n + i];
    grad[i] = (float)(s * kInv4Pi);
}

}  // namespace

gwn_status launch_gradient(const gwn_mesh *m, const float *q, int64_t n, float *grad, cudaStream_t s) {
    if (n <= 0) return GWN_OK;
    const int64_t nedge_pts = m->npts > 0 ? m->npts - 1 : 0;
    if (nedge_pts == 0) {   // no boundary: the gradient vanishes almost everywhere
        GWN_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * 3 * n, s));
        return GWN_OK;
    }
    constexpr int KP = 2;
    const int tile = m->cfg.boundary_tile > 0 ? m->cfg.boundary_tile : 512;
    const size_t smem = sizeof(float4) * (tile + 1) + sizeof(double) * 3 * 2 * KP * kGradThreads;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_gradient<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t per_block = kGradThreads * 2 * KP;
    const int64_t qblocks = (n + per_block - 1) / per_block;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t chunks = (8 * (int64_t)(sms > 0 ? sms : 148) + qblocks - 1) / qblocks;
    chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (nedge_pts + 2 * tile - 1) / (2 * tile)));
    chunks = std::min<int64_t>(chunks, 65535);
    const int64_t chunk_len = chunks > 1 ? (nedge_pts + chunks - 1) / chunks : nedge_pts;
    double *partial = nullptr;
    if (chunks > 1) GWN_CUDA_TRY(cudaMallocAsync(&partial, sizeof(double) * 3 * chunks * n, s));
    {
        ProfScope prof("gradient", s);
        dim3 grid((unsigned)qblocks, (unsigned)chunks);
        k_gradient<KP><<<grid, kGradThreads, smem, s>>>(q, n, m->bpts, m->npts, tile, chunk_len, partial, grad,
                                                        m->counters);
        if (partial) k_gradient_combine<<<grid_for(3 * n, 256), 256, 0, s>>>(partial, n, (int)chunks, grad);
    }
    if (partial) cudaFreeAsync(partial, s);
    GWN_LAUNCH_CHECK("k_gradient");
    return GWN_OK;
}

}  // namespace gwn
