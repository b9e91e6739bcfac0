// Set-up of the fixed-point frame of a mesh built with quantize_bits = 30
// (Supp. S2.1): the snapping centre and exponent from the vertices' bounding
// box, the snapped leaf triangles, and the frame itself in the mesh's device
// status block (after the counter slots), where the kernels read it.
#include <cmath>
#include <cstring>

#include "gwn_internal.cuh"
#include "quant.cuh"

namespace gwn {

namespace {

__device__ __forceinline__ int okey(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

// bounding box of the vertices as order-preserving integer keys (min xyz, max xyz)
__global__ void k_vertex_box(const float4 *__restrict__ V, int64_t nv, int *__restrict__ box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < nv;
    const float4 v = ok ? V[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float c[3] = {v.x, v.y, v.z};
    for (int d = 0; d < 3; ++d) {
        int lo = ok ? okey(c[d]) : 0x7fffffff, hi = ok ? okey(c[d]) : (int)0x80000000;
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&box[d], lo);
            atomicMax(&box[3 + d], hi);
        }
    }
}

__global__ void k_snap_leaves(const float4 *__restrict__ tri, int64_t n, QFrame f, int4 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = tri[i];
    out[i] = make_int4((int)qcoord(v.x, f.cx, f.scale), (int)qcoord(v.y, f.cy, f.scale),
                       (int)qcoord(v.z, f.cz, f.scale), 0);
}

float from_okey(int k) {
    const int i = k >= 0 ? k : k ^ 0x7fffffff;
    float f;
    std::memcpy(&f, &i, 4);
    return f;
}

}  // namespace

// Snapping exponent: the smallest e with max |v - c| 2^-e <= 2^29, from
// frexp (h = m 2^k, 1/2 <= m < 1, so h < 2^k and e = k - 29 suffices).
int quant_exponent(double half_extent) {
    if (!(half_extent > 0.0)) return 0;
    int k = 0;
    std::frexp(half_extent, &k);
    return k - 29;
}

gwn_status setup_quant(gwn_mesh *m, cudaStream_t s) {
    QFrame f{};
    if (m->leaf_q) {
        cudaFree(m->leaf_q);
        m->leaf_q = nullptr;
    }
    if (m->cfg.quantize_bits == 30 && m->nt > 0) {
        int *box = nullptr;
        GWN_CUDA_TRY(cudaMallocAsync(&box, sizeof(int) * 6, s));
        const int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
        GWN_CUDA_TRY(cudaMemcpyAsync(box, init, sizeof(init), cudaMemcpyHostToDevice, s));
        k_vertex_box<<<grid_for(m->nv, 256), 256, 0, s>>>(m->V, m->nv, box);
        int h[6];
        GWN_CUDA_TRY(cudaMemcpyAsync(h, box, sizeof(h), cudaMemcpyDeviceToHost, s));
        cudaFreeAsync(box, s);
        GWN_CUDA_TRY(cudaStreamSynchronize(s));
        double c[3], half = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double lo = from_okey(h[d]), hi = from_okey(h[3 + d]);
            c[d] = 0.5 * (lo + hi);
            half = std::fmax(half, std::fmax(hi - c[d], c[d] - lo));
        }
        const int e = quant_exponent(half);
        f.bits = 30;
        f.cx = c[0];
        f.cy = c[1];
        f.cz = c[2];
        f.scale = std::ldexp(1.0, -e);
        f.pad = (float)std::ldexp(1.0, e);
        int4 *lq = nullptr;
        GWN_CUDA_TRY(cudaMalloc(&lq, sizeof(int4) * 3 * m->nt));
        k_snap_leaves<<<grid_for(3 * m->nt, 256), 256, 0, s>>>(m->leaf_tri, 3 * m->nt, f, lq);
        m->leaf_q = lq;
        f.leaf_q = lq;
    }
    GWN_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<unsigned char *>(m->counters) + sizeof(unsigned long long) * CNT_SLOTS,
                                 &f, sizeof(f), cudaMemcpyHostToDevice, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    GWN_LAUNCH_CHECK("fixed-point frame");
    return GWN_OK;
}

}  // namespace gwn
