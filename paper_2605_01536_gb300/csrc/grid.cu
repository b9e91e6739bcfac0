// Queries on a rectilinear grid with ray reuse (Supp. S3): every cell of one
// (x, y) column shares the +z ray direction and the projected position, so
// one BVH walk per column finds every triangle whose projection contains the
// column (the perturbed 2-D edge tests do not depend on z), and for each of
// them the crossing test of cell k reduces to "the plane lies above z_k".
// That test is monotone in z_k (n.(a - q) changes sign once along the column;
// the perturbation decides the tie the same way at every point), so a binary
// search over the sorted z coordinates with the exact per-point predicate
// finds the first cell the triangle no longer counts for, k_T.  Then
// chi(z_k) = sum over the column's triangles with k < k_T of sign(n_z),
// a sweep up the column.  Every decision is taken by the same predicate call
// the per-query traversal makes at the same point, so the result is
// bit-identical to it; the work per column is one walk plus log2(nz)
// predicate calls per hit triangle instead of nz walks.
//
// A column with more than kMaxHits crossing triangles (a very deep stack of
// surfaces) is handed to a per-cell fallback that walks the tree once per
// cell.
#include <algorithm>

#include "gwn_internal.cuh"
#include "predicates.cuh"
#include "traverse.cuh"

namespace gwn {

namespace {

constexpr int kMaxHits = 48;

// One thread per column (i, j), i fastest, so that the writes of cell k by a
// warp are consecutive in x.  chi layout: [(k ny + j) nx + i].
__global__ void __launch_bounds__(128) k_grid_chi(const float *__restrict__ gx, int nx, const float *__restrict__ gy,
                                                  int ny, const float *__restrict__ gz, int nz,
                                                  const BvhNode *__restrict__ nodes, int64_t nnodes,
                                                  const float4 *__restrict__ tri, int32_t *__restrict__ chi,
                                                  int32_t *__restrict__ overflow, unsigned *__restrict__ n_overflow,
                                                  unsigned long long *__restrict__ counters) {
    const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= (int64_t)nx * ny) return;
    const int i = (int)(col % nx), j = (int)(col / nx);
    const float px = gx[i], py = gy[j], z0 = gz[0];
    int hk[kMaxHits];
    int hs[kMaxHits];
    int nh = 0;
    bool over = false;
    unsigned long long *ce = &counters[CNT_EXACT_EDGE], *cp = &counters[CNT_EXACT_PLANE];
    const bool ok = bvh_walk_up(make_float3(px, py, z0), nodes, nnodes, tri, counters,
                                [&](int, float3 a, float3 b, float3 c) {
        const float zmax = fmaxf(a.z, fmaxf(b.z, c.z));
        if (z0 >= zmax) return;                       // at or below every cell of the column
        const int s0 = edge_sos(px, py, a.x, a.y, b.x, b.y, ce);
        const int s1 = edge_sos(px, py, b.x, b.y, c.x, c.y, ce);
        if (s0 == 0 || s0 != s1) return;
        const int s2 = edge_sos(px, py, c.x, c.y, a.x, a.y, ce);
        if (s2 != s0) return;
        // first cell the triangle does not count for: counts(k) is true, then false
        int lo = 0, hi = nz;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const float z = gz[mid];
            const bool counts = z < zmax && plane_sos(make_float3(px, py, z), a, b, c, s0, cp) == s0;
            if (counts) lo = mid + 1;
            else hi = mid;
        }
        if (lo == 0) return;
        if (nh == kMaxHits) {
            over = true;
            return;
        }
        hk[nh] = lo;
        hs[nh] = s0;
        ++nh;
    });
    if (!ok || over) {   // corrupt tree (flagged) or too many hits: the per-cell walk decides
        const unsigned slot = atomicAdd(n_overflow, 1u);
        overflow[slot] = (int32_t)col;
        return;
    }
    // sort by k_T, then sweep up the column
    for (int a = 1; a < nh; ++a) {
        const int k = hk[a], s = hs[a];
        int b = a - 1;
        while (b >= 0 && hk[b] > k) {
            hk[b + 1] = hk[b];
            hs[b + 1] = hs[b];
            --b;
        }
        hk[b + 1] = k;
        hs[b + 1] = s;
    }
    int c = 0;
    for (int a = 0; a < nh; ++a) c += hs[a];
    int h = 0;
    const int64_t plane = (int64_t)nx * ny;
    for (int k = 0; k < nz; ++k) {
        while (h < nh && hk[h] == k) c -= hs[h++];
        chi[(int64_t)k * plane + col] = c;
    }
}

// Per-cell fallback for the listed columns: one thread per (listed column, k).
__global__ void k_grid_chi_cells(const float *__restrict__ gx, int nx, const float *__restrict__ gy,
                                 const float *__restrict__ gz, int nz, int ny, const int32_t *__restrict__ overflow,
                                 const unsigned *__restrict__ n_overflow, const BvhNode *__restrict__ nodes,
                                 int64_t nnodes, const float4 *__restrict__ tri, int32_t *__restrict__ chi,
                                 unsigned long long *__restrict__ counters) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)(*n_overflow) * nz;
    if (t >= total) return;
    const int64_t col = overflow[t / nz];
    const int k = (int)(t % nz);
    const int i = (int)(col % nx), j = (int)(col / nx);
    chi[(int64_t)k * nx * ny + col] = chi_one(make_float3(gx[i], gy[j], gz[k]), nodes, nnodes, tri, counters);
}

// Materialise the grid points ([(k ny + j) nx + i][3]) for the per-point kernels.
__global__ void k_grid_points(const float *__restrict__ gx, int nx, const float *__restrict__ gy, int ny,
                              const float *__restrict__ gz, int64_t n, float *__restrict__ pts) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % nx);
    const int64_t r = c / nx;
    const int j = (int)(r % ny), k = (int)(r / ny);
    pts[3 * c] = gx[i];
    pts[3 * c + 1] = gy[j];
    pts[3 * c + 2] = gz[k];
}

// A closed mesh: w = chi, label = (chi > 1/2).
__global__ void k_chi_to_w(const int32_t *__restrict__ chi, int64_t n, float *__restrict__ w,
                           uint8_t *__restrict__ label) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int32_t v = chi[c];
    if (w) w[c] = (float)v;
    if (label) label[c] = v > 0 ? 1 : 0;
}

}  // namespace

// chi of every cell of the grid (device axis arrays, gz non-decreasing).
gwn_status launch_grid_chi(const gwn_mesh *m, const float *gx, int nx, const float *gy, int ny, const float *gz,
                           int nz, int32_t *chi, cudaStream_t s) {
    const int64_t ncol = (int64_t)nx * ny;
    if (ncol == 0 || nz == 0) return GWN_OK;
    int32_t *overflow = nullptr;
    unsigned *n_over = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&overflow, sizeof(int32_t) * ncol, s));
    GWN_CUDA_TRY(cudaMallocAsync(&n_over, sizeof(unsigned), s));
    cudaMemsetAsync(n_over, 0, sizeof(unsigned), s);
    {
        ProfScope prof("grid_chi", s);
        k_grid_chi<<<grid_for(ncol, 128), 128, 0, s>>>(gx, nx, gy, ny, gz, nz, m->nodes, m->nnodes, m->leaf_tri,
                                                        chi, overflow, n_over, m->counters);
    }
    unsigned h_over = 0;
    GWN_CUDA_TRY(cudaMemcpyAsync(&h_over, n_over, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_over > 0) {
        ProfScope prof("grid_chi_cells", s);
        k_grid_chi_cells<<<grid_for((int64_t)h_over * nz, 256), 256, 0, s>>>(gx, nx, gy, gz, nz, ny, overflow, n_over,
                                                                             m->nodes, m->nnodes, m->leaf_tri, chi,
                                                                             m->counters);
    }
    cudaFreeAsync(overflow, s);
    cudaFreeAsync(n_over, s);
    GWN_LAUNCH_CHECK("k_grid_chi");
    return GWN_OK;
}

// Labels (and w) of every cell: chi by ray reuse, then the boundary sum and the
// FP64 re-evaluation near 1/2 on the materialised grid points (a closed mesh
// needs neither: w = chi).
gwn_status launch_classify_grid(const gwn_mesh *m, const float *gx, int nx, const float *gy, int ny, const float *gz,
                                int nz, uint8_t *label, float *w, cudaStream_t s) {
    const int64_t n = (int64_t)nx * ny * nz;
    if (n == 0) return GWN_OK;
    int32_t *chi = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, s));
    gwn_status st = launch_grid_chi(m, gx, nx, gy, ny, gz, nz, chi, s);
    if (st == GWN_OK && m->npts < 2) {
        k_chi_to_w<<<grid_for(n, 256), 256, 0, s>>>(chi, n, w, label);
    } else if (st == GWN_OK) {
        float *pts = nullptr, *wt = w;
        int32_t *list = nullptr;
        unsigned long long *len = nullptr;
        if ((st = [&]() -> gwn_status {
                 GWN_CUDA_TRY(cudaMallocAsync(&pts, sizeof(float) * 3 * n, s));
                 GWN_CUDA_TRY(cudaMallocAsync(&list, sizeof(int32_t) * n, s));
                 GWN_CUDA_TRY(cudaMallocAsync(&len, sizeof(unsigned long long), s));
                 if (!wt) GWN_CUDA_TRY(cudaMallocAsync(&wt, sizeof(float) * n, s));
                 return GWN_OK;
             }()) == GWN_OK) {
            cudaMemsetAsync(len, 0, sizeof(unsigned long long), s);
            k_grid_points<<<grid_for(n, 256), 256, 0, s>>>(gx, nx, gy, ny, gz, n, pts);
            if ((st = launch_boundary_sum_list(m, pts, n, chi, wt, label, true, list, len, s)) == GWN_OK)
                st = launch_fp64_fix_list(m, pts, chi, wt, label, list, len, s);
        }
        for (void *p : {(void *)pts, (void *)list, (void *)len}) if (p) cudaFreeAsync(p, s);
        if (wt && wt != w) cudaFreeAsync(wt, s);
    }
    cudaFreeAsync(chi, s);
    if (st != GWN_OK) return st;
    GWN_LAUNCH_CHECK("classify grid");
    return GWN_OK;
}

}  // namespace gwn
