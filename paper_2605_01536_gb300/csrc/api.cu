// C ABI of the library (declared in include/gwn.h): argument checking, mesh
// ingest and validation, host/device pointer staging, and call sequencing.
#include <cmath>
#include <cstring>
#include <vector>
#include <string>

#include "gwn_internal.cuh"
#include "ptr_kind.h"

namespace gwn {

namespace {
thread_local std::string g_error;

constexpr int TB = 256;

// Sets the mesh's device current for the duration of a call and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else if (prev == dev) prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};


__global__ void k_ingest_vertices(const float *__restrict__ V, int64_t nv, float4 *__restrict__ out,
                                  unsigned long long *bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    float x = V[3 * i], y = V[3 * i + 1], z = V[3 * i + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicAdd(bad, 1ull);
    out[i] = make_float4(x, y, z, 0.f);
}

__global__ void k_ingest_faces(const int32_t *__restrict__ F, int64_t nt, int64_t nv, const float4 *__restrict__ V,
                               float *__restrict__ tri9, unsigned long long *bad) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int32_t a = F[3 * t], b = F[3 * t + 1], c = F[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
        atomicAdd(bad + 1, 1ull);
        return;
    }
    const float4 P[3] = {V[a], V[b], V[c]};
    for (int k = 0; k < 3; ++k) {
        tri9[9 * t + 3 * k] = P[k].x;
        tri9[9 * t + 3 * k + 1] = P[k].y;
        tri9[9 * t + 3 * k + 2] = P[k].z;
    }
}

gwn_status check_mesh(const gwn_mesh *m) {
    if (!m) return set_error(GWN_ERR_INVALID_ARG, "mesh is NULL");
    return GWN_OK;
}

gwn_status check_query_args(const gwn_mesh *m, const void *q, int64_t n, bool need_built) {
    gwn_status st = check_mesh(m);
    if (st != GWN_OK) return st;
    if (n < 0) return set_error(GWN_ERR_INVALID_ARG, "negative query count");
    if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "at most 2^31-1 queries per call");
    if (n > 0 && !q) return set_error(GWN_ERR_INVALID_ARG, "query pointer is NULL");
    if (need_built && !m->built) return set_error(GWN_ERR_NOT_BUILT, "call gwn_build_accel first");
    return GWN_OK;
}

// A query call's device-side view of the caller's buffers: device pointers are
// used in place; host pointers are staged through stream-ordered allocations.
struct Staging {
    cudaStream_t s;
    int device;
    bool any_host = false;
    void *allocs[16] = {};
    int nalloc = 0;
    struct Out { void *host; void *dev; size_t bytes; } outs[4] = {};
    int nout = 0;
    Staging(cudaStream_t st, int dev) : s(st), device(dev) {}
    gwn_status foreign(const void *p) {
        return set_error(GWN_ERR_INVALID_ARG, "a buffer is device memory of another GPU than the mesh's (device " +
                                                  std::to_string(device) + ")");
    }
    gwn_status alloc(void **p, size_t bytes) {
        GWN_CUDA_TRY(cudaMallocAsync(p, bytes > 0 ? bytes : 16, s));
        allocs[nalloc++] = *p;
        return GWN_OK;
    }
    gwn_status input(const void *host_or_dev, size_t bytes, const void **dev) {
        const int kind = pointer_kind(host_or_dev, device);
        if (kind < 0) return foreign(host_or_dev);
        if (kind > 0) { *dev = host_or_dev; return GWN_OK; }
        any_host = true;
        void *p = nullptr;
        gwn_status st = alloc(&p, bytes);
        if (st != GWN_OK) return st;
        GWN_CUDA_TRY(cudaMemcpyAsync(p, host_or_dev, bytes, cudaMemcpyHostToDevice, s));
        *dev = p;
        return GWN_OK;
    }
    gwn_status output(void *host_or_dev, size_t bytes, void **dev) {
        if (!host_or_dev) {   // caller does not want it: scratch
            return alloc(dev, bytes);
        }
        const int kind = pointer_kind(host_or_dev, device);
        if (kind < 0) return foreign(host_or_dev);
        if (kind > 0) { *dev = host_or_dev; return GWN_OK; }
        any_host = true;
        gwn_status st = alloc(dev, bytes);
        if (st != GWN_OK) return st;
        outs[nout++] = Out{host_or_dev, *dev, bytes};
        return GWN_OK;
    }
    gwn_status finish(gwn_status st) {
        if (st == GWN_OK) {
            for (int i = 0; i < nout; ++i) {
                cudaError_t e = cudaMemcpyAsync(outs[i].host, outs[i].dev, outs[i].bytes, cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) { st = set_error(GWN_ERR_CUDA, cudaGetErrorString(e)); break; }
            }
        }
        for (int i = 0; i < nalloc; ++i) cudaFreeAsync(allocs[i], s);
        if (st == GWN_OK && any_host) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = set_error(GWN_ERR_CUDA, cudaGetErrorString(e));
        }
        return st;
    }
};

}  // namespace

gwn_status set_error(gwn_status code, const std::string &msg) {
    g_error = msg;
    return code;
}

void clear_error() { g_error.clear(); }

int pointer_kind(const void *p, int device) {
    if (!p) return 1;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return gwn_pointer_kind_of((int)a.type, a.device, device);
}

gwn_status check_device_buffers(int device, std::initializer_list<const void *> ptrs, const char *what) {
    for (const void *p : ptrs) {
        const int kind = pointer_kind(p, device);
        if (kind < 0)
            return set_error(GWN_ERR_INVALID_ARG, std::string(what) + ": a buffer is device memory of another GPU "
                                                                      "than the mesh's (device " +
                                                      std::to_string(device) + ")");
        if (kind == 0) return set_error(GWN_ERR_INVALID_ARG, std::string(what) + " takes device buffers");
    }
    return GWN_OK;
}

}  // namespace gwn

using namespace gwn;

extern "C" {

const char *gwn_version(void) { return "gwn-gb300 0.1 (sm_103a)"; }

const char *gwn_last_error(void) { return g_error.c_str(); }

gwn_status gwn_mesh_create(const float *V, int64_t nv, const int32_t *F, int64_t nt, const gwn_config *cfg,
                           void *stream, gwn_mesh **out) {
    clear_error();
    if (!out) return set_error(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nv < 0 || nt < 0) return set_error(GWN_ERR_INVALID_ARG, "negative size");
    if (nv > (int64_t)0x7fffffff || 3 * nt > (int64_t)0x7fffffff)
        return set_error(GWN_ERR_INVALID_ARG, "mesh too large (nv and 3 nt must fit in int32)");
    if ((nv > 0 && !V) || (nt > 0 && !F)) return set_error(GWN_ERR_INVALID_ARG, "vertex or face pointer is NULL");
    if (nt > 0 && nv == 0) return set_error(GWN_ERR_INVALID_MESH, "faces without vertices");
    cudaStream_t s = (cudaStream_t)stream;
    gwn_mesh *m = new gwn_mesh();
    cudaGetDevice(&m->device);
    m->nv = nv;
    m->nt = nt;
    if (cfg) m->cfg = *cfg;
    if (m->cfg.queries_per_thread != 0 && m->cfg.queries_per_thread != 1 && m->cfg.queries_per_thread != 2 &&
        m->cfg.queries_per_thread != 4 && m->cfg.queries_per_thread != 8) {
        delete m;
        return set_error(GWN_ERR_INVALID_ARG, "queries_per_thread must be 1, 2, 4 or 8");
    }
    if (m->cfg.boundary_tile < 0 || m->cfg.boundary_tile > 8192) {
        delete m;
        return set_error(GWN_ERR_INVALID_ARG, "boundary_tile must be in [0, 8192]");
    }
    if (m->cfg.quantize_bits != 0 && m->cfg.quantize_bits != 30) {
        delete m;
        return set_error(GWN_ERR_INVALID_ARG, "quantize_bits must be 0 (exact FP32 inputs) or 30");
    }
    if (m->cfg.fp64_cancel < -1 || m->cfg.fp64_cancel > 1) {
        delete m;
        return set_error(GWN_ERR_INVALID_ARG, "fp64_cancel must be -1, 0 or 1");
    }
    if (m->cfg.group_test < 0 || m->cfg.group_test > 2) {
        delete m;
        return set_error(GWN_ERR_INVALID_ARG, "group_test must be 0, 1 or 2");
    }
    auto fail = [&](gwn_status st) {
        gwn_mesh_destroy(m);
        return st;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&m->counters, kStatusBytes)) != cudaSuccess)
        return fail(set_error(GWN_ERR_OOM, cudaGetErrorString(e)));
    cudaMemsetAsync(m->counters, 0, kStatusBytes, s);
    if (nv > 0 && (e = cudaMalloc(&m->V, sizeof(float4) * nv)) != cudaSuccess)
        return fail(set_error(GWN_ERR_OOM, cudaGetErrorString(e)));
    if (nt > 0 && ((e = cudaMalloc(&m->F, sizeof(int32_t) * 3 * nt)) != cudaSuccess ||
                   (e = cudaMalloc(&m->tri9, sizeof(float) * 9 * nt)) != cudaSuccess))
        return fail(set_error(GWN_ERR_OOM, cudaGetErrorString(e)));
    unsigned long long *bad = nullptr;
    if ((e = cudaMallocAsync(&bad, sizeof(unsigned long long) * 2, s)) != cudaSuccess)
        return fail(set_error(GWN_ERR_OOM, cudaGetErrorString(e)));
    cudaMemsetAsync(bad, 0, sizeof(unsigned long long) * 2, s);
    float *vtmp = nullptr;
    const int vkind = nv > 0 ? pointer_kind(V, m->device) : 1, fkind = nt > 0 ? pointer_kind(F, m->device) : 1;
    if (vkind < 0 || fkind < 0)
        return fail(set_error(GWN_ERR_INVALID_ARG, "V or F is device memory of another GPU than the current one"));
    if (nv > 0) {
        const float *vdev = V;
        if (vkind == 0) {
            if ((e = cudaMallocAsync(&vtmp, sizeof(float) * 3 * nv, s)) != cudaSuccess)
                return fail(set_error(GWN_ERR_OOM, cudaGetErrorString(e)));
            cudaMemcpyAsync(vtmp, V, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice, s);
            vdev = vtmp;
        }
        k_ingest_vertices<<<grid_for(nv, TB), TB, 0, s>>>(vdev, nv, m->V, bad);
    }
    if (nt > 0) {
        cudaMemcpyAsync(m->F, F, sizeof(int32_t) * 3 * nt, fkind > 0 ? cudaMemcpyDeviceToDevice
                                                                       : cudaMemcpyHostToDevice, s);
        k_ingest_faces<<<grid_for(nt, TB), TB, 0, s>>>(m->F, nt, nv, m->V, m->tri9, bad);
    }
    unsigned long long bad_h[2] = {0, 0};
    cudaMemcpyAsync(bad_h, bad, sizeof(bad_h), cudaMemcpyDeviceToHost, s);
    if (vtmp) cudaFreeAsync(vtmp, s);
    cudaFreeAsync(bad, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(set_error(GWN_ERR_CUDA, cudaGetErrorString(e)));
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(set_error(GWN_ERR_CUDA, cudaGetErrorString(e)));
    if (bad_h[0]) return fail(set_error(GWN_ERR_INVALID_MESH, std::to_string(bad_h[0]) + " non-finite vertices"));
    if (bad_h[1])
        return fail(set_error(GWN_ERR_INVALID_MESH, std::to_string(bad_h[1]) + " faces with an index out of range"));
    *out = m;
    return GWN_OK;
}

gwn_status gwn_mesh_destroy(gwn_mesh *m) {
    clear_error();
    if (!m) return set_error(GWN_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard g(m->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)m->V, (void *)m->F, (void *)m->tri9, (void *)m->bedges, (void *)m->bpts,
                    (void *)m->nodes, (void *)m->leaf_tri, (void *)m->counters, (void *)m->leaf_q, (void *)m->box})
        if (p) cudaFree(p);
    surrogate_free(m->sur);
    delete m;
    return GWN_OK;
}

gwn_status gwn_build_accel(gwn_mesh *m, void *stream) {
    clear_error();
    if (!m) return set_error(GWN_ERR_INVALID_ARG, "mesh is NULL");
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    m->built = false;
    gwn_status st = build_box(m, s);
    if (st != GWN_OK) return st;
    st = build_boundary(m, s);
    if (st != GWN_OK) return st;
    st = build_bvh(m, s);
    if (st != GWN_OK) return st;
    st = setup_quant(m, s);
    if (st != GWN_OK) return st;
    m->built = true;
    return GWN_OK;
}

gwn_status gwn_mesh_get_info(const gwn_mesh *m, gwn_mesh_info *info) {
    clear_error();
    if (!m || !info) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->nv = m->nv;
    info->nt = m->nt;
    info->n_boundary_edges = m->nb;
    info->n_boundary_points = m->npts;
    info->n_boundary_loops = m->nloops;
    info->n_bvh_nodes = m->nnodes;
    info->built = m->built ? 1 : 0;
    info->device = m->device;
    return GWN_OK;
}

gwn_status gwn_mesh_get_boundary(const gwn_mesh *m, int32_t *edges, int64_t cap, int64_t *n_out, void *stream) {
    clear_error();
    if (!m || !n_out) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    if (!m->built) return set_error(GWN_ERR_NOT_BUILT, "call gwn_build_accel first");
    *n_out = m->nb;
    if (m->nb == 0) return GWN_OK;
    if (!edges || cap < m->nb) return set_error(GWN_ERR_INVALID_ARG, "edge buffer too small");
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    GWN_CUDA_TRY(cudaMemcpyAsync(edges, m->bedges, sizeof(int32_t) * 2 * m->nb, cudaMemcpyDefault, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    return GWN_OK;
}

gwn_status gwn_mesh_get_boundary_points(const gwn_mesh *m, float *points, int64_t cap, int64_t *n_out,
                                        void *stream) {
    clear_error();
    if (!m || !n_out) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    if (!m->built) return set_error(GWN_ERR_NOT_BUILT, "call gwn_build_accel first");
    *n_out = m->npts;
    if (m->npts == 0) return GWN_OK;
    if (!points || cap < m->npts) return set_error(GWN_ERR_INVALID_ARG, "point buffer too small");
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    GWN_CUDA_TRY(cudaMemcpyAsync(points, m->bpts, sizeof(float4) * m->npts, cudaMemcpyDefault, s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    return GWN_OK;
}

gwn_status gwn_query_chi(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi, void *stream) {
    clear_error();
    gwn_status st = check_query_args(m, q, n, true);
    if (st != GWN_OK) return st;
    if (n > 0 && !chi) return set_error(GWN_ERR_INVALID_ARG, "chi is NULL");
    if (n == 0) return GWN_OK;
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    const void *qd = nullptr;
    void *cd = nullptr;
    if ((st = stg.input(q, sizeof(float) * 3 * n, &qd)) == GWN_OK &&
        (st = stg.output(chi, sizeof(int32_t) * n, &cd)) == GWN_OK)
        st = launch_chi(m, (const float *)qd, n, (int32_t *)cd, stg.s);
    return stg.finish(st);
}

gwn_status gwn_query_chi_visits(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi, uint64_t *nodes_out,
                                uint64_t *triangles_out, void *stream) {
    clear_error();
    gwn_status st = check_query_args(m, q, n, true);
    if (st != GWN_OK) return st;
    if (n > 0 && !chi) return set_error(GWN_ERR_INVALID_ARG, "chi is NULL");
    if (m->cfg.quantize_bits) return set_error(GWN_ERR_INVALID_ARG, "the instrumented walk is the exact-predicate one");
    if (nodes_out) *nodes_out = 0;
    if (triangles_out) *triangles_out = 0;
    if (n == 0) return GWN_OK;
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    const void *qd = nullptr;
    void *cd = nullptr;
    unsigned long long *v = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&v, 2 * sizeof(unsigned long long), stg.s));
    GWN_CUDA_TRY(cudaMemsetAsync(v, 0, 2 * sizeof(unsigned long long), stg.s));
    if ((st = stg.input(q, sizeof(float) * 3 * n, &qd)) == GWN_OK &&
        (st = stg.output(chi, sizeof(int32_t) * n, &cd)) == GWN_OK)
        st = launch_chi_visits(m, (const float *)qd, n, (int32_t *)cd, v, stg.s);
    unsigned long long h[2] = {0, 0};
    if (st == GWN_OK) {
        const cudaError_t e = cudaMemcpyAsync(h, v, sizeof(h), cudaMemcpyDeviceToHost, stg.s);
        if (e != cudaSuccess) st = set_error(GWN_ERR_CUDA, cudaGetErrorString(e));
    }
    st = stg.finish(st);
    cudaStreamSynchronize(stg.s);
    cudaFreeAsync(v, stg.s);
    cudaStreamSynchronize(stg.s);
    if (st == GWN_OK) {
        if (nodes_out) *nodes_out = h[0];
        if (triangles_out) *triangles_out = h[1];
    }
    return st;
}

gwn_status gwn_query_batch(const gwn_mesh *m, const float *q, int64_t n, float *w, int32_t *chi, void *stream) {
    clear_error();
    gwn_status st = check_query_args(m, q, n, true);
    if (st != GWN_OK) return st;
    if (n > 0 && !w) return set_error(GWN_ERR_INVALID_ARG, "w is NULL");
    if (n == 0) return GWN_OK;
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    const void *qd = nullptr;
    void *wd = nullptr, *cd = nullptr;
    if ((st = stg.input(q, sizeof(float) * 3 * n, &qd)) != GWN_OK ||
        (st = stg.output(w, sizeof(float) * n, &wd)) != GWN_OK)
        return stg.finish(st);
    if (n >= kOrderMinQueries) {   // in the queries' Morton order, scattered back
        void *keys = nullptr, *perm = nullptr, *qs = nullptr, *ws = nullptr, *cs = nullptr;
        if ((st = stg.output(chi, sizeof(int32_t) * n, &cd)) == GWN_OK &&
            (st = stg.alloc(&keys, sizeof(uint32_t) * n)) == GWN_OK &&
            (st = stg.alloc(&perm, sizeof(uint32_t) * n)) == GWN_OK &&
            (st = stg.alloc(&qs, sizeof(float) * 3 * n)) == GWN_OK &&
            (st = stg.alloc(&ws, sizeof(float) * n)) == GWN_OK &&
            (st = stg.alloc(&cs, sizeof(int32_t) * n)) == GWN_OK &&
            (st = order_queries(m, (const float *)qd, n, (uint32_t *)keys, (uint32_t *)perm, (float *)qs,
                                stg.s)) == GWN_OK &&
            (st = launch_chi(m, (const float *)qs, n, (int32_t *)cs, stg.s)) == GWN_OK &&
            (st = launch_boundary_sum_list(m, (const float *)qs, n, (const int32_t *)cs, (float *)ws, nullptr, false,
                                           nullptr, nullptr, stg.s)) == GWN_OK &&
            (st = scatter_f32((const float *)ws, (const uint32_t *)perm, n, (float *)wd, stg.s)) == GWN_OK)
            st = scatter_i32((const int32_t *)cs, (const uint32_t *)perm, n, chi ? (int32_t *)cd : nullptr, stg.s);
        return stg.finish(st);
    }
    if ((st = stg.output(chi, sizeof(int32_t) * n, &cd)) == GWN_OK &&
        (st = launch_chi(m, (const float *)qd, n, (int32_t *)cd, stg.s)) == GWN_OK)
        st = launch_boundary_sum_list(m, (const float *)qd, n, (const int32_t *)cd, (float *)wd, nullptr, false,
                                      nullptr, nullptr, stg.s);
    return stg.finish(st);
}

gwn_status gwn_classify(const gwn_mesh *m, const float *q, int64_t n, uint8_t *label, float *w_or_null,
                        void *stream) {
    clear_error();
    gwn_status st = check_query_args(m, q, n, true);
    if (st != GWN_OK) return st;
    if (n > 0 && !label) return set_error(GWN_ERR_INVALID_ARG, "label is NULL");
    if (n == 0) return GWN_OK;
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    const void *qd = nullptr;
    void *wd = nullptr, *cd = nullptr, *ld = nullptr, *list = nullptr, *len = nullptr;
    if ((st = stg.input(q, sizeof(float) * 3 * n, &qd)) != GWN_OK ||
        (st = stg.output(label, sizeof(uint8_t) * n, &ld)) != GWN_OK)
        return stg.finish(st);
    if (surrogate_ready(m)) {
        // the gate needs w_hat somewhere even when the caller does not want w
        if ((st = stg.output(w_or_null, sizeof(float) * n, &wd)) != GWN_OK) return stg.finish(st);
        return stg.finish(classify_with_surrogate(m, (const float *)qd, n, (uint8_t *)ld, (float *)wd, stg.s));
    }
    const bool ordered = n >= kOrderMinQueries;
    void *keys = nullptr, *perm = nullptr, *qs = nullptr, *ws = nullptr, *ls = nullptr;
    if (ordered) {   // in the queries' Morton order, scattered back
        if (w_or_null && (st = stg.output(w_or_null, sizeof(float) * n, &wd)) != GWN_OK) return stg.finish(st);
        if ((st = stg.alloc(&keys, sizeof(uint32_t) * n)) != GWN_OK ||
            (st = stg.alloc(&perm, sizeof(uint32_t) * n)) != GWN_OK ||
            (st = stg.alloc(&qs, sizeof(float) * 3 * n)) != GWN_OK ||
            (st = stg.alloc(&ws, sizeof(float) * n)) != GWN_OK ||
            (st = stg.alloc(&ls, sizeof(uint8_t) * n)) != GWN_OK ||
            (st = order_queries(m, (const float *)qd, n, (uint32_t *)keys, (uint32_t *)perm, (float *)qs,
                                stg.s)) != GWN_OK)
            return stg.finish(st);
    } else {
        if ((st = stg.output(w_or_null, sizeof(float) * n, &wd)) != GWN_OK) return stg.finish(st);
        qs = const_cast<void *>(qd);
        ws = wd;
        ls = ld;
    }
    if ((st = stg.alloc(&cd, sizeof(int32_t) * n)) == GWN_OK &&
        (st = stg.alloc(&list, sizeof(int32_t) * n)) == GWN_OK &&
        (st = stg.alloc(&len, sizeof(unsigned long long))) == GWN_OK) {
        cudaMemsetAsync(len, 0, sizeof(unsigned long long), stg.s);
        if ((st = launch_chi(m, (const float *)qs, n, (int32_t *)cd, stg.s)) == GWN_OK &&
            (st = launch_boundary_sum_list(m, (const float *)qs, n, (const int32_t *)cd, (float *)ws,
                                           (uint8_t *)ls, true, (int32_t *)list, (unsigned long long *)len,
                                           stg.s)) == GWN_OK)
            st = launch_fp64_fix_list(m, (const float *)qs, (const int32_t *)cd, (float *)ws, (uint8_t *)ls,
                                      (const int32_t *)list, (const unsigned long long *)len, stg.s);
        if (st == GWN_OK && ordered &&
            (st = scatter_u8((const uint8_t *)ls, (const uint32_t *)perm, n, (uint8_t *)ld, stg.s)) == GWN_OK)
            st = scatter_f32((const float *)ws, (const uint32_t *)perm, n, (float *)wd, stg.s);
    }
    return stg.finish(st);
}

gwn_status gwn_query_direct(const gwn_mesh *m, const float *q, int64_t n, float *w, void *stream) {
    clear_error();
    gwn_status st = check_query_args(m, q, n, false);
    if (st != GWN_OK) return st;
    if (n > 0 && !w) return set_error(GWN_ERR_INVALID_ARG, "w is NULL");
    if (n == 0) return GWN_OK;
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    const void *qd = nullptr;
    void *wd = nullptr;
    if ((st = stg.input(q, sizeof(float) * 3 * n, &qd)) == GWN_OK &&
        (st = stg.output(w, sizeof(float) * n, &wd)) == GWN_OK)
        st = launch_direct(m, (const float *)qd, n, (float *)wd, stg.s);
    return stg.finish(st);
}

gwn_status gwn_query_gradient(const gwn_mesh *m, const float *q, int64_t n, float *grad, void *stream) {
    clear_error();
    gwn_status st = check_query_args(m, q, n, true);
    if (st != GWN_OK) return st;
    if (n > 0 && !grad) return set_error(GWN_ERR_INVALID_ARG, "grad is NULL");
    if (n == 0) return GWN_OK;
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    const void *qd = nullptr;
    void *gd = nullptr;
    if ((st = stg.input(q, sizeof(float) * 3 * n, &qd)) == GWN_OK &&
        (st = stg.output(grad, sizeof(float) * 3 * n, &gd)) == GWN_OK)
        st = launch_gradient(m, (const float *)qd, n, (float *)gd, stg.s);
    return stg.finish(st);
}

}  // extern "C"

namespace {

// Validate a grid's axes (host or device arrays) and copy them to the device:
// counts >= 0, at most 2^31 - 1 cells, finite coordinates, z non-decreasing.
struct GridAxes {
    float *d = nullptr;   // x | y | z on the device
    int64_t n = 0;
    cudaStream_t s{};
    ~GridAxes() {
        if (d) cudaFreeAsync(d, s);
    }
    gwn_status load(const float *x, int32_t nx, const float *y, int32_t ny, const float *z, int32_t nz,
                    cudaStream_t st) {
        s = st;
        if (nx < 0 || ny < 0 || nz < 0) return set_error(GWN_ERR_INVALID_ARG, "negative grid size");
        n = (int64_t)nx * ny * nz;
        if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "at most 2^31-1 grid cells per call");
        if (n == 0) return GWN_OK;
        if (!x || !y || !z) return set_error(GWN_ERR_INVALID_ARG, "grid axis pointer is NULL");
        std::vector<float> h((size_t)nx + ny + nz);
        GWN_CUDA_TRY(cudaMemcpy(h.data(), x, sizeof(float) * nx, cudaMemcpyDefault));
        GWN_CUDA_TRY(cudaMemcpy(h.data() + nx, y, sizeof(float) * ny, cudaMemcpyDefault));
        GWN_CUDA_TRY(cudaMemcpy(h.data() + nx + ny, z, sizeof(float) * nz, cudaMemcpyDefault));
        for (float v : h)
            if (!std::isfinite(v)) return set_error(GWN_ERR_INVALID_ARG, "grid coordinate is not finite");
        for (int32_t k = 1; k < nz; ++k)
            if (h[nx + ny + k] < h[nx + ny + k - 1])
                return set_error(GWN_ERR_INVALID_ARG, "grid z coordinates must be non-decreasing");
        GWN_CUDA_TRY(cudaMallocAsync(&d, sizeof(float) * h.size(), s));
        GWN_CUDA_TRY(cudaMemcpyAsync(d, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, s));
        GWN_CUDA_TRY(cudaStreamSynchronize(s));   // h goes out of scope
        return GWN_OK;
    }
};

}  // namespace

extern "C" {

gwn_status gwn_query_grid_chi(const gwn_mesh *m, const float *x, int32_t nx, const float *y, int32_t ny,
                              const float *z, int32_t nz, int32_t *chi, void *stream) {
    clear_error();
    gwn_status st = check_mesh(m);
    if (st != GWN_OK) return st;
    if (!m->built) return set_error(GWN_ERR_NOT_BUILT, "call gwn_build_accel first");
    if (m->cfg.quantize_bits) return set_error(GWN_ERR_INVALID_ARG, "grid queries need quantize_bits = 0");
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    GridAxes ax;
    if ((st = ax.load(x, nx, y, ny, z, nz, stg.s)) != GWN_OK) return st;
    if (ax.n == 0) return GWN_OK;
    if (!chi) return set_error(GWN_ERR_INVALID_ARG, "chi is NULL");
    void *cd = nullptr;
    if ((st = stg.output(chi, sizeof(int32_t) * ax.n, &cd)) == GWN_OK)
        st = launch_grid_chi(m, ax.d, nx, ax.d + nx, ny, ax.d + nx + ny, nz, (int32_t *)cd, stg.s);
    return stg.finish(st);
}

gwn_status gwn_classify_grid(const gwn_mesh *m, const float *x, int32_t nx, const float *y, int32_t ny,
                             const float *z, int32_t nz, uint8_t *label, float *w_or_null, void *stream) {
    clear_error();
    gwn_status st = check_mesh(m);
    if (st != GWN_OK) return st;
    if (!m->built) return set_error(GWN_ERR_NOT_BUILT, "call gwn_build_accel first");
    if (m->cfg.quantize_bits) return set_error(GWN_ERR_INVALID_ARG, "grid queries need quantize_bits = 0");
    DeviceGuard g(m->device);
    Staging stg((cudaStream_t)stream, m->device);
    GridAxes ax;
    if ((st = ax.load(x, nx, y, ny, z, nz, stg.s)) != GWN_OK) return st;
    if (ax.n == 0) return GWN_OK;
    if (!label) return set_error(GWN_ERR_INVALID_ARG, "label is NULL");
    void *ld = nullptr, *wd = nullptr;
    if ((st = stg.output(label, ax.n, &ld)) == GWN_OK &&
        (st = stg.output(w_or_null, sizeof(float) * ax.n, &wd)) == GWN_OK)
        st = launch_classify_grid(m, ax.d, nx, ax.d + nx, ny, ax.d + nx + ny, nz, (uint8_t *)ld, (float *)wd, stg.s);
    return stg.finish(st);
}

gwn_status gwn_get_counters(gwn_mesh *m, gwn_counters *out, int reset, void *stream) {
    clear_error();
    if (!m || !out) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long c[CNT_SLOTS];
    GWN_CUDA_TRY(cudaMemcpyAsync(c, m->counters, sizeof(c), cudaMemcpyDeviceToHost, s));
    if (reset) GWN_CUDA_TRY(cudaMemsetAsync(m->counters, 0, sizeof(c), s));
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    std::memset(out, 0, sizeof(*out));
    out->error_flags = c[CNT_ERROR];
    out->exact_edge = c[CNT_EXACT_EDGE];
    out->exact_plane = c[CNT_EXACT_PLANE];
    out->exact_branch = c[CNT_EXACT_BRANCH];
    out->apex_terms = c[CNT_APEX];
    out->degenerate_terms = c[CNT_DEGENERATE];
    out->fp64_reevaluations = c[CNT_FP64];
    out->surrogate_queries = c[CNT_SUR_QUERIES];
    out->surrogate_fallbacks = c[CNT_SUR_FALLBACK];
    out->gradient_skipped = c[CNT_GRAD_SKIPPED];
    out->cancel_terms = c[CNT_CANCEL];
    out->cancel_overflow = c[CNT_CANCEL_OVERFLOW];
    if (c[CNT_ERROR] & ERR_TRAVERSAL_LIMIT)
        return set_error(GWN_ERR_TRAVERSAL_LIMIT, "BVH traversal exceeded its node budget");
    return GWN_OK;
}

}  // extern "C"
