// Batched evaluation of many meshes with uneven query sets in one persistent,
// graph-captured launch, plus the autotuner that picks its schedule.
//
// The work of a batch is cut into items: for every tile of up to 512*KP
// queries of a mesh, one crossing-number item and one item per chunk of the
// mesh's boundary points.  Items are sorted by estimated cost, largest first
// (longest-processing-time order), and a persistent grid pulls them from an
// atomic queue head (k_batch).  The launch sequence (clearing the queue head,
// the per-tile counters and the FP64 accumulators, then the kernel) is
// captured once into a CUDA graph on a stream the batch owns and replayed on
// every run with the same buffers; the caller's stream is ordered before and
// after it with events.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gwn_internal.cuh"

using namespace gwn;

struct gwn_batch {
    int device = 0;
    std::vector<const gwn_mesh *> meshes;
    std::vector<int64_t> q_off;
    int64_t total_q = 0;
    gwn_batch_config cfg{};
    int kp = 2, chunk = 8192, tile = 512, grid = 0;
    // device data
    BatchMesh *d_meshes = nullptr;
    BatchTile *d_tiles = nullptr;
    BatchItem *d_items = nullptr;
    unsigned *d_tile_done = nullptr;
    unsigned long long *d_head = nullptr;
    double *d_acc = nullptr;
    int32_t *d_chi = nullptr;
    int64_t *d_off = nullptr;              // [n_mesh + 1] query offsets
    int32_t *d_list = nullptr;             // queries whose cancelling terms overflowed the kernel's queue
    unsigned long long *d_list_len = nullptr;
    unsigned *d_listed = nullptr;          // one bit per query
    // the queries in (mesh, Morton) order and the results in that order
    uint64_t *d_keys = nullptr;
    uint32_t *d_perm = nullptr;
    float *d_qs = nullptr, *d_ws = nullptr;
    int32_t *d_cs = nullptr;
    int64_t n_tiles = 0, n_items = 0, cap_tiles = 0, cap_items = 0;
    // execution
    cudaStream_t s_int = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void *g_q = nullptr;
    void *g_w = nullptr, *g_chi = nullptr;
};

namespace {

int sm_count(int dev) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

void drop_graph(gwn_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->g_q = nullptr;
    b->g_w = b->g_chi = nullptr;
}

// Build the tile and item lists for a schedule (kp, chunk) and upload them.
// With qcap > 0 only the first qcap queries of each mesh get tiles (the
// autotuner's timing subsample).
gwn_status build_schedule(gwn_batch *b, int kp, int chunk, int tile, int grid, int64_t qcap = 0) {
    const int T = 512 * kp;
    std::vector<BatchTile> tiles;
    std::vector<BatchItem> items;
    std::vector<double> cost;
    for (size_t mi = 0; mi < b->meshes.size(); ++mi) {
        const gwn_mesh *m = b->meshes[mi];
        const int64_t q0 = b->q_off[mi];
        const int64_t nq = qcap > 0 ? std::min<int64_t>(qcap, b->q_off[mi + 1] - q0) : b->q_off[mi + 1] - q0;
        const int64_t nedge_pts = m->npts > 0 ? m->npts - 1 : 0;
        const int64_t nchunks = nedge_pts > 0 ? (nedge_pts + chunk - 1) / chunk : 0;
        const double chi_unit = 40.0 + 8.0 * std::log2((double)m->nt + 2.0);   // ~ one traversal in point terms
        // the autotuner's subsample: whole tiles spread evenly over the mesh's
        // (spatially ordered) queries, so that it samples the whole domain
        const int64_t nq_all = b->q_off[mi + 1] - q0;
        const int64_t tiles_all = (nq_all + T - 1) / T, tiles_used = (nq + T - 1) / T;
        for (int64_t ti_m = 0; ti_m < tiles_used; ++ti_m) {
            const int64_t src = qcap > 0 && tiles_used < tiles_all ? ti_m * tiles_all / tiles_used : ti_m;
            const int64_t t0 = src * T;
            BatchTile tl{};
            tl.mesh = (int32_t)mi;
            tl.q_begin = q0 + t0;
            tl.q_count = (int32_t)std::min<int64_t>(T, nq_all - t0);
            tl.n_items = (int32_t)(1 + nchunks);
            const int32_t ti = (int32_t)tiles.size();
            tiles.push_back(tl);
            items.push_back(BatchItem{ti, 0, 0, 0});
            cost.push_back(chi_unit * tl.q_count);
            for (int64_t c = 0; c < nchunks; ++c) {
                const int64_t p0 = c * chunk, p1 = std::min<int64_t>(nedge_pts, p0 + chunk);
                items.push_back(BatchItem{ti, 1, p0, p1});
                cost.push_back((double)(p1 - p0) * (double)T);   // a partial tile costs about a full one
            }
        }
    }
    std::vector<int64_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int64_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return cost[a] > cost[c]; });
    std::vector<BatchItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];

    if ((int64_t)tiles.size() > b->cap_tiles) {
        if (b->d_tiles) cudaFree(b->d_tiles);
        if (b->d_tile_done) cudaFree(b->d_tile_done);
        b->d_tiles = nullptr;
        b->d_tile_done = nullptr;
        GWN_CUDA_TRY(cudaMalloc(&b->d_tiles, sizeof(BatchTile) * std::max<size_t>(tiles.size(), 1)));
        GWN_CUDA_TRY(cudaMalloc(&b->d_tile_done, sizeof(unsigned) * std::max<size_t>(tiles.size(), 1)));
        b->cap_tiles = (int64_t)tiles.size();
    }
    if ((int64_t)sorted.size() > b->cap_items) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        GWN_CUDA_TRY(cudaMalloc(&b->d_items, sizeof(BatchItem) * std::max<size_t>(sorted.size(), 1)));
        b->cap_items = (int64_t)sorted.size();
    }
    if (!tiles.empty())
        GWN_CUDA_TRY(cudaMemcpy(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice));
    if (!sorted.empty())
        GWN_CUDA_TRY(cudaMemcpy(b->d_items, sorted.data(), sizeof(BatchItem) * sorted.size(), cudaMemcpyHostToDevice));
    b->n_tiles = (int64_t)tiles.size();
    b->n_items = (int64_t)sorted.size();
    b->kp = kp;
    b->chunk = chunk;
    b->tile = tile;
    b->grid = grid > 0 ? grid : batch_blocks_per_sm(kp, tile) * sm_count(b->device);
    drop_graph(b);
    return GWN_OK;
}

// One run: the queries in (mesh, Morton) order, the persistent kernel and the
// FP64 re-evaluation of overflow queries on that order, the results scattered
// back to the caller's order.
gwn_status enqueue_run(gwn_batch *b, const float *q, float *w, int32_t *chi, cudaStream_t s) {
    if (b->n_tiles > 0) GWN_CUDA_TRY(cudaMemsetAsync(b->d_tile_done, 0, sizeof(unsigned) * b->n_tiles, s));
    GWN_CUDA_TRY(cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long), s));
    if (b->total_q > 0) GWN_CUDA_TRY(cudaMemsetAsync(b->d_acc, 0, sizeof(double) * b->total_q, s));
    GWN_CUDA_TRY(cudaMemsetAsync(b->d_list_len, 0, sizeof(unsigned long long), s));
    GWN_CUDA_TRY(cudaMemsetAsync(b->d_listed, 0, sizeof(unsigned) * (size_t)((b->total_q + 31) / 32 + 1), s));
    if (b->n_items == 0 || b->total_q == 0) return GWN_OK;
    const int n_mesh = (int)b->meshes.size();
    gwn_status st = order_batch_queries(q, b->total_q, b->d_off, n_mesh, b->d_meshes, b->d_keys, b->d_perm, b->d_qs, s);
    if (st != GWN_OK) return st;
    if ((st = launch_batch_kernel(b->kp, b->grid, b->tile, b->d_meshes, b->d_tiles, b->d_items, b->n_items, b->d_qs,
                                  b->d_cs, b->d_acc, b->d_ws, b->d_tile_done, b->d_head, b->d_list, b->d_list_len,
                                  b->d_listed, s)) != GWN_OK)
        return st;
    if ((st = launch_batch_fp64_fix(b->d_meshes, b->d_off, n_mesh, b->d_qs, b->d_cs, b->d_ws, b->d_list,
                                    b->d_list_len, s)) != GWN_OK)
        return st;
    if ((st = scatter_f32(b->d_ws, b->d_perm, b->total_q, w, s)) != GWN_OK) return st;
    return scatter_i32(b->d_cs, b->d_perm, b->total_q, chi, s);
}

std::string tune_key(const gwn_batch *b) {
    int64_t pts = 0, tris = 0;
    for (auto *m : b->meshes) {
        pts += m->npts;
        tris += m->nt;
    }
    auto lg = [](int64_t x) { return (int)std::floor(std::log2((double)x + 1.0)); };
    char buf[128];
    std::snprintf(buf, sizeof(buf), "m%zu_q%d_p%d_t%d", b->meshes.size(), lg(b->total_q), lg(pts), lg(tris));
    return buf;
}

bool read_cache(const char *path, const std::string &key, int *kp, int *chunk, int *tile, int *grid) {
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[128];
        int a, c, t, g;
        if (std::sscanf(line, " {\"key\": \"%127[^\"]\", \"kp\": %d, \"chunk\": %d, \"tile\": %d, \"grid\": %d", k, &a,
                        &c, &t, &g) == 5 &&
            key == k) {
            *kp = a;
            *chunk = c;
            *tile = t;
            *grid = g;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void write_cache(const char *path, const std::string &key, int kp, int chunk, int tile, int grid, double ms) {
    if (!path) return;
    std::vector<std::string> keep;
    if (FILE *f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof(line), f)) {
            std::string l(line);
            if (l.find("\"key\": \"" + key + "\"") == std::string::npos && l.find("{") != std::string::npos)
                keep.push_back(l);
        }
        std::fclose(f);
    }
    if (FILE *f = std::fopen(path, "w")) {
        for (auto &l : keep) std::fputs(l.c_str(), f);
        std::fprintf(f, "{\"key\": \"%s\", \"kp\": %d, \"chunk\": %d, \"tile\": %d, \"grid\": %d, \"ms\": %.4f}\n",
                     key.c_str(), kp, chunk, tile, grid, ms);
        std::fclose(f);
    }
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

gwn_status gwn_batch_create(const gwn_mesh *const *meshes, int32_t n_mesh, const int64_t *q_offsets,
                            const gwn_batch_config *cfg, gwn_batch **out) {
    clear_error();
    if (!out) return set_error(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_mesh < 0 || (n_mesh > 0 && (!meshes || !q_offsets)))
        return set_error(GWN_ERR_INVALID_ARG, "meshes / q_offsets");
    if (n_mesh > 0 && q_offsets[0] != 0) return set_error(GWN_ERR_INVALID_ARG, "q_offsets[0] must be 0");
    for (int i = 0; i < n_mesh; ++i) {
        if (!meshes[i]) return set_error(GWN_ERR_INVALID_ARG, "mesh " + std::to_string(i) + " is NULL");
        if (!meshes[i]->built) return set_error(GWN_ERR_NOT_BUILT, "mesh " + std::to_string(i) + " is not built");
        if (q_offsets[i + 1] < q_offsets[i]) return set_error(GWN_ERR_INVALID_ARG, "q_offsets must not decrease");
        if (i > 0 && meshes[i]->device != meshes[0]->device)
            return set_error(GWN_ERR_INVALID_ARG, "all meshes must live on one device");
    }
    gwn_batch *b = new gwn_batch();
    if (n_mesh > 0) b->device = meshes[0]->device;
    else cudaGetDevice(&b->device);
    Guard g(b->device);
    b->meshes.assign(meshes, meshes + n_mesh);
    b->q_off.assign(q_offsets, q_offsets + n_mesh + 1);
    if (n_mesh == 0) b->q_off.assign(1, 0);
    b->total_q = b->q_off.back();
    if (b->total_q > (int64_t)0x7fffffff) {
        delete b;
        return set_error(GWN_ERR_INVALID_ARG, "at most 2^31-1 queries per batch");
    }
    if (cfg) b->cfg = *cfg;
    auto fail = [&](gwn_status st) {
        gwn_batch_destroy(b);
        return st;
    };
    std::vector<BatchMesh> md(std::max(n_mesh, 1));
    for (int i = 0; i < n_mesh; ++i) {
        const gwn_mesh *m = meshes[i];
        md[i] = BatchMesh{m->nodes, m->leaf_tri, m->bpts, m->nnodes, m->npts, m->counters, m->box};
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_meshes, sizeof(BatchMesh) * md.size())) != cudaSuccess ||
        (e = cudaMemcpy(b->d_meshes, md.data(), sizeof(BatchMesh) * md.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc(&b->d_head, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_acc, sizeof(double) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_chi, sizeof(int32_t) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_off, sizeof(int64_t) * b->q_off.size())) != cudaSuccess ||
        (e = cudaMemcpy(b->d_off, b->q_off.data(), sizeof(int64_t) * b->q_off.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc(&b->d_list, sizeof(int32_t) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_list_len, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_listed, sizeof(unsigned) * (size_t)((b->total_q + 31) / 32 + 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_keys, sizeof(uint64_t) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_perm, sizeof(uint32_t) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_qs, sizeof(float) * 3 * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_ws, sizeof(float) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_cs, sizeof(int32_t) * std::max<int64_t>(b->total_q, 1))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->s_int, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess)
        return fail(set_error(e == cudaErrorMemoryAllocation ? GWN_ERR_OOM : GWN_ERR_CUDA, cudaGetErrorString(e)));
    const int kp = (b->cfg.queries_per_thread == 2) ? 1 : 2;
    const int chunk = b->cfg.points_per_item > 0 ? b->cfg.points_per_item : 8192;
    const int tile = b->cfg.tile > 0 ? b->cfg.tile : 512;
    if (tile > 8192 || chunk < 1) return fail(set_error(GWN_ERR_INVALID_ARG, "tile must be <= 8192, chunk >= 1"));
    gwn_status st = build_schedule(b, kp, chunk, tile, b->cfg.grid_blocks);
    if (st != GWN_OK) return fail(st);
    *out = b;
    return GWN_OK;
}

gwn_status gwn_batch_destroy(gwn_batch *b) {
    clear_error();
    if (!b) return set_error(GWN_ERR_INVALID_ARG, "batch is NULL");
    Guard g(b->device);
    if (b->s_int) cudaStreamSynchronize(b->s_int);
    drop_graph(b);
    for (void *p : {(void *)b->d_meshes, (void *)b->d_tiles, (void *)b->d_items, (void *)b->d_tile_done,
                    (void *)b->d_head, (void *)b->d_acc, (void *)b->d_chi, (void *)b->d_off, (void *)b->d_list,
                    (void *)b->d_list_len, (void *)b->d_listed, (void *)b->d_keys, (void *)b->d_perm,
                    (void *)b->d_qs, (void *)b->d_ws, (void *)b->d_cs})
        if (p) cudaFree(p);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->s_int) cudaStreamDestroy(b->s_int);
    delete b;
    return GWN_OK;
}

gwn_status gwn_batch_run(gwn_batch *b, const float *q, float *w, int32_t *chi, void *stream) {
    clear_error();
    if (!b) return set_error(GWN_ERR_INVALID_ARG, "batch is NULL");
    if (b->total_q > 0 && (!q || !w)) return set_error(GWN_ERR_INVALID_ARG, "q or w is NULL");
    Guard g(b->device);
    for (const void *p : {(const void *)q, (const void *)w, (const void *)chi}) {
        const int kind = pointer_kind(p, b->device);
        if (kind < 0) return set_error(GWN_ERR_INVALID_ARG, "gwn_batch_run: a buffer is device memory of another GPU");
        if (kind == 0) return set_error(GWN_ERR_INVALID_ARG, "gwn_batch_run takes device pointers");
    }
    int32_t *chi_out = chi ? chi : b->d_chi;
    cudaStream_t cs = (cudaStream_t)stream;
    GWN_CUDA_TRY(cudaEventRecord(b->ev_in, cs));
    GWN_CUDA_TRY(cudaStreamWaitEvent(b->s_int, b->ev_in, 0));
    gwn_status st = GWN_OK;
    if (b->cfg.use_graph >= 0) {
        if (!b->gexec || b->g_q != q || b->g_w != w || b->g_chi != chi_out) {
            drop_graph(b);
            cudaGraph_t graph = nullptr;
            GWN_CUDA_TRY(cudaStreamBeginCapture(b->s_int, cudaStreamCaptureModeThreadLocal));
            st = enqueue_run(b, q, w, chi_out, b->s_int);
            cudaError_t e = cudaStreamEndCapture(b->s_int, &graph);
            if (st != GWN_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return set_error(GWN_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                return set_error(GWN_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            }
            b->g_q = q;
            b->g_w = w;
            b->g_chi = chi_out;
        }
        ProfScope prof("batch_graph", b->s_int);
        GWN_CUDA_TRY(cudaGraphLaunch(b->gexec, b->s_int));
    } else {
        st = enqueue_run(b, q, w, chi_out, b->s_int);
        if (st != GWN_OK) return st;
    }
    GWN_CUDA_TRY(cudaEventRecord(b->ev_out, b->s_int));
    GWN_CUDA_TRY(cudaStreamWaitEvent(cs, b->ev_out, 0));
    return GWN_OK;
}

gwn_status gwn_batch_get_config(const gwn_batch *b, gwn_batch_config *cfg, int64_t *n_items) {
    clear_error();
    if (!b || !cfg) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    *cfg = b->cfg;
    cfg->queries_per_thread = 2 * b->kp;
    cfg->points_per_item = b->chunk;
    cfg->tile = b->tile;
    cfg->grid_blocks = b->grid;
    if (n_items) *n_items = b->n_items;
    return GWN_OK;
}

gwn_status gwn_batch_autotune(gwn_batch *b, const float *q, float *w, void *stream, const char *cache_path,
                              gwn_batch_config *chosen) {
    clear_error();
    if (!b) return set_error(GWN_ERR_INVALID_ARG, "batch is NULL");
    Guard g(b->device);
    const std::string key = tune_key(b);
    int kp = 0, chunk = 0, tile = 0, grid = 0;
    gwn_status st;
    if (read_cache(cache_path, key, &kp, &chunk, &tile, &grid)) {
        if ((st = build_schedule(b, kp, chunk, tile, grid)) != GWN_OK) return st;
        return chosen ? gwn_batch_get_config(b, chosen, nullptr) : GWN_OK;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    GWN_CUDA_TRY(cudaStreamSynchronize(cs));
    cudaEvent_t e0, e1;
    GWN_CUDA_TRY(cudaEventCreate(&e0));
    GWN_CUDA_TRY(cudaEventCreate(&e1));
    const int sms = sm_count(b->device);
    const int64_t qcap = b->cfg.tune_queries_per_mesh > 0 ? b->cfg.tune_queries_per_mesh : 16384;
    double best = 1e30;
    int bkp = 2, bchunk = 8192, btile = 512, bgrid = 0;
    for (int ckp : {1, 2}) {
        for (int cchunk : {2048, 8192, 32768}) {
            const int occ = batch_blocks_per_sm(ckp, 512);
            for (int mult : {1, 2}) {
                const int cgrid = occ * sms * mult;
                if ((st = build_schedule(b, ckp, cchunk, 512, cgrid, qcap)) != GWN_OK) break;
                double ms_best = 1e30;
                for (int rep = 0; rep < 3 && st == GWN_OK; ++rep) {
                    cudaEventRecord(e0, b->s_int);
                    st = enqueue_run(b, q, w, b->d_chi, b->s_int);
                    cudaEventRecord(e1, b->s_int);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_best = std::min(ms_best, (double)ms);   // the first run warms up
                }
                if (st != GWN_OK) break;
                if (ms_best < best) {
                    best = ms_best;
                    bkp = ckp;
                    bchunk = cchunk;
                    btile = 512;
                    bgrid = cgrid;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GWN_OK) return st;
    if ((st = build_schedule(b, bkp, bchunk, btile, bgrid)) != GWN_OK) return st;
    write_cache(cache_path, key, bkp, bchunk, btile, bgrid, best);
    return chosen ? gwn_batch_get_config(b, chosen, nullptr) : GWN_OK;
}

}  // extern "C"
