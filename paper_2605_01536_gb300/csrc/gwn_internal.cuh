// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <initializer_list>
#include <string>

#include "../../include/gwn.h"

namespace gwn {

// ---------------------------------------------------------------------------
// Error handling: every C entry point returns a status; a thread-local string
// carries the message.
// ---------------------------------------------------------------------------
gwn_status set_error(gwn_status code, const std::string &msg);
void clear_error();
// Where a caller's buffer lives: 1 = device memory of `device` (or managed
// memory, or NULL), 0 = host memory, -1 = device memory of another GPU, which
// the kernels launched for `device` must not dereference.
int pointer_kind(const void *p, int device);
// GWN_OK if every non-NULL buffer is device memory of `device` (or managed);
// otherwise GWN_ERR_INVALID_ARG naming `what`.
gwn_status check_device_buffers(int device, std::initializer_list<const void *> ptrs, const char *what);

// Makes `dev` current for the scope (the caller's device is restored).
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define GWN_CUDA_TRY(expr)                                                        \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            return ::gwn::set_error(e_ == cudaErrorMemoryAllocation ? GWN_ERR_OOM \
                                                                   : GWN_ERR_CUDA, \
                                    std::string(#expr) + ": " + cudaGetErrorString(e_)); \
        }                                                                         \
    } while (0)

#define GWN_LAUNCH_CHECK(what)                                                    \
    do {                                                                          \
        cudaError_t e_ = cudaGetLastError();                                      \
        if (e_ != cudaSuccess)                                                    \
            return ::gwn::set_error(GWN_ERR_CUDA, std::string(what) + ": " +      \
                                                      cudaGetErrorString(e_));    \
    } while (0)

// ---------------------------------------------------------------------------
// Device data of a mesh.
// ---------------------------------------------------------------------------

// One BVH node (internal or leaf), 32 bytes.  The box is the xy extent of the
// node's triangles and their maximum z: a +z ray from q can only cross a
// triangle of the node if q.xy lies in the closed xy box and q.z <= zmax.
struct __align__(16) BvhNode {
    float xmin, xmax, ymin, ymax;
    float zmax;
    int32_t child;   // internal: index of the left child; leaf: triangle slot (>= 0)
    int32_t skip;    // next node in depth-first order after this subtree (-1 = end)
    int32_t is_leaf;
};
static_assert(sizeof(BvhNode) == 32, "BvhNode must be 32 bytes");

// Counter slots in the device status array.
enum CounterSlot {
    CNT_ERROR = 0,
    CNT_EXACT_EDGE = 1,
    CNT_EXACT_PLANE = 2,
    CNT_EXACT_BRANCH = 3,
    CNT_APEX = 4,
    CNT_DEGENERATE = 5,
    CNT_FP64 = 6,
    CNT_SUR_QUERIES = 7,
    CNT_SUR_FALLBACK = 8,
    CNT_GRAD_SKIPPED = 9,
    CNT_CANCEL = 10,
    CNT_CANCEL_OVERFLOW = 11,
    CNT_SLOTS = 16
};

enum ErrorBits { ERR_TRAVERSAL_LIMIT = 1 };

struct Surrogate;   // mlp.cu

// bytes of a mesh's device status block: the counters and the fixed-point frame
constexpr size_t kStatusBytes = sizeof(unsigned long long) * CNT_SLOTS + 64;

}  // namespace gwn

struct gwn_mesh {
    int device = 0;
    int64_t nv = 0, nt = 0;
    gwn_config cfg{};

    float4 *V = nullptr;        // [nv] (x, y, z, 0)
    int32_t *F = nullptr;       // [3 nt]
    float *tri9 = nullptr;      // [9 nt] the three vertices of each face, input order

    bool built = false;
    int64_t nb = 0;             // boundary edges (with multiplicity)
    int32_t *bedges = nullptr;  // [2 nb], sorted by undirected key
    int64_t npts = 0;           // chained boundary points
    int64_t nloops = 0;
    float4 *bpts = nullptr;     // [npts] (x, y, z, flag): flag 1 = an edge runs to the next point
    int64_t nnodes = 0;
    gwn::BvhNode *nodes = nullptr;   // [2 nt - 1]
    float4 *leaf_tri = nullptr;      // [3 nt] triangles in BVH leaf order
    bool bvh_xy = false;             // the tree was built over xy Morton codes (columns), else xyz

    unsigned long long *counters = nullptr;   // status block: [CNT_SLOTS] counters, then the
                                               // fixed-point frame (quant.cuh), kStatusBytes in all
    int4 *leaf_q = nullptr;                    // [3 nt] snapped leaf triangles (quantize_bits = 30)
    float *box = nullptr;                      // [6] vertex box: min x, y, z, max x, y, z (after the build)
    gwn::Surrogate *sur = nullptr;             // optional learned surrogate (mlp.cu)
};

namespace gwn {

// build.cu
gwn_status build_boundary(gwn_mesh *m, cudaStream_t s);
gwn_status build_bvh(gwn_mesh *m, cudaStream_t s);
gwn_status build_box(gwn_mesh *m, cudaStream_t s);   // m->box from the vertices

// order.cu: Morton order of a query batch in the mesh's box (keys, perm: [n]
// scratch; qs: [3 n] the queries in that order), and the scatter of results
// back to the caller's order (out[perm[i]] = in[i]; out NULL: nothing)
gwn_status order_queries(const gwn_mesh *m, const float *q, int64_t n, uint32_t *keys, uint32_t *perm, float *qs,
                         cudaStream_t s);
// list: n indices into q, reordered by their queries' Morton codes (lists
// shorter than kOrderMinQueries are left as they are)
gwn_status order_query_list(const gwn_mesh *m, const float *q, int32_t *list, int64_t n, cudaStream_t s);
gwn_status scatter_f32(const float *in, const uint32_t *perm, int64_t n, float *out, cudaStream_t s);
gwn_status scatter_i32(const int32_t *in, const uint32_t *perm, int64_t n, int32_t *out, cudaStream_t s);
gwn_status scatter_u8(const uint8_t *in, const uint32_t *perm, int64_t n, uint8_t *out, cudaStream_t s);
// batches at least this large are evaluated in Morton order
constexpr int64_t kOrderMinQueries = 16384;

// sort.cu: stable LSD radix sort of (key, value) pairs on the low `bits` bits.
// keys/vals are sorted in place (temporaries from the stream-ordered allocator).
gwn_status radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s);
gwn_status radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s);
// exclusive prefix sum of n uint32 values into out (out may alias in); *total (device) gets the sum
gwn_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                              cudaStream_t s);

// query.cu
gwn_status launch_chi(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi, cudaStream_t s);
gwn_status launch_chi_visits(const gwn_mesh *m, const float *q, int64_t n, int32_t *chi,
                             unsigned long long *visits, cudaStream_t s);
// boundary-curve sum + combine; with classify, labels and appends queries within
// the margin to list (length counter list_len, zeroed by the caller)
gwn_status launch_boundary_sum_list(const gwn_mesh *m, const float *q, int64_t n, const int32_t *chi,
                                    float *w, uint8_t *label, bool classify, int32_t *list,
                                    unsigned long long *list_len, cudaStream_t s);
// FP64 re-evaluation of the listed queries (rewrites w and label)
gwn_status launch_fp64_fix_list(const gwn_mesh *m, const float *q, const int32_t *chi, float *w,
                                uint8_t *label, const int32_t *list, const unsigned long long *list_len,
                                cudaStream_t s);
gwn_status launch_direct(const gwn_mesh *m, const float *q, int64_t n, float *w, cudaStream_t s);
// quant.cu: the fixed-point frame of the mesh (quantize_bits), written into the
// status block; bits = 0 (exact FP32 predicates) unless configured
gwn_status setup_quant(gwn_mesh *m, cudaStream_t s);
// grid.cu: ray reuse on a rectilinear grid (Supp. S3); axis arrays on the device,
// gz non-decreasing; outputs indexed [(k ny + j) nx + i]
gwn_status launch_grid_chi(const gwn_mesh *m, const float *gx, int nx, const float *gy, int ny, const float *gz,
                           int nz, int32_t *chi, cudaStream_t s);
gwn_status launch_classify_grid(const gwn_mesh *m, const float *gx, int nx, const float *gy, int ny, const float *gz,
                                int nz, uint8_t *label, float *w, cudaStream_t s);
// gradient.cu: grad w (float [n][3]) by Supp. S4, Algorithm 3
gwn_status launch_gradient(const gwn_mesh *m, const float *q, int64_t n, float *grad, cudaStream_t s);
// mlp.cu: the surrogate
void surrogate_free(Surrogate *s);
bool surrogate_ready(const gwn_mesh *m);
gwn_status classify_with_surrogate(const gwn_mesh *m, const float *q, int64_t n, uint8_t *label, float *w,
                                   cudaStream_t s);
// the classify sequence on caller-provided scratch; allocates nothing
gwn_status launch_classify_on_scratch(const gwn_mesh *m, const float *q, int64_t n, uint8_t *label, float *w,
                                      int32_t *chi_tmp, int32_t *list, unsigned long long *list_len,
                                      unsigned *listed, double *partial, int64_t partial_cap, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched evaluation of many meshes (one persistent launch over a work queue).
// ---------------------------------------------------------------------------
struct BatchMesh {
    const BvhNode *nodes;
    const float4 *tri;
    const float4 *pts;
    int64_t nnodes;
    int64_t npts;
    unsigned long long *counters;
    const float *box;   // vertex box (min xyz, max xyz), for the query order
};
// order.cu: the batch's queries (mesh ranges given by mesh_off [n_mesh + 1]) in
// (mesh, Morton code in the mesh's box) order: keys, perm [n] scratch, qs [3 n]
gwn_status order_batch_queries(const float *q, int64_t n, const int64_t *mesh_off, int n_mesh,
                               const BatchMesh *meshes, uint64_t *keys, uint32_t *perm, float *qs, cudaStream_t s);
struct BatchTile {      // up to 512 * KP queries of one mesh
    int32_t mesh;
    int32_t n_items;    // work items of the tile (the crossing item + boundary chunks)
    int64_t q_begin;
    int32_t q_count;
    int32_t pad;
};
struct BatchItem {      // kind 0: crossing numbers of the tile; 1: boundary chunk
    int32_t tile;
    int32_t kind;
    int64_t p_begin, p_end;   // edge start points of the chunk
};
// list / list_len / listed: queries whose cancelling boundary terms overflow the
// kernel's queue, for launch_batch_fp64_fix (listed: zeroed bits, one per query)
gwn_status launch_batch_kernel(int kp, int grid, int tile_pts, const BatchMesh *meshes, const BatchTile *tiles,
                               const BatchItem *items, int64_t n_items, const float *q, int32_t *chi, double *acc,
                               float *w, unsigned *tile_done, unsigned long long *head, int32_t *list,
                               unsigned long long *list_len, unsigned *listed, cudaStream_t s);
// FP64 boundary sum of the listed queries of a batch (mesh_off: [n_mesh + 1]
// query offsets of the meshes), rewriting w = chi + S / 2pi
gwn_status launch_batch_fp64_fix(const BatchMesh *meshes, const int64_t *mesh_off, int n_mesh, const float *q,
                                 const int32_t *chi, float *w, const int32_t *list,
                                 const unsigned long long *list_len, cudaStream_t s);
int batch_blocks_per_sm(int kp, int tile_pts);

// Optional timing of one launch (see gwn_profile_enable): records CUDA events
// on the launching stream around the scope when profiling is on.
// Scopes nest; note_launches(k) adds k kernels to the innermost active scope
// of the calling thread (a scope that notes none counts as one kernel).
class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
    int64_t kernels_ = 0;

  private:
    const char *name_;
    cudaStream_t s_;
    cudaEvent_t a_{}, b_{};
    bool active_ = false;
    ProfScope *parent_ = nullptr;
};
void note_launches(int k);

inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace gwn
