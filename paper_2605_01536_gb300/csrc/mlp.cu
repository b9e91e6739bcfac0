// Per-mesh surrogate of the winding number: a small MLP trained on w values
// produced by the antipodal kernels, evaluated and trained on the tensor cores
// (tcgen05, BF16 operands, FP32 accumulators in TMEM).
//
// Network (all sizes fixed):
//   x = 2 (q - lo) / (hi - lo) - 1 (the padded bounding box maps to [-1, 1]^3)
//   f = [x, y, z, sin(pi s_k x_d), cos(pi s_k x_d)]  k < 16, d < 3, s_k = 2^(7k/15)
//       (99 features, zero-padded to 128)
//   h1 = relu(W1 f + b1), h2..h4 = relu(W_l h_{l-1} + b_l)   (64 wide)
//   w_hat = w5 . h4 + b5
// Loss: mean squared error to the exact w; Adam on FP32 master weights; the
// matrix products take BF16 copies of the weights and BF16 activations.
//
// Every matrix product is a 128 x 64 tile D = A B^T computed by one chain of
// tcgen05.mma (K = 16 each) on operands staged in shared memory in the
// core-matrix layout of tc.cuh:
//   forward     D[b][n]  = sum_k h_{l-1}[b][k] W_l[n][k]       (A = activations, B = W_l)
//   input grad  D[b][k]  = sum_n delta_l[b][n] W_l[n][k]        (A = delta_l, B = W_l^T)
//   weight grad D[k][n]  = sum_b h_{l-1}[b][k] delta_l[b][n]   (A = h^T, B = delta^T)
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gwn_internal.cuh"
#include "tc.cuh"

namespace gwn {

namespace {

constexpr uint32_t kWaitPolls = 1u << 24;
constexpr int kIn = 128;      // padded feature width
constexpr int kFeat = 99;     // real features
constexpr int kHid = 64;
constexpr int kNFreq = 16;
// parameter offsets in the flat FP32 vector
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn;
constexpr int oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid;
constexpr int oW3 = oB2 + kHid, oB3 = oW3 + kHid * kHid;
constexpr int oW4 = oB3 + kHid, oB4 = oW4 + kHid * kHid;
constexpr int oW5 = oB4 + kHid, oB5 = oW5 + kHid;
constexpr int kParams = oB5 + 1;
// BF16 weight copies: W1 [64][128], then W2, W3, W4 [64][64]
constexpr int kWbf = kHid * kIn + 3 * kHid * kHid;

__constant__ float c_freq[kNFreq];   // s_k = 2^(7k/15) (FP32)

struct MlpDev {
    const __nv_bfloat16 *wbf;   // BF16 weights
    const float *params;        // FP32 master parameters (biases, w5, b5 read from here)
    float scale[3], offset[3];  // x = q * scale + offset
    const uint32_t *band;       // surface band: one bit per cell of a band_res^3 grid over the box (or NULL)
    int band_res;
};

// True when q lies in a cell of the surface band (cells touched by a triangle's
// bounding box, dilated): there w jumps across the surface and the network's
// answer is not used.  Outside the box there is no surface.
__device__ __forceinline__ bool in_band(const MlpDev &P, float qx, float qy, float qz) {
    if (!P.band) return false;
    const float R = (float)P.band_res;
    const float fx = (fmaf(qx, P.scale[0], P.offset[0]) + 1.f) * 0.5f * R;
    const float fy = (fmaf(qy, P.scale[1], P.offset[1]) + 1.f) * 0.5f * R;
    const float fz = (fmaf(qz, P.scale[2], P.offset[2]) + 1.f) * 0.5f * R;
    if (!(fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < R && fy < R && fz < R)) return false;
    const int64_t c = ((int64_t)fz * P.band_res + (int64_t)fy) * P.band_res + (int64_t)fx;
    return (P.band[c >> 5] >> (c & 31)) & 1u;
}

// Shared-memory layout of the forward kernel (bytes).
constexpr int kSmemW1 = 0;                                  // [64][128] bf16 core layout: 16 KB
constexpr int kSmemW2 = kSmemW1 + kHid * kIn * 2;           // [64][64]: 8 KB each
constexpr int kSmemW3 = kSmemW2 + kHid * kHid * 2;
constexpr int kSmemW4 = kSmemW3 + kHid * kHid * 2;
constexpr int kSmemX = kSmemW4 + kHid * kHid * 2;           // [128][128] features: 32 KB
// [128][64] activations: 16 KB inside the feature buffer (layer 1 has read the
// features by the time its output is written), so three CTAs fit on an SM
constexpr int kSmemH = kSmemX;
constexpr int kSmemBias = kSmemX + 128 * kIn * 2;           // b1..b4, w5 (5 x 64 floats) + b5
constexpr int kSmemFwd = kSmemBias + (5 * kHid + 4) * 4;

__device__ __forceinline__ void store_row_bf16(unsigned char *sA, int r, const float *v, int K) {
    // 8 consecutive k of row r are one 16-byte chunk of a core matrix
    for (int kc = 0; kc < K / 8; ++kc) {
        __nv_bfloat162 p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[kc * 8 + 2 * i], v[kc * 8 + 2 * i + 1]);
        *reinterpret_cast<uint4 *>(sA + tc::core_offset(r, kc * 8, K)) = *reinterpret_cast<uint4 *>(p);
    }
}

// sin(pi t) and cos(pi t): t is reduced to r = t - 2 rint(t / 2) in [-1, 1]
// (exact in FP32 for |t| < 2^22), then the SFU sine and cosine of pi r
// (absolute error below 1e-6, far under the BF16 rounding the features get).
__device__ __forceinline__ float2 sincos_halfturns(float t) {
    const float r = fmaf(-2.f, rintf(0.5f * t), t);
    float sn, cs;
    __sincosf(3.14159265358979f * r, &sn, &cs);
    return make_float2(sn, cs);
}

// Features of one query written as BF16 into row r of the core-layout matrix
// sX, eight at a time (one 16-byte store per core-matrix row chunk).
__device__ __forceinline__ void features_to_smem(float qx, float qy, float qz, const MlpDev &P, unsigned char *sX,
                                                 int r) {
    const float x[3] = {fmaf(qx, P.scale[0], P.offset[0]), fmaf(qy, P.scale[1], P.offset[1]),
                        fmaf(qz, P.scale[2], P.offset[2])};
    float buf[8];
    float2 sc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        float v = 0.f;
        if (i < 3) {
            v = x[i];
        } else if (i < kFeat) {
            const int j = i - 3, k = j / 6, d = (j % 6) / 2;
            if ((j & 1) == 0) {
                sc = sincos_halfturns(c_freq[k] * x[d]);
                v = sc.x;
            } else {
                v = sc.y;
            }
        }
        buf[i & 7] = v;
        if ((i & 7) == 7) {
            __nv_bfloat162 p[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) p[t] = __floats2bfloat162_rn(buf[2 * t], buf[2 * t + 1]);
            *reinterpret_cast<uint4 *>(sX + tc::core_offset(r, i - 7, kIn)) = *reinterpret_cast<uint4 *>(p);
        }
    }
}

// Stage a row-major BF16 [R][K] matrix from global memory into the core layout.
__device__ __forceinline__ void stage_matrix(unsigned char *s, const __nv_bfloat16 *g, int R, int K) {
    for (int i = threadIdx.x; i < R * K / 8; i += blockDim.x) {
        const int r = (i * 8) / K, k = (i * 8) % K;
        *reinterpret_cast<uint4 *>(s + tc::core_offset(r, k, K)) = *reinterpret_cast<const uint4 *>(g + (size_t)r * K + k);
    }
}

// One layer: D = A (K wide) x W^T into TMEM, wait, and read the thread's row.
// Returns false (and records the error) if the MMA never completed.
__device__ __forceinline__ bool mma_layer(uint32_t tm, unsigned char *sA, unsigned char *sW, int K, uint64_t *bar,
                                          uint32_t &phase, float *out, unsigned *err) {
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        tc::gemm_128x64(tm, sA, sW, K, false);
        tc::mma_commit(bar);
    }
    // the decision must be the same in every thread, or later barriers would split the block
    const bool ok = __syncthreads_and(tc::mbar_wait(bar, phase, kWaitPolls)) != 0;
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(err, 1u);
        return false;
    }
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) tc::tmem_ld16(tm + ((uint32_t)(warp * 32) << 16) + c * 16, out + c * 16);
    tc::fence_before_sync();
    return true;
}

// Forward pass over queries (one thread per query row, 128 per tile, persistent
// CTAs).  mode 0: inference + gate (label where |w_hat - 1/2| > margin, the query
// lies outside the surface band and, when chi_gate is given, |w_hat - chi| <=
// chi_tol; else the query goes to the fallback list); mode 1: training (gathered samples, stores
// the features and activations, the loss, delta4 = dL/dz4 (ReLU mask applied),
// and the gradients of w5 and b5); mode 2: the raw output w_hat for every query.
// Gradients are summed across CTAs in 64-bit fixed point (units of 2^-40):
// integer addition does not depend on the order in which CTAs arrive, so a
// training run is bit-reproducible for a given seed (FP32 atomics were not).
// Range +-2^22 per entry, far above any gradient of this loss.
constexpr float kGradScale = 0x1p40f;
__device__ __forceinline__ void grad_add(long long *acc, float g) {
    atomicAdd(reinterpret_cast<unsigned long long *>(acc), (unsigned long long)__float2ll_rn(g * kGradScale));
}

__global__ void __launch_bounds__(128) k_mlp_forward(
    MlpDev P, const float *__restrict__ q, int64_t n, int mode, float margin,
    // inference outputs
    float *__restrict__ w_out, uint8_t *__restrict__ label, int32_t *__restrict__ fb_list,
    unsigned long long *__restrict__ fb_len, const int32_t *__restrict__ chi_gate, float chi_tol,
    // training
    const int64_t *__restrict__ sample_idx, const float *__restrict__ target, __nv_bfloat16 *__restrict__ Xs,
    __nv_bfloat16 *__restrict__ H, __nv_bfloat16 *__restrict__ D4, long long *__restrict__ grad,
    long long *__restrict__ loss,
    float inv_batch, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sW1 = smem + kSmemW1, *sW2 = smem + kSmemW2, *sW3 = smem + kSmemW3, *sW4 = smem + kSmemW4;
    // cross-warp sums of the training epilogue: in the upper half of the feature
    // buffer, unused once layer 1 has run (the activations take the lower half)
    float(*red)[kHid + 2] = reinterpret_cast<float(*)[kHid + 2]>(smem + kSmemX + 128 * kHid * 2);
    unsigned char *sX = smem + kSmemX, *sH = smem + kSmemH;
    float *sB = reinterpret_cast<float *>(smem + kSmemBias);
    stage_matrix(sW1, P.wbf, kHid, kIn);
    stage_matrix(sW2, P.wbf + kHid * kIn, kHid, kHid);
    stage_matrix(sW3, P.wbf + kHid * kIn + kHid * kHid, kHid, kHid);
    stage_matrix(sW4, P.wbf + kHid * kIn + 2 * kHid * kHid, kHid, kHid);
    for (int i = tid; i < kHid; i += blockDim.x) {
        sB[i] = P.params[oB1 + i];
        sB[kHid + i] = P.params[oB2 + i];
        sB[2 * kHid + i] = P.params[oB3 + i];
        sB[3 * kHid + i] = P.params[oB4 + i];
        sB[4 * kHid + i] = P.params[oW5 + i];
    }
    if (tid == 0) sB[5 * kHid] = P.params[oB5];
    if (warp == 0) tc::tmem_alloc(&tmem_base, 64);
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    uint32_t phase = 0;
    bool alive = true;
    const int64_t ntiles = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
        const int64_t row = tile * 128 + tid;
        const bool valid = row < n;
        int64_t src = row;
        if (mode == 1 && valid) src = sample_idx[row];
        const float qx = valid ? q[3 * src] : 0.f, qy = valid ? q[3 * src + 1] : 0.f,
                    qz = valid ? q[3 * src + 2] : 0.f;
        {
            features_to_smem(qx, qy, qz, P, sX, tid);
            if (mode == 1 && valid)
                for (int kc = 0; kc < kIn / 8; ++kc)
                    *reinterpret_cast<uint4 *>(Xs + (size_t)row * kIn + kc * 8) =
                        *reinterpret_cast<const uint4 *>(sX + tc::core_offset(tid, kc * 8, kIn));
        }
        unsigned char *sW[4] = {sW1, sW2, sW3, sW4};
        float h[kHid];
        for (int l = 0; l < 4 && alive; ++l) {
            alive = mma_layer(tm, l == 0 ? sX : sH, sW[l], l == 0 ? kIn : kHid, &bar, phase, h, err);
            if (!alive) break;
#pragma unroll
            for (int j = 0; j < kHid; ++j) h[j] = fmaxf(h[j] + sB[l * kHid + j], 0.f);
            // the MMA that read sH has completed: overwrite it with this layer's output
            store_row_bf16(sH, tid, h, kHid);
            if (mode == 1 && valid) {
#pragma unroll
                for (int kc = 0; kc < kHid / 8; ++kc) {
                    __nv_bfloat162 p[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(h[kc * 8 + 2 * i], h[kc * 8 + 2 * i + 1]);
                    *reinterpret_cast<uint4 *>(H + ((size_t)l * n + row) * kHid + kc * 8) =
                        *reinterpret_cast<uint4 *>(p);
                }
            }
        }
        if (!alive) break;
        // output layer (FP32 on the CUDA cores: a 64-wide dot product per query)
        float y = sB[5 * kHid];
#pragma unroll
        for (int j = 0; j < kHid; ++j) y = fmaf(sB[4 * kHid + j], h[j], y);
        if (mode == 2) {
            if (valid) w_out[row] = y;
        } else if (mode == 0) {
            if (valid) {
                if (fabsf(y - 0.5f) > margin && !in_band(P, qx, qy, qz) &&
                    (!chi_gate || fabsf(y - (float)chi_gate[row]) <= chi_tol)) {
                    w_out[row] = y;
                    label[row] = y > 0.5f ? 1 : 0;
                } else {
                    const unsigned long long slot = atomicAdd(fb_len, 1ull);
                    fb_list[slot] = (int32_t)row;
                }
            }
        } else {
            // dL/dy for L = mean (y - t)^2; dL/dh4 = dy * w5 (the ReLU mask of h4 is applied with h4 > 0)
            const float dy = valid ? 2.f * (y - target[src]) * inv_batch : 0.f;
            float d4[kHid];
#pragma unroll
            for (int j = 0; j < kHid; ++j) d4[j] = h[j] > 0.f ? dy * sB[4 * kHid + j] : 0.f;
            if (valid) {
#pragma unroll
                for (int kc = 0; kc < kHid / 8; ++kc) {
                    __nv_bfloat162 p[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(d4[kc * 8 + 2 * i], d4[kc * 8 + 2 * i + 1]);
                    *reinterpret_cast<uint4 *>(D4 + (size_t)row * kHid + kc * 8) = *reinterpret_cast<uint4 *>(p);
                }
            }
            // gradients of w5, b5 and the loss: warp sums, then one atomic per block
            const float e = valid ? (y - target[src]) : 0.f;
#pragma unroll
            for (int j = 0; j < kHid + 2; ++j) {
                float g = j < kHid ? dy * h[j] : (j == kHid ? dy : e * e * inv_batch);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                if (lane == 0) red[warp][j] = g;
            }
            __syncthreads();
            if (tid < kHid + 2) {
                const float g = red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
                if (tid < kHid) grad_add(&grad[oW5 + tid], g);
                else if (tid == kHid) grad_add(&grad[oB5], g);
                else grad_add(loss, g);
            }
            __syncthreads();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, 64);
}

// delta_{l-1}[b][k] = (sum_n delta_l[b][n] W_l[n][k]) * (h_{l-1}[b][k] > 0), one
// 128-row tile per CTA (layers 2..4, all 64 wide).  Also accumulates
// grad b_l = sum_b delta_l[b][.].
__global__ void __launch_bounds__(128) k_mlp_back_dx(const __nv_bfloat16 *__restrict__ Wl,
                                                      const __nv_bfloat16 *__restrict__ Dl,
                                                      const __nv_bfloat16 *__restrict__ Hprev, int64_t nb,
                                                      __nv_bfloat16 *__restrict__ Dprev, long long *__restrict__ grad_b,
                                                      unsigned *err) {
    __shared__ __align__(1024) unsigned char sA[128 * kHid * 2];
    __shared__ __align__(1024) unsigned char sWt[kHid * kHid * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float red[4][kHid];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row = (int64_t)blockIdx.x * 128 + tid;
    const bool valid = row < nb;
    // B operand rows k, K-index n: W_l^T
    for (int i = tid; i < kHid * kHid; i += blockDim.x) {
        const int nn = i / kHid, k = i % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sWt + tc::core_offset(k, nn, kHid)) = Wl[i];
    }
    float d[kHid];
#pragma unroll
    for (int j = 0; j < kHid; ++j) d[j] = valid ? __bfloat162float(Dl[row * kHid + j]) : 0.f;
    store_row_bf16(sA, tid, d, kHid);
    // grad of the bias of layer l
#pragma unroll
    for (int j = 0; j < kHid; ++j) {
        float g = d[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) red[warp][j] = g;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 64);
    if (tid == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    if (tid < kHid) grad_add(&grad_b[tid], red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid]);
    uint32_t phase = 0;
    float out[kHid];
    const bool ok = mma_layer(tmem_base, sA, sWt, kHid, &bar, phase, out, err);
    if (ok && valid) {
        float v[kHid];
#pragma unroll
        for (int j = 0; j < kHid; ++j) v[j] = __bfloat162float(Hprev[row * kHid + j]) > 0.f ? out[j] : 0.f;
#pragma unroll
        for (int kc = 0; kc < kHid / 8; ++kc) {
            __nv_bfloat162 p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[kc * 8 + 2 * i], v[kc * 8 + 2 * i + 1]);
            *reinterpret_cast<uint4 *>(Dprev + row * kHid + kc * 8) = *reinterpret_cast<uint4 *>(p);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, 64);
}

// grad W_l[n][k] += sum_b delta_l[b][n] h_{l-1}[b][k] over a chunk of the batch:
// D[k][n] (TMEM, 128 x 64; k < K_l, rows past K_l are zero padding) with
// A[k][b] = h_{l-1}[b][k] and B[n][b] = delta_l[b][n] staged transposed, the
// batch chunk as the reduction dimension (kChunkB rows per MMA chain).
constexpr int kChunkB = 128;
__global__ void __launch_bounds__(128) k_mlp_back_dw(const __nv_bfloat16 *__restrict__ Hprev, int Kl,
                                                      const __nv_bfloat16 *__restrict__ Dl, int64_t nb,
                                                      int64_t rows_per_cta, long long *__restrict__ gradW,
                                                      unsigned *err) {
    __shared__ __align__(1024) unsigned char sA[128 * kChunkB * 2];
    __shared__ __align__(1024) unsigned char sB[kHid * kChunkB * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc::tmem_alloc(&tmem_base, 64);
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    uint32_t phase = 0;
    const int64_t b0 = (int64_t)blockIdx.x * rows_per_cta, b1 = min(nb, b0 + rows_per_cta);
    bool first = true, ok = true;
    for (int64_t c0 = b0; c0 < b1 && ok; c0 += kChunkB) {
        // stage: thread t owns batch column (c0 + t); writes its column of A (K_l rows) and B (64 rows)
        const int64_t b = c0 + tid;
        const bool valid = b < b1;
        for (int k = 0; k < 128; ++k) {
            const __nv_bfloat16 hv = (valid && k < Kl) ? Hprev[b * Kl + k] : __float2bfloat16(0.f);
            *reinterpret_cast<__nv_bfloat16 *>(sA + tc::core_offset(k, tid, kChunkB)) = hv;
        }
        for (int nn = 0; nn < kHid; ++nn) {
            const __nv_bfloat16 dv = valid ? Dl[b * kHid + nn] : __float2bfloat16(0.f);
            *reinterpret_cast<__nv_bfloat16 *>(sB + tc::core_offset(nn, tid, kChunkB)) = dv;
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            tc::gemm_128x64(tm, sA, sB, kChunkB, !first);
            tc::mma_commit(&bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&bar, phase, kWaitPolls)) != 0;
        phase ^= 1u;
        tc::fence_after_sync();
        first = false;
        if (!ok && tid == 0) atomicOr(err, 1u);
    }
    if (ok && !first) {
        // thread t holds row k = t of D: grad W_l[n][k] += D[k][n]
        float out[kHid];
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::tmem_ld16(tm + ((uint32_t)(warp * 32) << 16) + c * 16, out + c * 16);
        if (tid < Kl)
#pragma unroll
            for (int nn = 0; nn < kHid; ++nn) grad_add(&gradW[nn * Kl + tid], out[nn]);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, 64);
}

// grad b[n] += sum_b delta[b][n] (the bias of layer 1)
__global__ void k_colsum64(const __nv_bfloat16 *__restrict__ Dl, int64_t nb, long long *__restrict__ grad_b) {
    __shared__ float red[4][kHid];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row = (int64_t)blockIdx.x * 128 + tid;
#pragma unroll 8
    for (int j = 0; j < kHid; ++j) {
        float g = row < nb ? __bfloat162float(Dl[row * kHid + j]) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) red[warp][j] = g;
    }
    __syncthreads();
    if (tid < kHid) grad_add(&grad_b[tid], red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid]);
}

// The fixed-point sums of one step to FP32 (gradient and loss), clearing them
// for the next step.
__global__ void k_grad_to_float(long long *__restrict__ acc, float *__restrict__ grad, float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kParams) return;
    const float v = (float)((double)acc[i] * (1.0 / (double)kGradScale));
    if (i < kParams) grad[i] = v;
    else *loss = v;
    acc[i] = 0;
}

// Adam step on the FP32 master weights (bias-corrected moments), then the BF16
// copies of W1..W4; clears the gradient.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, float *__restrict__ g,
                       __nv_bfloat16 *__restrict__ wbf, float lr, float b1, float b2, float eps, float c1, float c2,
                       int do_update) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float pi = p[i];
    if (do_update) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        pi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        g[i] = 0.f;
    }
    int wi = -1;
    if (i < oB1) wi = i;
    else if (i >= oW2 && i < oB2) wi = kHid * kIn + (i - oW2);
    else if (i >= oW3 && i < oB3) wi = kHid * kIn + kHid * kHid + (i - oW3);
    else if (i >= oW4 && i < oB4) wi = kHid * kIn + 2 * kHid * kHid + (i - oW4);
    if (wi >= 0) wbf[wi] = __float2bfloat16(pi);
}

// Counter-based generator (SplitMix64 finaliser) for initial weights and batch
// indices: uniform in [0, 1) from (seed, stream, index).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t seed, uint64_t stream, uint64_t i) {
    return (double)(mix64(seed ^ mix64(stream * 0x100000001B3ull + i)) >> 11) * (1.0 / 9007199254740992.0);
}

// He-normal weights (Box-Muller), zero biases.
__global__ void k_mlp_init(float *__restrict__ p, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float fan_in = 0.f;
    if (i < oB1) fan_in = kIn;
    else if ((i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) || (i >= oW4 && i < oB4) || (i >= oW5 && i < oB5))
        fan_in = kHid;
    if (fan_in == 0.f) {
        p[i] = 0.f;
        return;
    }
    const double u1 = fmax(u01(seed, 1, i), 1e-300), u2 = u01(seed, 2, i);
    const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    p[i] = (float)(z * sqrt(2.0 / fan_in) * (i >= oW5 ? 0.5 : 1.0));
}

__global__ void k_batch_indices(int64_t *__restrict__ idx, int64_t nb, int64_t n, uint64_t seed, uint64_t step) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    idx[i] = (int64_t)(u01(seed, 3 + step, (uint64_t)i) * (double)n) % n;
}

__global__ void k_iota64(int64_t *__restrict__ idx, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) idx[i] = i;
}

__global__ void k_gather_i32(const int32_t *__restrict__ v, const int32_t *__restrict__ list,
                             const unsigned long long *__restrict__ len, int32_t *__restrict__ out) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *len) return;
    out[i] = v[list[i]];
}

__global__ void k_gather3(const float *__restrict__ q, const int32_t *__restrict__ list,
                          const unsigned long long *__restrict__ len, float *__restrict__ out) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *len) return;
    const int32_t j = list[i];
    out[3 * i] = q[3 * j];
    out[3 * i + 1] = q[3 * j + 1];
    out[3 * i + 2] = q[3 * j + 2];
}

__global__ void k_scatter_wl(const int32_t *__restrict__ list, const unsigned long long *__restrict__ len,
                             const float *__restrict__ w_in, const uint8_t *__restrict__ l_in, float *__restrict__ w,
                             uint8_t *__restrict__ label) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *len) return;
    const int32_t j = list[i];
    w[j] = w_in[i];
    label[j] = l_in[i];
}

// C[128][64] = A[128][K] x B[64][K]^T with A, B row-major BF16 in global memory.
__global__ void __launch_bounds__(128) k_tc_selftest(const __nv_bfloat16 *__restrict__ A,
                                                      const __nv_bfloat16 *__restrict__ B, int K,
                                                      float *__restrict__ C, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    unsigned char *sA = smem;
    unsigned char *sB = smem + 128 * K * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 128 * K; i += blockDim.x)
        *reinterpret_cast<__nv_bfloat16 *>(sA + tc::core_offset(i / K, i % K, K)) = A[i];
    for (int i = tid; i < 64 * K; i += blockDim.x)
        *reinterpret_cast<__nv_bfloat16 *>(sB + tc::core_offset(i / K, i % K, K)) = B[i];
    if (warp == 0) tc::tmem_alloc(&tmem_base, 64);
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = tmem_base;
    if (tid == 0) {
        tc::gemm_128x64(tm, sA, sB, K, false);
        tc::mma_commit(&bar);
    }
    const bool ok = tc::mbar_wait(&bar, 0, kWaitPolls);
    if (!ok && lane == 0) atomicOr(err, 1u);
    tc::fence_after_sync();
    if (ok) {
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tc::tmem_ld16(tm + ((uint32_t)(warp * 32) << 16) + c * 16, v);
            for (int i = 0; i < 16; ++i) C[(warp * 32 + lane) * 64 + c * 16 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, 64);
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

bool g_freq_set[64] = {};

gwn_status set_freq_table() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && g_freq_set[dev]) return GWN_OK;
    float f[kNFreq];
    for (int k = 0; k < kNFreq; ++k) f[k] = (float)std::exp2(7.0 * k / 15.0);
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_freq, f, sizeof(f)));
    if (dev >= 0 && dev < 64) g_freq_set[dev] = true;
    return GWN_OK;
}

// Mark the cells overlapped by each triangle's bounding box.
__global__ void k_band_mark(const float *__restrict__ tri9, int64_t nt, MlpDev P, uint32_t *__restrict__ bits) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int R = P.band_res;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        const float a = tri9[9 * t + d], b = tri9[9 * t + 3 + d], c = tri9[9 * t + 6 + d];
        const float mn = (fmaf(fminf(a, fminf(b, c)), P.scale[d], P.offset[d]) + 1.f) * 0.5f * (float)R;
        const float mx = (fmaf(fmaxf(a, fmaxf(b, c)), P.scale[d], P.offset[d]) + 1.f) * 0.5f * (float)R;
        if (!(mx >= 0.f && mn < (float)R)) return;    // outside the box (or NaN)
        lo[d] = (int)floorf(fmaxf(mn, 0.f));
        hi[d] = (int)floorf(fminf(mx, (float)(R - 1)));
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                const int64_t c = ((int64_t)z * R + y) * R + x;
                atomicOr(&bits[c >> 5], 1u << (c & 31));
            }
}

// out = cells within Chebyshev distance r of a marked cell of in.
__global__ void k_band_dilate(const uint32_t *__restrict__ in, int R, int r, uint32_t *__restrict__ out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ncell = (int64_t)R * R * R;
    const bool inside = c < ncell;   // no early exit: the whole warp takes part in the ballot
    const int x = (int)(c % R), y = (int)((c / R) % R), z = (int)(c / ((int64_t)R * R));
    bool hit = false;
    for (int dz = -r; dz <= r && !hit && inside; ++dz)
        for (int dy = -r; dy <= r && !hit; ++dy)
            for (int dx = -r; dx <= r && !hit; ++dx) {
                const int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx < 0 || yy < 0 || zz < 0 || xx >= R || yy >= R || zz >= R) continue;
                const int64_t k = ((int64_t)zz * R + yy) * R + xx;
                hit = (in[k >> 5] >> (k & 31)) & 1u;
            }
    const unsigned ball = __ballot_sync(0xffffffffu, hit);
    // a warp covers 32 consecutive cells starting at a multiple of 32: one word
    if ((threadIdx.x & 31) == 0 && inside) out[c >> 5] = ball;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: the surrogate attached to a mesh.
// ---------------------------------------------------------------------------
struct Surrogate {
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    long long *gacc = nullptr;   // [kParams + 1] fixed-point gradient and loss of one step (zero between steps)
    __nv_bfloat16 *wbf = nullptr;
    unsigned *err = nullptr;
    float lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    int64_t steps = 0;
    bool trained = false;
    gwn_mlp_config cfg{};
    // training buffers
    int64_t cap_b = 0;
    int64_t *idx = nullptr;
    __nv_bfloat16 *Xs = nullptr, *H = nullptr, *D[2] = {nullptr, nullptr};
    // surface band of the gate
    uint32_t *band = nullptr;
    int band_res = 0;
};

void surrogate_free(Surrogate *s) {
    if (!s) return;
    for (void *p : {(void *)s->params, (void *)s->m, (void *)s->v, (void *)s->grad, (void *)s->loss, (void *)s->gacc,
                    (void *)s->wbf,
                    (void *)s->err, (void *)s->idx, (void *)s->Xs, (void *)s->H, (void *)s->D[0], (void *)s->D[1],
                    (void *)s->band})
        if (p) cudaFree(p);
    delete s;
}

static MlpDev mlp_dev(const Surrogate *s) {
    MlpDev P;
    P.wbf = s->wbf;
    P.params = s->params;
    for (int d = 0; d < 3; ++d) {
        const float ext = s->hi[d] - s->lo[d];
        P.scale[d] = ext > 0.f ? 2.f / ext : 0.f;
        P.offset[d] = ext > 0.f ? -1.f - 2.f * s->lo[d] / ext : 0.f;
    }
    P.band = s->band;
    P.band_res = s->band_res;
    return P;
}

// (Re)build the surface band over the surrogate's box from the mesh triangles.
static gwn_status build_band(gwn_mesh *m, cudaStream_t st) {
    Surrogate *s = m->sur;
    if (s->band) cudaFree(s->band);
    s->band = nullptr;
    s->band_res = 0;
    const int R = s->cfg.band_res;
    if (R <= 0 || m->nt == 0) return GWN_OK;
    const int64_t ncell = (int64_t)R * R * R, nwords = (ncell + 31) / 32;
    uint32_t *marked = nullptr, *band = nullptr;
    GWN_CUDA_TRY(cudaMalloc(&band, sizeof(uint32_t) * nwords));
    GWN_CUDA_TRY(cudaMallocAsync(&marked, sizeof(uint32_t) * nwords, st));
    cudaMemsetAsync(marked, 0, sizeof(uint32_t) * nwords, st);
    MlpDev P = mlp_dev(s);
    P.band_res = R;
    k_band_mark<<<grid_for(m->nt, 256), 256, 0, st>>>(m->tri9, m->nt, P, marked);
    const int r = s->cfg.band_dilate < 0 ? 0 : s->cfg.band_dilate;
    k_band_dilate<<<grid_for(ncell, 256), 256, 0, st>>>(marked, R, r, band);
    cudaFreeAsync(marked, st);
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
    GWN_LAUNCH_CHECK("surface band");
    s->band = band;
    s->band_res = R;
    return GWN_OK;
}

static gwn_status ensure_surrogate(gwn_mesh *m) {
    if (m->sur) return GWN_OK;
    Surrogate *s = new Surrogate();
    cudaError_t e;
    if ((e = cudaMalloc(&s->params, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&s->m, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&s->v, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&s->grad, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&s->loss, sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&s->gacc, sizeof(long long) * (kParams + 1))) != cudaSuccess ||
        (e = cudaMemset(s->gacc, 0, sizeof(long long) * (kParams + 1))) != cudaSuccess ||
        (e = cudaMalloc(&s->wbf, sizeof(__nv_bfloat16) * kWbf)) != cudaSuccess ||
        (e = cudaMalloc(&s->err, sizeof(unsigned))) != cudaSuccess) {
        surrogate_free(s);
        return set_error(GWN_ERR_OOM, cudaGetErrorString(e));
    }
    cudaMemset(s->m, 0, sizeof(float) * kParams);
    cudaMemset(s->v, 0, sizeof(float) * kParams);
    cudaMemset(s->grad, 0, sizeof(float) * kParams);
    cudaMemset(s->err, 0, sizeof(unsigned));
    m->sur = s;
    return set_freq_table();
}

static gwn_status ensure_batch_buffers(Surrogate *s, int64_t nb) {
    if (nb <= s->cap_b) return GWN_OK;
    for (void *p : {(void *)s->idx, (void *)s->Xs, (void *)s->H, (void *)s->D[0], (void *)s->D[1]})
        if (p) cudaFree(p);
    GWN_CUDA_TRY(cudaMalloc(&s->idx, sizeof(int64_t) * nb));
    GWN_CUDA_TRY(cudaMalloc(&s->Xs, sizeof(__nv_bfloat16) * nb * kIn));
    GWN_CUDA_TRY(cudaMalloc(&s->H, sizeof(__nv_bfloat16) * nb * kHid * 4));
    GWN_CUDA_TRY(cudaMalloc(&s->D[0], sizeof(__nv_bfloat16) * nb * kHid));
    GWN_CUDA_TRY(cudaMalloc(&s->D[1], sizeof(__nv_bfloat16) * nb * kHid));
    s->cap_b = nb;
    return GWN_OK;
}

// Forward + backward on nb samples (indices in s->idx): the gradient into s->grad
// and the loss (mean squared error) into s->loss, summed in fixed point across
// CTAs (s->gacc, left zero) so that the result does not depend on their order.
static gwn_status mlp_fwd_bwd(Surrogate *s, const float *q, const float *target, int64_t nb, cudaStream_t st) {
    const MlpDev P = mlp_dev(s);
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
    const int64_t ntiles = (nb + 127) / 128;
    const int grid = (int)std::min<int64_t>(ntiles, 3 * sm_count());
    k_mlp_forward<<<grid, 128, kSmemFwd, st>>>(P, q, nb, 1, 0.f, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f,
                                               s->idx, target,
                                               s->Xs, s->H, s->D[0], s->gacc, s->gacc + kParams, 1.f / (float)nb,
                                               s->err);
    // layers 4, 3, 2: delta_{l-1} and the grads of W_l, b_l
    const __nv_bfloat16 *Wbf[4] = {s->wbf, s->wbf + kHid * kIn, s->wbf + kHid * kIn + kHid * kHid,
                                   s->wbf + kHid * kIn + 2 * kHid * kHid};
    const int oW[4] = {oW1, oW2, oW3, oW4}, oB[4] = {oB1, oB2, oB3, oB4};
    int cur = 0;
    const int64_t rows_per_cta = 1024;
    const unsigned dw_grid = (unsigned)((nb + rows_per_cta - 1) / rows_per_cta);
    for (int l = 3; l >= 0; --l) {
        const __nv_bfloat16 *Hprev = l == 0 ? s->Xs : s->H + (size_t)(l - 1) * nb * kHid;
        const int Kl = l == 0 ? kIn : kHid;
        k_mlp_back_dw<<<dw_grid, 128, 0, st>>>(Hprev, Kl, s->D[cur], nb, rows_per_cta, s->gacc + oW[l], s->err);
        if (l > 0) {
            k_mlp_back_dx<<<(unsigned)ntiles, 128, 0, st>>>(Wbf[l], s->D[cur], Hprev, nb, s->D[cur ^ 1],
                                                            s->gacc + oB[l], s->err);
            cur ^= 1;
        } else {
            k_colsum64<<<(unsigned)ntiles, 128, 0, st>>>(s->D[cur], nb, s->gacc + oB[0]);
        }
    }
    k_grad_to_float<<<grid_for(kParams + 1, 256), 256, 0, st>>>(s->gacc, s->grad, s->loss);
    GWN_LAUNCH_CHECK("mlp forward/backward");
    return GWN_OK;
}

namespace {

__device__ __forceinline__ int okey(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void k_bbox(const float *__restrict__ q, int64_t n, int *__restrict__ box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int d = 0; d < 3; ++d) {
        int lo = 0x7fffffff, hi = (int)0x80000000;
        if (i < n) lo = hi = okey(q[3 * i + d]);
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

__global__ void k_count_surrogate(unsigned long long *counters, unsigned long long n,
                                  const unsigned long long *__restrict__ fb_len) {
    if (threadIdx.x == 0) {
        counters[CNT_SUR_QUERIES] += n;
        counters[CNT_SUR_FALLBACK] += *fb_len;
    }
}

// Confidence |w_hat - 1/2| of the misclassified samples, binned by 1/2048 over [0, 2).
constexpr int kCalibBins = 4096;
__global__ void k_calib_hist(MlpDev P, const float *__restrict__ q, const float *__restrict__ w_hat,
                             const uint8_t *__restrict__ label, const int32_t *__restrict__ chi, float chi_tol,
                             int64_t n, unsigned long long *__restrict__ hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (in_band(P, q[3 * i], q[3 * i + 1], q[3 * i + 2])) return;   // never answered by the network
    if (chi_tol >= 0.f && fabsf(w_hat[i] - (float)chi[i]) > chi_tol) return;   // nor by the chi test
    const float y = w_hat[i];
    const bool says_in = y > 0.5f;
    if (says_in == (label[i] != 0)) return;
    const int b = min(kCalibBins - 1, (int)(fabsf(y - 0.5f) * 2048.f));
    atomicAdd(&hist[b], 1ull);
}

float from_okey(int k) {
    const int i = k >= 0 ? k : k ^ 0x7fffffff;
    float f;
    std::memcpy(&f, &i, 4);
    return f;
}

gwn_status check_err(Surrogate *s, cudaStream_t st) {
    unsigned h = 0;
    GWN_CUDA_TRY(cudaMemcpyAsync(&h, s->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(s->err, 0, sizeof(unsigned), st);
        return set_error(GWN_ERR_CUDA, "surrogate: a tensor-core MMA did not complete (wait limit reached)");
    }
    return GWN_OK;
}

gwn_mlp_config defaults(const gwn_mlp_config *c) {
    gwn_mlp_config d{};
    if (c) d = *c;
    if (d.steps <= 0) d.steps = 3000;
    if (d.batch <= 0) d.batch = 16384;
    if (d.lr <= 0.f) d.lr = 1e-3f;
    if (d.margin <= 0.f) d.margin = 0.1f;
    if (d.beta1 <= 0.f) d.beta1 = 0.9f;
    if (d.beta2 <= 0.f) d.beta2 = 0.999f;
    if (d.eps <= 0.f) d.eps = 1e-8f;
    if (d.band_res == 0) d.band_res = 256;
    if (d.band_res > 1024) d.band_res = 1024;
    if (d.band_dilate == 0) d.band_dilate = 1;
    if (d.chi_tol == 0.f) d.chi_tol = 0.25f;
    return d;
}

}  // namespace

bool surrogate_ready(const gwn_mesh *m) { return m->sur && m->sur->trained; }

// Labels and w through the surrogate: confident queries (|w_hat - 1/2| > margin,
// outside the surface band, w_hat within chi_tol of the exact crossing count)
// are answered by the network, the rest are compacted, evaluated by the exact
// path (their crossing counts already known; boundary sum, FP64 re-evaluation
// near 1/2) and scattered back.  Device pointers; synchronises once to size
// the fallback launch.
gwn_status classify_with_surrogate(const gwn_mesh *m, const float *q, int64_t n, uint8_t *label, float *w,
                                   cudaStream_t st) {
    Surrogate *s = m->sur;
    const MlpDev P = mlp_dev(s);
    int32_t *list = nullptr, *chi_all = nullptr;
    unsigned long long *len = nullptr;
    const bool chi_test = s->cfg.chi_tol >= 0.f;
    GWN_CUDA_TRY(cudaMallocAsync(&list, sizeof(int32_t) * n, st));
    GWN_CUDA_TRY(cudaMallocAsync(&len, sizeof(unsigned long long), st));
    GWN_CUDA_TRY(cudaMemsetAsync(len, 0, sizeof(unsigned long long), st));
    if (chi_test) {
        GWN_CUDA_TRY(cudaMallocAsync(&chi_all, sizeof(int32_t) * n, st));
        if (gwn_status r0 = launch_chi(m, q, n, chi_all, st)) {
            cudaFreeAsync(chi_all, st);
            cudaFreeAsync(list, st);
            cudaFreeAsync(len, st);
            return r0;
        }
    }
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
    {
        ProfScope prof("surrogate_forward", st);
        const int64_t ntiles = (n + 127) / 128;
        const int grid = (int)std::min<int64_t>(ntiles, 3 * sm_count());
        k_mlp_forward<<<grid, 128, kSmemFwd, st>>>(P, q, n, 0, s->cfg.margin, w, label, list, len, chi_all,
                                                   s->cfg.chi_tol, nullptr, nullptr,
                                                   nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, s->err);
    }
    unsigned long long nfb = 0;
    GWN_CUDA_TRY(cudaMemcpyAsync(&nfb, len, sizeof(nfb), cudaMemcpyDeviceToHost, st));
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
    k_count_surrogate<<<1, 32, 0, st>>>(m->counters, (unsigned long long)n, len);
    gwn_status r = check_err(s, st);
    if (r == GWN_OK && nfb > 0) {
        float *qf = nullptr, *wf = nullptr;
        uint8_t *lf = nullptr;
        int32_t *cf = nullptr, *l2 = nullptr;
        unsigned long long *len2 = nullptr;
        GWN_CUDA_TRY(cudaMallocAsync(&qf, sizeof(float) * 3 * nfb, st));
        GWN_CUDA_TRY(cudaMallocAsync(&wf, sizeof(float) * nfb, st));
        GWN_CUDA_TRY(cudaMallocAsync(&lf, nfb, st));
        GWN_CUDA_TRY(cudaMallocAsync(&cf, sizeof(int32_t) * nfb, st));
        GWN_CUDA_TRY(cudaMallocAsync(&l2, sizeof(int32_t) * nfb, st));
        GWN_CUDA_TRY(cudaMallocAsync(&len2, sizeof(unsigned long long), st));
        GWN_CUDA_TRY(cudaMemsetAsync(len2, 0, sizeof(unsigned long long), st));
        const unsigned g = grid_for((int64_t)nfb, 256);
        const int64_t nf = (int64_t)nfb;
        // the fallback queries in Morton order (the atomic compaction scrambled them)
        r = order_query_list(m, q, list, nf, st);
        if (r == GWN_OK) {
            k_gather3<<<g, 256, 0, st>>>(q, list, len, qf);
            if (chi_test) k_gather_i32<<<g, 256, 0, st>>>(chi_all, list, len, cf);
        }
        if (r == GWN_OK && (r = chi_test ? GWN_OK : launch_chi(m, qf, nf, cf, st)) == GWN_OK &&
            (r = launch_boundary_sum_list(m, qf, nf, cf, wf, lf, true, l2, len2, st)) == GWN_OK &&
            (r = launch_fp64_fix_list(m, qf, cf, wf, lf, l2, len2, st)) == GWN_OK)
            k_scatter_wl<<<g, 256, 0, st>>>(list, len, wf, lf, w, label);
        for (void *p : {(void *)qf, (void *)wf, (void *)lf, (void *)cf, (void *)l2, (void *)len2}) cudaFreeAsync(p, st);
    }
    cudaFreeAsync(list, st);
    cudaFreeAsync(len, st);
    if (chi_all) cudaFreeAsync(chi_all, st);
    if (r != GWN_OK) return r;
    GWN_LAUNCH_CHECK("surrogate classify");
    return GWN_OK;
}

}  // namespace gwn

using namespace gwn;

extern "C" {

gwn_status gwn_debug_tc_gemm(const void *A, const void *B, int32_t K, float *C, void *stream) {
    clear_error();
    if (!A || !B || !C) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    if (K != 64 && K != 128) return set_error(GWN_ERR_INVALID_ARG, "K must be 64 or 128");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *err = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&err, sizeof(unsigned), s));
    GWN_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    // operands plus slack so that every address a descriptor can form stays inside the allocation
    const size_t smem = (size_t)(128 + 64) * K * 2 + 32768;
    cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tc_selftest<<<1, 128, smem, s>>>((const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, K, C, err);
    unsigned h = 0;
    cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    GWN_CUDA_TRY(cudaStreamSynchronize(s));
    GWN_LAUNCH_CHECK("k_tc_selftest");
    if (h) return set_error(GWN_ERR_CUDA, "tensor-core self-test: mbarrier wait timed out");
    return GWN_OK;
}

int32_t gwn_surrogate_num_params(void) { return kParams; }

gwn_status gwn_surrogate_train(gwn_mesh *m, const float *samples, const float *targets, int64_t n,
                               const gwn_mlp_config *cfg, float *final_loss, void *stream) {
    clear_error();
    if (!m || !samples || n <= 0) return set_error(GWN_ERR_INVALID_ARG, "mesh, samples and n > 0 are required");
    if (n > (int64_t)0x7fffffff) return set_error(GWN_ERR_INVALID_ARG, "at most 2^31-1 samples");
    if (!targets && !m->built) return set_error(GWN_ERR_NOT_BUILT, "labelling needs gwn_build_accel");
    if (gwn_status e = check_device_buffers(m->device, {samples, targets}, "gwn_surrogate_train")) return e;
    DeviceScope dev_scope(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    gwn_status r = ensure_surrogate(m);
    if (r != GWN_OK) return r;
    Surrogate *s = m->sur;
    s->cfg = defaults(cfg);
    const int64_t nb = std::min<int64_t>(s->cfg.batch, n);
    if ((r = ensure_batch_buffers(s, nb)) != GWN_OK) return r;
    // input box of the samples
    int *box = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&box, sizeof(int) * 6, st));
    const int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
    GWN_CUDA_TRY(cudaMemcpyAsync(box, init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_bbox<<<grid_for(n, 256), 256, 0, st>>>(samples, n, box);
    int hbox[6];
    GWN_CUDA_TRY(cudaMemcpyAsync(hbox, box, sizeof(hbox), cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(box, st);
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
    for (int d = 0; d < 3; ++d) {
        s->lo[d] = from_okey(hbox[d]);
        s->hi[d] = from_okey(hbox[3 + d]);
    }
    // labels from the antipodal path when none are given
    float *tgt = const_cast<float *>(targets), *own = nullptr;
    if (!tgt) {
        int32_t *chi = nullptr;
        GWN_CUDA_TRY(cudaMallocAsync(&own, sizeof(float) * n, st));
        GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, st));
        if ((r = launch_chi(m, samples, n, chi, st)) == GWN_OK)
            r = launch_boundary_sum_list(m, samples, n, chi, own, nullptr, false, nullptr, nullptr, st);
        cudaFreeAsync(chi, st);
        if (r != GWN_OK) return r;
        tgt = own;
    }
    k_mlp_init<<<grid_for(kParams, 256), 256, 0, st>>>(s->params, s->cfg.seed);
    cudaMemsetAsync(s->m, 0, sizeof(float) * kParams, st);
    cudaMemsetAsync(s->v, 0, sizeof(float) * kParams, st);
    cudaMemsetAsync(s->grad, 0, sizeof(float) * kParams, st);
    k_adam<<<grid_for(kParams, 256), 256, 0, st>>>(s->params, s->m, s->v, s->grad, s->wbf, 0.f, 0.f, 0.f, 1.f, 1.f,
                                                     1.f, 0);
    s->steps = 0;
    {
        ProfScope prof("surrogate_train", st);
        for (int it = 0; it < s->cfg.steps; ++it) {
            k_batch_indices<<<grid_for(nb, 256), 256, 0, st>>>(s->idx, nb, n, s->cfg.seed, (uint64_t)it);
            if ((r = mlp_fwd_bwd(s, samples, tgt, nb, st)) != GWN_OK) break;
            ++s->steps;
            const float c1 = 1.f - std::pow(s->cfg.beta1, (float)s->steps);
            const float c2 = 1.f - std::pow(s->cfg.beta2, (float)s->steps);
            k_adam<<<grid_for(kParams, 256), 256, 0, st>>>(s->params, s->m, s->v, s->grad, s->wbf, s->cfg.lr,
                                                             s->cfg.beta1, s->cfg.beta2, s->cfg.eps, c1, c2, 1);
        }
    }
    if (own) cudaFreeAsync(own, st);
    if (r != GWN_OK) return r;
    GWN_LAUNCH_CHECK("surrogate training");
    if ((r = check_err(s, st)) != GWN_OK) return r;
    if (final_loss) {
        GWN_CUDA_TRY(cudaMemcpyAsync(final_loss, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        GWN_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if ((r = build_band(m, st)) != GWN_OK) return r;
    s->trained = true;
    return GWN_OK;
}

gwn_status gwn_surrogate_predict(const gwn_mesh *m, const float *q, int64_t n, float *w_hat, void *stream) {
    clear_error();
    if (!m || !m->sur) return set_error(GWN_ERR_INVALID_ARG, "mesh has no surrogate");
    if (n < 0 || (n > 0 && (!q || !w_hat))) return set_error(GWN_ERR_INVALID_ARG, "q / w_hat");
    if (n == 0) return GWN_OK;
    if (gwn_status e = check_device_buffers(m->device, {q, w_hat}, "gwn_surrogate_predict")) return e;
    DeviceScope dev_scope(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    Surrogate *s = m->sur;
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
    const int64_t ntiles = (n + 127) / 128;
    const int grid = (int)std::min<int64_t>(ntiles, 3 * sm_count());
    k_mlp_forward<<<grid, 128, kSmemFwd, st>>>(mlp_dev(s), q, n, 2, 0.f, w_hat, nullptr, nullptr, nullptr, nullptr, 0.f,
                                               nullptr,
                                               nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, s->err);
    GWN_LAUNCH_CHECK("surrogate predict");
    return check_err(s, st);
}

// get (set = 0) or set (set = 1) the FP32 parameters and the input box [lo, hi]
gwn_status gwn_surrogate_params(gwn_mesh *m, float *params, float *box, int32_t set) {
    clear_error();
    if (!m || !params) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    if (set) {
        gwn_status r = ensure_surrogate(m);
        if (r != GWN_OK) return r;
    } else if (!m->sur) {
        return set_error(GWN_ERR_INVALID_ARG, "mesh has no surrogate");
    }
    Surrogate *s = m->sur;
    if (set) {
        GWN_CUDA_TRY(cudaMemcpy(s->params, params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
        if (box)
            for (int d = 0; d < 3; ++d) {
                s->lo[d] = box[d];
                s->hi[d] = box[3 + d];
            }
        if (s->cfg.margin <= 0.f) s->cfg = defaults(nullptr);
        k_adam<<<grid_for(kParams, 256), 256, 0>>>(s->params, s->m, s->v, s->grad, s->wbf, 0.f, 0.f, 0.f, 1.f, 1.f,
                                                   1.f, 0);
        GWN_CUDA_TRY(cudaDeviceSynchronize());
        gwn_status r = build_band(m, 0);
        if (r != GWN_OK) return r;
        s->trained = true;
    } else {
        GWN_CUDA_TRY(cudaMemcpy(params, s->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
        if (box)
            for (int d = 0; d < 3; ++d) {
                box[d] = s->lo[d];
                box[3 + d] = s->hi[d];
            }
    }
    return GWN_OK;
}

gwn_status gwn_surrogate_grad(gwn_mesh *m, const float *q, const float *target, int64_t n, float *grad, float *loss,
                              void *stream) {
    clear_error();
    if (!m || !m->sur) return set_error(GWN_ERR_INVALID_ARG, "mesh has no surrogate");
    if (!q || !target || !grad || n <= 0 || n > (1 << 22)) return set_error(GWN_ERR_INVALID_ARG, "arguments");
    if (gwn_status e = check_device_buffers(m->device, {q, target}, "gwn_surrogate_grad")) return e;
    DeviceScope dev_scope(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    Surrogate *s = m->sur;
    gwn_status r = ensure_batch_buffers(s, n);
    if (r != GWN_OK) return r;
    k_iota64<<<grid_for(n, 256), 256, 0, st>>>(s->idx, n);
    if ((r = mlp_fwd_bwd(s, q, target, n, st)) != GWN_OK) return r;
    GWN_CUDA_TRY(cudaMemcpyAsync(grad, s->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, st));
    if (loss) GWN_CUDA_TRY(cudaMemcpyAsync(loss, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    GWN_CUDA_TRY(cudaMemsetAsync(s->grad, 0, sizeof(float) * kParams, st));
    return check_err(s, st);
}

// Checkpoint: magic, version, parameter count, steps, box, config, parameters,
// Adam moments (so training can resume).
gwn_status gwn_surrogate_save(const gwn_mesh *m, const char *path) {
    clear_error();
    if (!m || !m->sur || !path) return set_error(GWN_ERR_INVALID_ARG, "mesh has no surrogate / path");
    Surrogate *s = m->sur;
    std::vector<float> p(kParams), mm(kParams), vv(kParams);
    GWN_CUDA_TRY(cudaMemcpy(p.data(), s->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    GWN_CUDA_TRY(cudaMemcpy(mm.data(), s->m, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    GWN_CUDA_TRY(cudaMemcpy(vv.data(), s->v, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(GWN_ERR_INVALID_ARG, std::string("cannot write ") + path);
    const uint32_t head[4] = {0x534E5747u /* "GWNS" */, 1u, (uint32_t)kParams, 0u};
    std::fwrite(head, sizeof(head), 1, f);
    std::fwrite(&s->steps, sizeof(s->steps), 1, f);
    std::fwrite(s->lo, sizeof(float), 3, f);
    std::fwrite(s->hi, sizeof(float), 3, f);
    std::fwrite(&s->cfg, sizeof(s->cfg), 1, f);
    std::fwrite(p.data(), sizeof(float), kParams, f);
    std::fwrite(mm.data(), sizeof(float), kParams, f);
    const bool ok = std::fwrite(vv.data(), sizeof(float), kParams, f) == (size_t)kParams;
    std::fclose(f);
    return ok ? GWN_OK : set_error(GWN_ERR_INVALID_ARG, "short write");
}

gwn_status gwn_surrogate_load(gwn_mesh *m, const char *path) {
    clear_error();
    if (!m || !path) return set_error(GWN_ERR_INVALID_ARG, "NULL argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(GWN_ERR_INVALID_ARG, std::string("cannot read ") + path);
    uint32_t head[4];
    int64_t steps = 0;
    float lo[3], hi[3];
    gwn_mlp_config cfg;
    std::vector<float> p(kParams), mm(kParams), vv(kParams);
    bool ok = std::fread(head, sizeof(head), 1, f) == 1 && head[0] == 0x534E5747u && head[1] == 1u &&
              head[2] == (uint32_t)kParams && std::fread(&steps, sizeof(steps), 1, f) == 1 &&
              std::fread(lo, sizeof(float), 3, f) == 3 && std::fread(hi, sizeof(float), 3, f) == 3 &&
              std::fread(&cfg, sizeof(cfg), 1, f) == 1 && std::fread(p.data(), sizeof(float), kParams, f) == (size_t)kParams &&
              std::fread(mm.data(), sizeof(float), kParams, f) == (size_t)kParams &&
              std::fread(vv.data(), sizeof(float), kParams, f) == (size_t)kParams;
    std::fclose(f);
    if (!ok) return set_error(GWN_ERR_INVALID_ARG, std::string("not a surrogate checkpoint: ") + path);
    gwn_status r = ensure_surrogate(m);
    if (r != GWN_OK) return r;
    Surrogate *s = m->sur;
    s->steps = steps;
    s->cfg = cfg;
    if (s->cfg.chi_tol == 0.f) s->cfg.chi_tol = 0.25f;   // a checkpoint written before the field existed
    for (int d = 0; d < 3; ++d) {
        s->lo[d] = lo[d];
        s->hi[d] = hi[d];
    }
    GWN_CUDA_TRY(cudaMemcpy(s->params, p.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice));
    GWN_CUDA_TRY(cudaMemcpy(s->m, mm.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice));
    GWN_CUDA_TRY(cudaMemcpy(s->v, vv.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice));
    k_adam<<<grid_for(kParams, 256), 256, 0>>>(s->params, s->m, s->v, s->grad, s->wbf, 0.f, 0.f, 0.f, 1.f, 1.f, 1.f,
                                               0);
    GWN_CUDA_TRY(cudaDeviceSynchronize());
    if ((r = build_band(m, 0)) != GWN_OK) return r;
    s->trained = true;
    return GWN_OK;
}

gwn_status gwn_surrogate_calibrate(gwn_mesh *m, const float *samples, int64_t n, double max_error_rate,
                                   float min_margin, float *margin_out, int64_t *errors_at_margin, void *stream) {
    clear_error();
    if (!m || !surrogate_ready(m)) return set_error(GWN_ERR_INVALID_ARG, "mesh has no trained surrogate");
    if (!m->built) return set_error(GWN_ERR_NOT_BUILT, "calibration needs gwn_build_accel");
    if (!samples || n <= 0 || n > (int64_t)0x7fffffff || !(max_error_rate >= 0.0) || !(min_margin >= 0.f) ||
        min_margin >= 0.5f)
        return set_error(GWN_ERR_INVALID_ARG, "samples, 0 < n < 2^31, max_error_rate >= 0, 0 <= min_margin < 1/2");
    if (gwn_status e = check_device_buffers(m->device, {samples}, "gwn_surrogate_calibrate")) return e;
    DeviceScope dev_scope(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    Surrogate *s = m->sur;
    float *w_hat = nullptr, *w = nullptr;
    uint8_t *lab = nullptr;
    int32_t *chi = nullptr, *list = nullptr;
    unsigned long long *len = nullptr, *hist = nullptr;
    GWN_CUDA_TRY(cudaMallocAsync(&w_hat, sizeof(float) * n, st));
    GWN_CUDA_TRY(cudaMallocAsync(&w, sizeof(float) * n, st));
    GWN_CUDA_TRY(cudaMallocAsync(&lab, n, st));
    GWN_CUDA_TRY(cudaMallocAsync(&chi, sizeof(int32_t) * n, st));
    GWN_CUDA_TRY(cudaMallocAsync(&list, sizeof(int32_t) * n, st));
    GWN_CUDA_TRY(cudaMallocAsync(&len, sizeof(unsigned long long), st));
    GWN_CUDA_TRY(cudaMallocAsync(&hist, sizeof(unsigned long long) * kCalibBins, st));
    cudaMemsetAsync(len, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kCalibBins, st);
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
    const int grid = (int)std::min<int64_t>((n + 127) / 128, 3 * sm_count());
    k_mlp_forward<<<grid, 128, kSmemFwd, st>>>(mlp_dev(s), samples, n, 2, 0.f, w_hat, nullptr, nullptr, nullptr,
                                               nullptr, 0.f, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                               nullptr, 0.f, s->err);
    gwn_status r;
    if ((r = launch_chi(m, samples, n, chi, st)) == GWN_OK &&
        (r = launch_boundary_sum_list(m, samples, n, chi, w, lab, true, list, len, st)) == GWN_OK &&
        (r = launch_fp64_fix_list(m, samples, chi, w, lab, list, len, st)) == GWN_OK)
        k_calib_hist<<<grid_for(n, 256), 256, 0, st>>>(mlp_dev(s), samples, w_hat, lab, chi, s->cfg.chi_tol, n,
                                                       hist);
    std::vector<unsigned long long> h(kCalibBins, 0);
    if (r == GWN_OK)
        cudaMemcpyAsync(h.data(), hist, sizeof(unsigned long long) * kCalibBins, cudaMemcpyDeviceToHost, st);
    for (void *p : {(void *)w_hat, (void *)w, (void *)lab, (void *)chi, (void *)list, (void *)len, (void *)hist})
        cudaFreeAsync(p, st);
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
    if (r != GWN_OK) return r;
    GWN_LAUNCH_CHECK("surrogate calibration");
    if ((r = check_err(s, st)) != GWN_OK) return r;
    // smallest bin edge m with #{misclassified, |w_hat - 1/2| > m} <= rate * n
    const unsigned long long allowed = (unsigned long long)std::floor(max_error_rate * (double)n);
    unsigned long long above = 0;
    float mcal = 0.f;
    for (int b = kCalibBins - 1; b >= 0; --b) {
        if (above + h[b] > allowed) {
            mcal = (float)(b + 1) / 2048.f;
            break;
        }
        above += h[b];
    }
    const float margin = std::max(mcal, min_margin);
    unsigned long long errs = 0;
    for (int b = 0; b < kCalibBins; ++b)
        if ((float)b / 2048.f >= margin) errs += h[b];
    s->cfg.margin = margin;
    if (margin_out) *margin_out = margin;
    if (errors_at_margin) *errors_at_margin = (int64_t)errs;
    return GWN_OK;
}

gwn_status gwn_surrogate_detach(gwn_mesh *m) {
    clear_error();
    if (!m) return set_error(GWN_ERR_INVALID_ARG, "mesh is NULL");
    cudaDeviceSynchronize();
    surrogate_free(m->sur);
    m->sur = nullptr;
    return GWN_OK;
}

}  // extern "C"
