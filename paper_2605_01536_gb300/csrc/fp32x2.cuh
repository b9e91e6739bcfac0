// Small arithmetic building blocks shared by the query kernels: the raw SFU
// reciprocal and reciprocal square root, and paired-FP32 forms.
#pragma once

#include <cuda_runtime.h>

namespace gwn {

// Raw SFU reciprocal and reciprocal square root (PTX rcp.approx / rsqrt.approx,
// relative error below 2^-22).  Callers keep the operand in the normal range,
// so the flush-to-zero forms lose nothing and carry no denormal fix-up code.
__device__ __forceinline__ float sfu_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sfu_rsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- paired-FP32 forms (Blackwell FFMA2 / FADD2 / FMUL2): one instruction
// evaluates the same operation for two queries held in a float2.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

}  // namespace gwn
