// Generated by fit_atan.py: do not edit.
// atan(t) ~= t * P(t^2), 0 <= t <= 1, P of degree 8 (Remez, minimax relative error).
// Minimax relative error of the exact-coefficient fit: 1.523e-08
// FP32 coefficients, FP32 Horner: max relative error 1.570e-07, max absolute error 1.172e-07
#pragma once
#define GWN_ATAN_DEGREE 8
// P(s) in Horner form
__device__ __forceinline__ float gwn_atan_poly(float s) {
    float p = 0.0028498894535005093f;
    p = fmaf(p, s, -0.016068628057837486f);
    p = fmaf(p, s, 0.04269151762127876f);
    p = fmaf(p, s, -0.07504294812679291f);
    p = fmaf(p, s, 0.10640934109687805f);
    p = fmaf(p, s, -0.14203643798828125f);
    p = fmaf(p, s, 0.1999261975288391f);
    p = fmaf(p, s, -0.3333307206630707f);
    p = fmaf(p, s, 1.0f);
    return p;
}
// the same coefficients for the paired-FP32 evaluation
#define GWN_ATAN_C0 1.0f
#define GWN_ATAN_C1 -0.3333307206630707f
#define GWN_ATAN_C2 0.1999261975288391f
#define GWN_ATAN_C3 -0.14203643798828125f
#define GWN_ATAN_C4 0.10640934109687805f
#define GWN_ATAN_C5 -0.07504294812679291f
#define GWN_ATAN_C6 0.04269151762127876f
#define GWN_ATAN_C7 -0.016068628057837486f
#define GWN_ATAN_C8 0.0028498894535005093f
