// Double-float arithmetic for the FISTA state.
//
// A value is carried as an unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2), about 48 significant bits, stored in the same 8 bytes
// per pixel an FP64 value would take.  The state update then runs on the FP32
// pipe instead of GB300's much narrower FP64 pipe.  The error-free
// transforms are Knuth's TwoSum, the Fast-TwoSum of Dekker (|a| >= |b|) and
// the FMA-based TwoProduct; every step uses __fadd_rn / __fmul_rn / __fmaf_rn
// so the compiler cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace sfista {
namespace dfp {

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 add(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return add(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    float e = __fmaf_rn(a.x, b, -p);
    e = __fmaf_rn(a.y, b, e);
    return fast_two_sum(p, e);
}
// Renormalises a pair: Fast-TwoSum's |a| >= |b| precondition can fail in
// add() under cancellation (values near zero), leaving |lo| slightly above
// ulp(hi)/2.  Such a pair converts to FP64 and back as a different pair of
// the same value, so the state is renormalised where it is stored, and a
// solve resumed from FP64 continues bit for bit.
__device__ __forceinline__ float2 normalize(float2 a) { return fast_two_sum(a.x, a.y); }
// Y = X + beta (X - Xp): Step 3 of Alg. 2, renormalised.
__device__ __forceinline__ float2 momentum(float2 x, float2 xp, float2 beta) {
    return normalize(add(x, mul(beta, sub(x, xp))));
}
// Conversions (FP64 only at the boundaries of a solve).
__host__ __device__ __forceinline__ float2 from_double(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__host__ __device__ __forceinline__ double to_double(float2 a) { return (double)a.x + (double)a.y; }
// Nearest float to hi + lo (hi is already the rounded sum for a normalised pair).
__device__ __forceinline__ float to_float(float2 a) { return __fadd_rn(a.x, a.y); }

}  // namespace dfp
}  // namespace sfista
