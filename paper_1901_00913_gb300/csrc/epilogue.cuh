// Device helpers shared by the banded and tensor-core kernels: operand
// rounding and the fused Step 1 / Step 3 epilogue of Alg. 2.
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace sfista {

static __device__ __forceinline__ float tf32_round(float x) {
    unsigned u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

// Step 1 shrink (+ projection) and Step 3 momentum for one pixel, FP64 state.
static __device__ __forceinline__ void prox_momentum(const ProxArgs &pa, size_t idx, double g) {
    double y = __ldcg(pa.Y + idx);
    double xprev = __ldcg(pa.Xin + idx);
    // (L y - g) / (L + lambda^2) with the two constants folded on the host
    double x = fma(pa.shrink, y, -pa.inv_den * g);
    if (pa.project && x < 0.0) x = 0.0;
    if (!isfinite(x)) atomicOr(pa.status, DEV_NONFINITE);
    double beta = pa.beta[pa.k - 1];
    double yn = x + beta * (x - xprev);
    pa.Xout[idx] = x;
    pa.Y[idx] = yn;
    if (pa.Yop) pa.Yop[idx] = (float)yn;
    if (pa.split_kind == 1) {
        __nv_bfloat16 hi = __double2bfloat16(yn);
        __nv_bfloat16 lo = __double2bfloat16(yn - (double)__bfloat162float(hi));
        reinterpret_cast<__nv_bfloat16 *>(pa.Yhi)[idx] = hi;
        if (pa.Ylo) reinterpret_cast<__nv_bfloat16 *>(pa.Ylo)[idx] = lo;
    } else if (pa.split_kind == 2) {
        float hi = tf32_round((float)yn);
        float lo = tf32_round((float)(yn - (double)hi));
        reinterpret_cast<float *>(pa.Yhi)[idx] = hi;
        if (pa.Ylo) reinterpret_cast<float *>(pa.Ylo)[idx] = lo;
    }
}

// Two neighbouring pixels idx, idx + 1 (idx even): vector loads and stores.
static __device__ __forceinline__ void prox_momentum2(const ProxArgs &pa, size_t idx, double g0, double g1) {
    const double2 y = __ldcg(reinterpret_cast<const double2 *>(pa.Y + idx));
    const double2 xp = __ldcg(reinterpret_cast<const double2 *>(pa.Xin + idx));
    double x0 = fma(pa.shrink, y.x, -pa.inv_den * g0);
    double x1 = fma(pa.shrink, y.y, -pa.inv_den * g1);
    if (pa.project) {
        x0 = x0 < 0.0 ? 0.0 : x0;
        x1 = x1 < 0.0 ? 0.0 : x1;
    }
    if (!isfinite(x0) || !isfinite(x1)) atomicOr(pa.status, DEV_NONFINITE);
    const double beta = pa.beta[pa.k - 1];
    const double y0 = x0 + beta * (x0 - xp.x), y1 = x1 + beta * (x1 - xp.y);
    *reinterpret_cast<double2 *>(pa.Xout + idx) = make_double2(x0, x1);
    *reinterpret_cast<double2 *>(pa.Y + idx) = make_double2(y0, y1);
    if (pa.Yop) *reinterpret_cast<float2 *>(pa.Yop + idx) = make_float2((float)y0, (float)y1);
    if (pa.split_kind == 1) {
        __nv_bfloat16 h0 = __double2bfloat16(y0), h1 = __double2bfloat16(y1);
        __nv_bfloat162 h;
        h.x = h0;
        h.y = h1;
        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(pa.Yhi) + idx) = h;
        if (pa.Ylo) {
            __nv_bfloat162 l;
            l.x = __double2bfloat16(y0 - (double)__bfloat162float(h0));
            l.y = __double2bfloat16(y1 - (double)__bfloat162float(h1));
            *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(pa.Ylo) + idx) = l;
        }
    } else if (pa.split_kind == 2) {
        const float h0 = tf32_round((float)y0), h1 = tf32_round((float)y1);
        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(pa.Yhi) + idx) = make_float2(h0, h1);
        if (pa.Ylo)
            *reinterpret_cast<float2 *>(reinterpret_cast<float *>(pa.Ylo) + idx) =
                make_float2(tf32_round((float)(y0 - (double)h0)), tf32_round((float)(y1 - (double)h1)));
    }
}

}  // namespace sfista
