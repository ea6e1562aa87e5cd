// Device helpers shared by the banded and tensor-core kernels: operand
// rounding and the fused Step 1 / Step 3 epilogue of Alg. 2.
#pragma once

#include <cuda_bf16.h>

#include "dfloat.cuh"
#include "internal.h"

namespace sfista {

static __device__ __forceinline__ float tf32_round(float x) {
    unsigned u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
}

// Step 1 shrink (+ l1 soft threshold, + projection) and Step 3 momentum for one pixel, with the
// state in double-float:  X_k = s Y_k - d G  (s = L/(L+lambda^2),
// d = 1/(L+lambda^2)),  Y_{k+1} = X_k + beta_k (X_k - X_{k-1}).
// Also writes the operand copies of Y_{k+1}: FP32 (banded operator) and/or a
// hi/lo split (BF16 or TF32) for the tensor-core operator.
// With the l1 term the shrunk value is soft-thresholded by tau = mu/(L+lambda^2)
// first (S_mu(v)/(L+lambda^2) = S_tau(v/(L+lambda^2)) since L+lambda^2 > 0).
static __device__ __forceinline__ float2 soft_threshold(float2 x, float2 tau) {
    const bool neg = x.x < 0.0f;   // the hi word carries the sign of a normalised pair
    const float2 d = dfp::sub(neg ? make_float2(-x.x, -x.y) : x, tau);
    if (!(d.x > 0.0f)) return make_float2(0.0f, 0.0f);
    return neg ? make_float2(-d.x, -d.y) : d;
}

static __device__ __forceinline__ float2 prox_step(const ProxArgs &pa, float2 y, float2 xp, float g, float2 beta,
                                                   float2 *xout, bool *bad) {
    float2 x = dfp::sub(dfp::mul(pa.shrink, y), dfp::mul_f(pa.inv_den, g));
    if (pa.tau.x > 0.0f) x = soft_threshold(x, pa.tau);
    if (pa.project && x.x < 0.0f) x = make_float2(0.0f, 0.0f);
    x = dfp::normalize(x);
    *bad |= !isfinite(x.x);
    *xout = x;
    return dfp::momentum(x, xp, beta);
}

static __device__ __forceinline__ void store_operands(const ProxArgs &pa, size_t idx, float2 yn) {
    const float yf = dfp::to_float(yn);
    if (pa.Yop) pa.Yop[idx] = yf;
    if (pa.split_kind == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(yf);
        reinterpret_cast<__nv_bfloat16 *>(pa.Yhi)[idx] = h;
        if (pa.Ylo)
            reinterpret_cast<__nv_bfloat16 *>(pa.Ylo)[idx] =
                __float2bfloat16_rn(__fadd_rn(__fsub_rn(yn.x, __bfloat162float(h)), yn.y));
    } else if (pa.split_kind == 2) {
        const float h = tf32_round(yf);
        reinterpret_cast<float *>(pa.Yhi)[idx] = h;
        if (pa.Ylo) reinterpret_cast<float *>(pa.Ylo)[idx] = tf32_round(__fadd_rn(__fsub_rn(yn.x, h), yn.y));
    }
}

static __device__ __forceinline__ void prox_momentum(const ProxArgs &pa, size_t idx, float g) {
    const float2 y = __ldcg(pa.Y + idx), xp = __ldcg(pa.Xin + idx);
    bool bad = false;
    float2 x;
    const float2 yn = prox_step(pa, y, xp, g, pa.beta[pa.k - 1], &x, &bad);
    if (bad) atomicOr(pa.status, DEV_NONFINITE);
    pa.Xout[idx] = x;
    pa.Y[idx] = yn;
    store_operands(pa, idx, yn);
}

// State loads of N pixels (Y_k and X_{k-1}), all issued before any use.
template <int N>
static __device__ __forceinline__ void prox_load_n(const ProxArgs &pa, const size_t *idx, const bool *valid, float2 *y,
                                                   float2 *xp) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
        y[q] = valid[q] ? __ldcg(pa.Y + idx[q]) : make_float2(0.f, 0.f);
        xp[q] = valid[q] ? __ldcg(pa.Xin + idx[q]) : make_float2(0.f, 0.f);
    }
}

// Step 1 + Step 3 for N pixels whose state (y, xp) and momentum weight
// beta = beta[k-1] are already loaded.
template <int N>
static __device__ __forceinline__ void prox_apply_n(const ProxArgs &pa, const size_t *idx, const float *g,
                                                    const bool *valid, const float2 *y, const float2 *xp,
                                                    float2 beta) {
    bool bad = false;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        if (!valid[q]) continue;
        float2 x;
        const float2 yn = prox_step(pa, y[q], xp[q], g[q], beta, &x, &bad);
        pa.Xout[idx[q]] = x;
        pa.Y[idx[q]] = yn;
        store_operands(pa, idx[q], yn);
    }
    if (bad) atomicOr(pa.status, DEV_NONFINITE);
}

static __device__ __forceinline__ float prox_step32(const ProxArgs &pa, float y, float xp, float g, float beta,
                                                    float *xout, bool *bad);
static __device__ __forceinline__ void store_operands32(const ProxArgs &pa, size_t idx, float yn);

// N pixels at once: every state load is issued before any arithmetic or
// store, so a thread keeps 2N loads in flight.  With an FP32 state (pa.Y32:
// the tensor-core forms, when an FP32 iteration of residual refinement runs
// its adjoint on the band kernels) the step is prox_step32 on that state.
template <int N>
static __device__ __forceinline__ void prox_momentum_n(const ProxArgs &pa, const size_t *idx, const float *g,
                                                       const bool *valid) {
    if (pa.Y32) {
        float y[N], xp[N];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            y[q] = valid[q] ? __ldcg(pa.Y32 + idx[q]) : 0.f;
            xp[q] = valid[q] ? __ldcg(pa.Xin32 + idx[q]) : 0.f;
        }
        const float beta = pa.beta[pa.k - 1].x;
        bool bad = false;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (!valid[q]) continue;
            float x;
            const float yn = prox_step32(pa, y[q], xp[q], g[q], beta, &x, &bad);
            pa.Xout32[idx[q]] = x;
            pa.Y32[idx[q]] = yn;
            store_operands32(pa, idx[q], yn);
        }
        if (bad) atomicOr(pa.status, DEV_NONFINITE);
        return;
    }
    float2 y[N], xp[N];
    prox_load_n<N>(pa, idx, valid, y, xp);
    prox_apply_n<N>(pa, idx, g, valid, y, xp, pa.beta[pa.k - 1]);
}

// FP32 state (tensor-core forms, whose operator error is far above FP32
// rounding): Step 1 (+ l1 threshold, + projection) and Step 3 in FP32 with
// the constants rounded to FP32; the operand copies of Y_{k+1} as in
// store_operands.
static __device__ __forceinline__ float prox_step32(const ProxArgs &pa, float y, float xp, float g, float beta,
                                                    float *xout, bool *bad) {
    float x = fmaf(-pa.inv_den.x, g, pa.shrink.x * y);
    if (pa.tau.x > 0.0f) x = x > 0.0f ? fmaxf(x - pa.tau.x, 0.0f) : fminf(x + pa.tau.x, 0.0f);
    if (pa.project && x < 0.0f) x = 0.0f;
    *bad |= !isfinite(x);
    *xout = x;
    return fmaf(beta, x - xp, x);
}

static __device__ __forceinline__ void store_operands32(const ProxArgs &pa, size_t idx, float yn) {
    if (pa.Yop) pa.Yop[idx] = yn;
    if (pa.split_kind == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(yn);
        reinterpret_cast<__nv_bfloat16 *>(pa.Yhi)[idx] = h;
        if (pa.Ylo) reinterpret_cast<__nv_bfloat16 *>(pa.Ylo)[idx] = __float2bfloat16_rn(__fsub_rn(yn, __bfloat162float(h)));
    } else if (pa.split_kind == 2) {
        const float h = tf32_round(yn);
        reinterpret_cast<float *>(pa.Yhi)[idx] = h;
        if (pa.Ylo) reinterpret_cast<float *>(pa.Ylo)[idx] = tf32_round(__fsub_rn(yn, h));
    }
}

// Pairs of neighbouring pixels (idx[q] even) for N rows at once, FP32 state.
template <int N>
static __device__ __forceinline__ void prox_momentum2_n32(const ProxArgs &pa, const size_t *idx, const float *g0,
                                                          const float *g1, const bool *valid) {
    float2 y[N], xp[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        y[q] = valid[q] ? __ldcg(reinterpret_cast<const float2 *>(pa.Y32 + idx[q])) : make_float2(0.f, 0.f);
        xp[q] = valid[q] ? __ldcg(reinterpret_cast<const float2 *>(pa.Xin32 + idx[q])) : make_float2(0.f, 0.f);
    }
    const float beta = pa.beta[pa.k - 1].x;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        if (!valid[q]) continue;
        float x0, x1;
        const float y0 = prox_step32(pa, y[q].x, xp[q].x, g0[q], beta, &x0, &bad);
        const float y1 = prox_step32(pa, y[q].y, xp[q].y, g1[q], beta, &x1, &bad);
        *reinterpret_cast<float2 *>(pa.Xout32 + idx[q]) = make_float2(x0, x1);
        *reinterpret_cast<float2 *>(pa.Y32 + idx[q]) = make_float2(y0, y1);
        store_operands32(pa, idx[q], y0);
        store_operands32(pa, idx[q] + 1, y1);
    }
    if (bad) atomicOr(pa.status, DEV_NONFINITE);
}

// Pairs of neighbouring pixels (idx[q] even) for N rows at once (FP32
// state: prox_momentum2_n32).
template <int N>
static __device__ __forceinline__ void prox_momentum2_n(const ProxArgs &pa, const size_t *idx, const float *g0,
                                                        const float *g1, const bool *valid) {
    if (pa.Y32) {
        prox_momentum2_n32<N>(pa, idx, g0, g1, valid);
        return;
    }
    float4 y[N], xp[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        y[q] = valid[q] ? __ldcg(reinterpret_cast<const float4 *>(pa.Y + idx[q])) : make_float4(0.f, 0.f, 0.f, 0.f);
        xp[q] = valid[q] ? __ldcg(reinterpret_cast<const float4 *>(pa.Xin + idx[q])) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float2 beta = pa.beta[pa.k - 1];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        if (!valid[q]) continue;
        float2 x0, x1;
        const float2 y0 = prox_step(pa, make_float2(y[q].x, y[q].y), make_float2(xp[q].x, xp[q].y), g0[q], beta, &x0,
                                    &bad);
        const float2 y1 = prox_step(pa, make_float2(y[q].z, y[q].w), make_float2(xp[q].z, xp[q].w), g1[q], beta, &x1,
                                    &bad);
        *reinterpret_cast<float4 *>(pa.Xout + idx[q]) = make_float4(x0.x, x0.y, x1.x, x1.y);
        *reinterpret_cast<float4 *>(pa.Y + idx[q]) = make_float4(y0.x, y0.y, y1.x, y1.y);
        store_operands(pa, idx[q], y0);
        store_operands(pa, idx[q] + 1, y1);
    }
    if (bad) atomicOr(pa.status, DEV_NONFINITE);
}

// Four neighbouring pixels (idx a multiple of 4, every array 16-byte aligned
// there): the operand copies of Y_{k+1} as store_operands32 writes them, one
// 16-byte (FP32 / TF32) or 8-byte (BF16) store per array.
static __device__ __forceinline__ void store_operands32x4(const ProxArgs &pa, size_t idx, float4 v) {
    if (pa.Yop) *reinterpret_cast<float4 *>(pa.Yop + idx) = v;
    if (pa.split_kind == 1) {
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
        *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(pa.Yhi) + idx) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&h01), *reinterpret_cast<const uint32_t *>(&h23));
        if (pa.Ylo) {
            const __nv_bfloat162 l01 = __floats2bfloat162_rn(__fsub_rn(v.x, __bfloat162float(h01.x)),
                                                             __fsub_rn(v.y, __bfloat162float(h01.y)));
            const __nv_bfloat162 l23 = __floats2bfloat162_rn(__fsub_rn(v.z, __bfloat162float(h23.x)),
                                                             __fsub_rn(v.w, __bfloat162float(h23.y)));
            *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(pa.Ylo) + idx) =
                make_uint2(*reinterpret_cast<const uint32_t *>(&l01), *reinterpret_cast<const uint32_t *>(&l23));
        }
    } else if (pa.split_kind == 2) {
        const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(pa.Yhi) + idx) = h;
        if (pa.Ylo)
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(pa.Ylo) + idx) =
                make_float4(tf32_round(__fsub_rn(v.x, h.x)), tf32_round(__fsub_rn(v.y, h.y)),
                            tf32_round(__fsub_rn(v.z, h.z)), tf32_round(__fsub_rn(v.w, h.w)));
    }
}

// Groups of four neighbouring pixels (idx[q] a multiple of 4) for N rows at
// once, FP32 state: 16-byte state loads and stores, every load issued before
// any arithmetic.  Same arithmetic as prox_momentum2_n32.
template <int N>
static __device__ __forceinline__ void prox_momentum4_n32(const ProxArgs &pa, const size_t *idx, const float4 *g,
                                                          const bool *valid) {
    float4 y[N], xp[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        y[q] = valid[q] ? __ldcg(reinterpret_cast<const float4 *>(pa.Y32 + idx[q])) : make_float4(0.f, 0.f, 0.f, 0.f);
        xp[q] = valid[q] ? __ldcg(reinterpret_cast<const float4 *>(pa.Xin32 + idx[q])) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float beta = pa.beta[pa.k - 1].x;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        if (!valid[q]) continue;
        float4 x, yn;
        yn.x = prox_step32(pa, y[q].x, xp[q].x, g[q].x, beta, &x.x, &bad);
        yn.y = prox_step32(pa, y[q].y, xp[q].y, g[q].y, beta, &x.y, &bad);
        yn.z = prox_step32(pa, y[q].z, xp[q].z, g[q].z, beta, &x.z, &bad);
        yn.w = prox_step32(pa, y[q].w, xp[q].w, g[q].w, beta, &x.w, &bad);
        *reinterpret_cast<float4 *>(pa.Xout32 + idx[q]) = x;
        *reinterpret_cast<float4 *>(pa.Y32 + idx[q]) = yn;
        store_operands32x4(pa, idx[q], yn);
    }
    if (bad) atomicOr(pa.status, DEV_NONFINITE);
}

}  // namespace sfista
