// Reverse mode of the unrolled Alg. 2 (no projection, L held fixed), for
// gradients of a loss l(X_K) with respect to B, lambda and the dense factors.
//
// Each step is X_k = M Y_k + A_s^T B / den with M = (L I - A_s^T A_s) / den,
// den = L + lambda^2, and Y_{k+1} = X_k + beta_k (X_k - X_{k-1}).  M is
// symmetric, so the adjoint of a step reuses the forward operator kernels:
//   y_bar_k = M x_bar_k,  x_bar_{k-1} += (1 + beta_{k-1}) y_bar_k,
//   x_bar_{k-2} -= beta_{k-1} y_bar_k,
// and the gradients collect, with V = x_bar_k, W = A_s V, R_k = A_s Y_k - B:
//   dl/dB      = A_s (sum_k V) / den
//   dl/dlambda = -2 lambda / den * sum_k <V, X_k>
//   dl/dA_i   -= (R_k^T B_i V + W^T B_i Y_k) / den
//   dl/dB_i   -= (R_k A_i V^T + W A_i Y_k^T) / den
// The forward keeps (X_k, X_{k-1}) every `ckpt` iterations; the backward
// recomputes one segment at a time from its checkpoint.  Operator products run
// in FP32 on the banded kernels; the adjoint state x_bar is FP64.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ctx.h"

namespace sfista {
namespace {

// ybar = (L V - T) * inv, and sumV += V (one pass over V).
__global__ void ybar_kernel(double *ybar, double *sumV, const double *V, const float *T, double L, double inv,
                            size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = V[i];
        ybar[i] = (L * v - (double)T[i]) * inv;
        sumV[i] += 1.0 * v;
    }
}
// End of a reverse step: xa += (1 + beta) ybar, xb += -beta ybar (when
// `update`), and V = 0 (three distinct buffers).
__global__ void step_update_kernel(double *xa, double *xb, double *V, const double *ybar, double beta, int update,
                                   size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (update) {
            const double y = ybar[i];
            xa[i] += (1.0 + beta) * y;
            xb[i] += -beta * y;
        }
        V[i] = 0.0;
    }
}
// FP32 copies of V and (when Y is not NULL) Y in one pass.
__global__ void to_f32_pair_kernel(const double *V, float *Vf, const double *Y, float *Yf, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        Vf[i] = (float)V[i];
        if (Y) Yf[i] = (float)Y[i];
    }
}
__global__ void scale_f32(float *y, const float *x, float a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// Factor gradients, batched over the buffered steps of a checkpoint segment:
//   C_i[I][J] += alpha * sum_{part < 2} sum_{s < S} sum_{t < T} P_part(i, s)(I, t) Q_part(i, s)(J, t)
// with operand (i, s) at base + i * term + s * step.  TN: element (I, t) at
// [t * ld + I] (I contiguous, contraction over rows); NT: at [I * ld + t]
// (contraction over columns).  128 x 128 output tiles, 16-deep slices, 8 x 8
// outputs per thread, the next slice prefetched into registers while the
// current one is multiplied from shared memory.  The contraction (2 parts x S
// steps x T rounded up to 16) is split across blockIdx.z for parallelism; each
// split writes its partial tile and grad_reduce adds the splits in a fixed
// order (deterministic).  Held to two blocks per SM (128 registers, a few
// spilled): measured faster than one block with 150-160 registers.
struct GradOperands {
    const float *P[2], *Q[2];
    long p_term, q_term, p_step, q_step, ld;
    int S, T, I, J, r, splits, slices_per_split;
};

constexpr int GB = 128, GK = 16, GLD = GB + 4;

// VEC: 16-byte loads (ld, and I, J (TN) or T (NT), multiples of 4, bases
// 16-byte aligned); otherwise four predicated scalar loads.
template <bool NT, bool VEC>
__device__ __forceinline__ void grad_load(const float *base, long ld, int n_idx, int T, int idx0, int t0, int tid,
                                          float4 *v) {
    // 512 float4 per 128 x 16 slice, two per thread.
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = tid + h * 256;
        int I, t;
        if (NT) {
            I = f & 127;
            t = (f >> 7) * 4;
        } else {
            t = f >> 5;
            I = (f & 31) * 4;
        }
        const int gI = idx0 + I, gt = t0 + t;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (VEC) {
            if (gI < n_idx && gt < T) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(NT ? base + (long)gI * ld + gt
                                                                           : base + (long)gt * ld + gI));
                x[0] = q.x;
                x[1] = q.y;
                x[2] = q.z;
                x[3] = q.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (NT) {
                    if (gI < n_idx && gt + j < T) x[j] = __ldg(base + (long)gI * ld + gt + j);
                } else {
                    if (gI + j < n_idx && gt < T) x[j] = __ldg(base + (long)gt * ld + gI + j);
                }
            }
        }
        v[h] = make_float4(x[0], x[1], x[2], x[3]);
    }
}

template <bool NT>
__device__ __forceinline__ void grad_store(float (*S)[GLD], int tid, const float4 *v) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = tid + h * 256;
        if (NT) {
            const int I = f & 127, t = (f >> 7) * 4;
            S[t][I] = v[h].x;
            S[t + 1][I] = v[h].y;
            S[t + 2][I] = v[h].z;
            S[t + 3][I] = v[h].w;
        } else {
            *reinterpret_cast<float4 *>(&S[f >> 5][(f & 31) * 4]) = v[h];
        }
    }
}

template <bool NT, bool VEC>
__global__ void __launch_bounds__(256, 2) grad_gemm(GradOperands o, float *partial) {
    __shared__ __align__(16) float Ps[2][GK][GLD];
    __shared__ __align__(16) float Qs[2][GK][GLD];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int I0 = blockIdx.y * GB, J0 = blockIdx.x * GB;
    const int term = blockIdx.z / o.splits, split = blockIdx.z % o.splits;
    const int Tp = (o.T + GK - 1) / GK;                    // slices per (part, step)
    const int total = 2 * o.S * Tp;
    const int u0 = split * o.slices_per_split, u1 = min(total, u0 + o.slices_per_split);
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    auto operands = [&](int u, const float **P, const float **Q, int *t0) {
        const int part = u / (o.S * Tp), rem = u - part * o.S * Tp, s = rem / Tp;
        *t0 = (rem - s * Tp) * GK;
        *P = (part ? o.P[1] : o.P[0]) + term * o.p_term + s * o.p_step;
        *Q = (part ? o.Q[1] : o.Q[0]) + term * o.q_term + s * o.q_step;
    };
    float4 pv[2], qv[2];
    if (u0 < u1) {
        const float *P, *Q;
        int t0;
        operands(u0, &P, &Q, &t0);
        grad_load<NT, VEC>(P, o.ld, o.I, o.T, I0, t0, tid, pv);
        grad_load<NT, VEC>(Q, o.ld, o.J, o.T, J0, t0, tid, qv);
        grad_store<NT>(Ps[0], tid, pv);
        grad_store<NT>(Qs[0], tid, qv);
    }
    __syncthreads();
    int cur = 0;
    for (int u = u0; u < u1; ++u) {
        const bool next = u + 1 < u1;
        if (next) {
            const float *P, *Q;
            int t0;
            operands(u + 1, &P, &Q, &t0);
            grad_load<NT, VEC>(P, o.ld, o.I, o.T, I0, t0, tid, pv);
            grad_load<NT, VEC>(Q, o.ld, o.J, o.T, J0, t0, tid, qv);
        }
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&Ps[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&Ps[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Qs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Qs[cur][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
        if (next) {
            grad_store<NT>(Ps[cur ^ 1], tid, pv);
            grad_store<NT>(Qs[cur ^ 1], tid, qv);
        }
        __syncthreads();
        cur ^= 1;
    }
    float *out = partial + ((size_t)term * o.splits + split) * o.I * o.J;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int gI = I0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + x - 4);
        if (gI >= o.I) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gJ = J0 + h * 64 + tx * 4;
            float *o4 = out + (size_t)gI * o.J + gJ;
            if (VEC) {
                if (gJ < o.J)
                    *reinterpret_cast<float4 *>(o4) =
                        make_float4(acc[x][4 * h], acc[x][4 * h + 1], acc[x][4 * h + 2], acc[x][4 * h + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (gJ + j < o.J) o4[j] = acc[x][4 * h + j];
            }
        }
    }
}

// C[i][x] += alpha * sum_split partial[i][split][x], splits in order.
__global__ void grad_reduce(float *C, const float *partial, int r, int splits, size_t IJ, float alpha) {
    const size_t total = (size_t)r * IJ;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / IJ, x = e - i * IJ;
        const float *p = partial + i * splits * IJ + x;
        float sum = 0.f;
        for (int sp = 0; sp < splits; ++sp) sum += p[(size_t)sp * IJ];
        C[e] += alpha * sum;
    }
}

int grid1(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

constexpr size_t kGradBufferBytes = (size_t)2 << 30;   // factor-gradient step buffers

// Contraction splits: the smallest count (at most 16, at least four slices
// each) whose blocks fill at least one wave of one block per SM to 90 %.
int grad_splits(const GradOperands &o, int sms) {
    const int tiles = ((o.I + GB - 1) / GB) * ((o.J + GB - 1) / GB) * o.r;
    const int total = 2 * o.S * ((o.T + GK - 1) / GK);
    const int cap = std::max(1, std::min(16, total / 4));
    int best = 1;
    double best_use = 0.0;
    for (int sp = 1; sp <= cap; ++sp) {
        const long blocks = (long)tiles * sp;
        const double use = (double)blocks / ((double)((blocks + sms - 1) / sms) * sms);
        if (blocks >= sms && use >= 0.9) return sp;
        if (use > best_use + 1e-9) best_use = use, best = sp;
    }
    return best;
}

// vec: every leading dimension, extent and base suits 16-byte access (the
// caller checks m, n multiples of 4; buffers are cudaMalloc'ed).
void launch_grad_gemm(bool nt, bool vec, GradOperands o, float *C, float *partial, float alpha, cudaStream_t s) {
    const int total = 2 * o.S * ((o.T + GK - 1) / GK);
    o.slices_per_split = (total + o.splits - 1) / o.splits;
    dim3 g((o.J + GB - 1) / GB, (o.I + GB - 1) / GB, o.r * o.splits);
    if (nt && vec)
        grad_gemm<true, true><<<g, 256, 0, s>>>(o, partial);
    else if (nt)
        grad_gemm<true, false><<<g, 256, 0, s>>>(o, partial);
    else if (vec)
        grad_gemm<false, true><<<g, 256, 0, s>>>(o, partial);
    else
        grad_gemm<false, false><<<g, 256, 0, s>>>(o, partial);
    const size_t IJ = (size_t)o.I * o.J;
    grad_reduce<<<grid1((size_t)o.r * IJ), 256, 0, s>>>(C, partial, o.r, o.splits, IJ, alpha);
}

struct Scratch {
    std::vector<void *> ptrs;
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(count, 1));
        if (!e) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
};

sfista_status check_unrolled(sfista_ctx *c, int iters, int ckpt) {
    if (!c) return fail(SFISTA_EINVAL, "context is NULL");
    if (!is_banded(c->op))
        return fail(SFISTA_ENOTSUP, "the unrolled adjoint runs on the banded FP32 operator form");
    if (c->opts.project_nonneg) return fail(SFISTA_ENOTSUP, "the projection is not differentiable");
    if (c->opts.l1 > 0.0) return fail(SFISTA_ENOTSUP, "the l1 soft threshold is not differentiable");
    if (iters < 1 || ckpt < 1) return fail(SFISTA_EINVAL, "iters and ckpt_every must be >= 1");
    return SFISTA_OK;
}

// A_s x (FP32, banded) into out: one fused launch when the context uses the
// fused form, else the two passes through the context's Z.  EPI_RESIDUAL
// subtracts the context's B (A_s x - B).
void As_apply(sfista_ctx *c, const float *x, float *out, cudaStream_t s, EpiKind epi = EPI_STORE) {
    const HostSetup &h = c->hs;
    ProxArgs pa{};
    pa.Bd = c->Bd;
    if (fused_apply(c)) {
        launch_band_op_fused(x, c->m, c->n, c->r, c->fA, h.A.lo, h.A.w, c->fB, h.B.lo, h.B.w, epi, out, pa,
                             interior_fwd(c), s);
        return;
    }
    launch_band_rows<float>(x, c->m, c->n, c->fA, h.A.lo, h.A.w, c->r, c->Z, s);
    launch_band_cols<float>(c->Z, c->m, c->n, c->fB, h.B.lo, h.B.w, c->r, epi, out, pa, s);
}
void AsT_apply(sfista_ctx *c, const float *x, float *out, cudaStream_t s) {
    const HostSetup &h = c->hs;
    ProxArgs pa{};
    if (fused_apply(c)) {
        launch_band_op_fused(x, c->m, c->n, c->r, c->fAT, h.AT.lo, h.AT.w, c->fBT, h.BT.lo, h.BT.w, EPI_STORE, out, pa,
                             interior_adj(c), s);
        return;
    }
    launch_band_rows<float>(x, c->m, c->n, c->fAT, h.AT.lo, h.AT.w, c->r, c->Z, s);
    launch_band_cols<float>(c->Z, c->m, c->n, c->fBT, h.BT.lo, h.BT.w, c->r, EPI_STORE, out, pa, s);
}

}  // namespace
}  // namespace sfista

using namespace sfista;

extern "C" sfista_status sfista_unrolled_fwd(sfista_ctx *c, const float *d_b, double lambda, int iters, int ckpt_every,
                                             double *d_ckpt, float *d_x, void *stream) {
    sfista_status st = check_unrolled(c, iters, ckpt_every);
    if (st) return st;
    if (!d_ckpt || !d_x) return fail(SFISTA_EINVAL, "NULL checkpoint or output buffer");
    DeviceGuard g(c->dev);
    cudaStream_t user = (cudaStream_t)stream;
    st = solve_core(c, d_b, lambda, 0, 0, nullptr, nullptr, user);
    if (st) return st;
    st = ensure_beta(c, iters + 1);
    if (st) return st;
    const size_t N = c->N;
    const int nseg = (iters + ckpt_every - 1) / ckpt_every;
    for (int j = 0; j < nseg; ++j) {
        const int k0 = j * ckpt_every, k1 = std::min(iters, k0 + ckpt_every);
        launch_df_to_f64(c->Xb[k0 & 1], d_ckpt + (size_t)2 * j * N, N, c->stream);
        launch_df_to_f64(c->Xb[(k0 + 1) & 1], d_ckpt + (size_t)(2 * j + 1) * N, N, c->stream);
        for (int k = k0 + 1; k <= k1; ++k) enqueue_iteration(c, k, lambda);
    }
    launch_df_to_f32(c->Xb[iters & 1], d_x, N, c->stream);
    SF_CUDA(cudaGetLastError());
    return finish_on_user(c, user);
}

extern "C" sfista_status sfista_unrolled_bwd(sfista_ctx *c, const float *d_b, double lambda, int iters, int ckpt_every,
                                             const double *d_ckpt, const float *d_gX, float *d_gb, double *g_lambda,
                                             float *d_gA, float *d_gB, void *stream) {
    sfista_status st = check_unrolled(c, iters, ckpt_every);
    if (st) return st;
    if (!d_ckpt || !d_gX || !d_gb || !g_lambda) return fail(SFISTA_EINVAL, "NULL argument");
    DeviceGuard g(c->dev);
    cudaStream_t user = (cudaStream_t)stream;
    st = ensure_beta(c, iters + 1);
    if (st) return st;
    const size_t N = c->N;
    const int m = c->m, n = c->n, r = c->r;
    const HostSetup &h = c->hs;
    const double L = c->L, den = L + lambda * lambda, inv = 1.0 / den;
    const int ce = ckpt_every, nseg = (iters + ce - 1) / ce;
    const bool factors = d_gA || d_gB;
    // Factor-gradient operands of up to `scap` steps are buffered and
    // contracted together (one batched GEMM per family per flush).
    const size_t step_floats = N * (4 + 4 * (size_t)r);   // R, W, V, Y and U, U2, R A_i, W A_i (r each)
    const int scap = factors ? (int)std::max<size_t>(1, std::min<size_t>(ce, kGradBufferBytes / (4 * step_floats))) : 0;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
    const bool vec = m % 4 == 0 && n % 4 == 0;
    GradOperands oa{}, ob{};
    oa.S = ob.S = scap;
    oa.r = ob.r = r;
    oa.ld = ob.ld = n;
    oa.T = m, oa.I = n, oa.J = n;   // dl/dA_i = R^T (B_i V) + W^T (B_i Y):  TN over image rows
    ob.T = n, ob.I = m, ob.J = m;   // dl/dB_i = (R A_i) V^T + (W A_i) Y^T:  NT over image columns
    oa.splits = factors ? grad_splits(oa, sms) : 1;
    ob.splits = factors ? grad_splits(ob, sms) : 1;
    const size_t part_floats = factors ? (size_t)r * std::max((size_t)oa.splits * n * n, (size_t)ob.splits * m * m) : 1;
    Scratch sc;
    double *segX, *segY, *xb, *sumV, *ybar, *dots, *partial;
    float *Vf, *Wf, *Tf, *Rseg = nullptr, *Wseg = nullptr, *Vseg = nullptr, *Yseg = nullptr, *Useg = nullptr,
                         *U2seg = nullptr, *Zsseg = nullptr, *Zqseg = nullptr, *gpart = nullptr;
    cudaError_t e;
    if ((e = sc.get(&segX, (size_t)ce * N)) || (e = sc.get(&segY, (size_t)ce * N)) || (e = sc.get(&xb, 3 * N)) ||
        (e = sc.get(&sumV, N)) || (e = sc.get(&ybar, N)) || (e = sc.get(&dots, 2 * (size_t)iters)) ||
        (e = sc.get(&partial, 512)) || (e = sc.get(&Vf, N)) || (e = sc.get(&Wf, N)) ||
        (e = sc.get(&Tf, N)))
        return fail(SFISTA_ENOMEM, std::string("adjoint buffers: ") + cudaGetErrorString(e));
    if (factors &&
        ((e = sc.get(&Rseg, scap * N)) || (e = sc.get(&Wseg, scap * N)) || (e = sc.get(&Vseg, scap * N)) ||
         (e = sc.get(&Yseg, scap * N)) || (e = sc.get(&Useg, scap * r * N)) || (e = sc.get(&U2seg, scap * r * N)) ||
         (e = sc.get(&Zsseg, scap * r * N)) || (e = sc.get(&Zqseg, scap * r * N)) ||
         (e = sc.get(&gpart, part_floats))))
        return fail(SFISTA_ENOMEM, std::string("factor-gradient buffers: ") + cudaGetErrorString(e));
    SF_CUDA(cudaEventRecord(c->ev_in, user));
    SF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    cudaStream_t s = c->stream;
    SF_CUDA(cudaMemcpyAsync(c->Bd, d_b, N * 4, cudaMemcpyDeviceToDevice, s));
    SF_CUDA(cudaMemsetAsync(xb, 0, 3 * N * 8, s));
    SF_CUDA(cudaMemsetAsync(sumV, 0, N * 8, s));
    launch_f32_to_f64(d_gX, xb + (size_t)(iters % 3) * N, N, s);
    if (d_gA) SF_CUDA(cudaMemsetAsync(d_gA, 0, (size_t)r * n * n * 4, s));
    if (d_gB) SF_CUDA(cudaMemsetAsync(d_gB, 0, (size_t)r * m * m * 4, s));
    const float minus_inv = (float)(-inv);
    for (int j = nseg - 1; j >= 0; --j) {
        const int k0 = j * ce, k1 = std::min(iters, k0 + ce);
        // Re-run the segment from its checkpoint, keeping X_k and Y_k.
        launch_f64_to_df(d_ckpt + (size_t)2 * j * N, c->Xb[k0 & 1], N, s);
        launch_f64_to_df(d_ckpt + (size_t)(2 * j + 1) * N, c->Xb[(k0 + 1) & 1], N, s);
        launch_init_state(c->Xb[k0 & 1], c->Xb[(k0 + 1) & 1], c->Y, c->Yop, nullptr, nullptr, 0, N,
                          k0 > 0 ? c->beta_host[k0 - 1] : 0.0, s);
        for (int k = k0 + 1; k <= k1; ++k) {
            launch_df_to_f64(c->Y, segY + (size_t)(k - k0 - 1) * N, N, s);
            enqueue_iteration(c, k, lambda);
            launch_df_to_f64(c->Xb[k & 1], segX + (size_t)(k - k0 - 1) * N, N, s);
        }
        // Reverse sweep over the segment.
        int nb = 0;   // factor-gradient steps buffered
        for (int k = k1; k > k0; --k) {
            double *V = xb + (size_t)(k % 3) * N;
            const double *Xk = segX + (size_t)(k - k0 - 1) * N, *Yk = segY + (size_t)(k - k0 - 1) * N;
            float *Vk = factors ? Vseg + (size_t)nb * N : Vf, *Wk = factors ? Wseg + (size_t)nb * N : Wf;
            float *Yf = factors ? Yseg + (size_t)nb * N : nullptr;
            to_f32_pair_kernel<<<grid1(N), 256, 0, s>>>(V, Vk, factors ? Yk : nullptr, Yf, N);
            As_apply(c, Vk, Wk, s);
            AsT_apply(c, Wk, Tf, s);
            ybar_kernel<<<grid1(N), 256, 0, s>>>(ybar, sumV, V, Tf, L, inv, N);
            launch_dots(Xk, V, N, partial, 256, dots + 2 * (size_t)(k - 1), s);
            if (factors) {
                float *Rf = Rseg + (size_t)nb * N;
                As_apply(c, Yf, Rf, s, EPI_RESIDUAL);   // R_k = A_s Y_k - B
                if (d_gA) {   // B_i V and B_i Y for every term, one launch each
                    launch_band_cols_each(Vk, m, n, c->fB, h.B.lo, h.B.w, r, Useg + (size_t)nb * r * N, s);
                    launch_band_cols_each(Yf, m, n, c->fB, h.B.lo, h.B.w, r, U2seg + (size_t)nb * r * N, s);
                }
                if (d_gB) {
                    launch_band_rows<float>(Rf, m, n, c->fAT, h.AT.lo, h.AT.w, r, Zsseg + (size_t)nb * r * N, s);
                    launch_band_rows<float>(Wk, m, n, c->fAT, h.AT.lo, h.AT.w, r, Zqseg + (size_t)nb * r * N, s);
                }
                if (++nb == scap || k == k0 + 1) {
                    if (d_gA) {
                        GradOperands o = oa;
                        o.S = nb;
                        o.P[0] = Rseg, o.P[1] = Wseg, o.Q[0] = Useg, o.Q[1] = U2seg;
                        o.p_term = 0, o.p_step = (long)N, o.q_term = (long)N, o.q_step = (long)(r * N);
                        launch_grad_gemm(false, vec, o, d_gA, gpart, minus_inv, s);
                    }
                    if (d_gB) {
                        GradOperands o = ob;
                        o.S = nb;
                        o.P[0] = Zsseg, o.P[1] = Zqseg, o.Q[0] = Vseg, o.Q[1] = Yseg;
                        o.p_term = (long)N, o.p_step = (long)(r * N), o.q_term = 0, o.q_step = (long)N;
                        launch_grad_gemm(true, vec, o, d_gB, gpart, minus_inv, s);
                    }
                    nb = 0;
                }
            }
            {
                const double beta = k >= 2 ? c->beta_host[k - 2] : 0.0;   // beta_{k-1}
                step_update_kernel<<<grid1(N), 256, 0, s>>>(xb + (size_t)((k + 2) % 3) * N,
                                                           xb + (size_t)((k + 1) % 3) * N, V, ybar, beta, k >= 2,
                                                           N);
            }
        }
    }
    // dl/dB = A_s (sum_k V) / den
    launch_f64_to_f32(sumV, Vf, N, s);
    As_apply(c, Vf, Wf, s);
    scale_f32<<<grid1(N), 256, 0, s>>>(d_gb, Wf, (float)inv, N);
    std::vector<double> hd(2 * (size_t)iters);
    SF_CUDA(cudaMemcpyAsync(hd.data(), dots, hd.size() * 8, cudaMemcpyDeviceToHost, s));
    SF_CUDA(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int k = 0; k < iters; ++k) acc += hd[2 * (size_t)k];
    *g_lambda = -2.0 * lambda * inv * acc;
    SF_CUDA(cudaGetLastError());
    st = finish_on_user(c, user);
    if (st) return st;
    return drain_status(c);
}
