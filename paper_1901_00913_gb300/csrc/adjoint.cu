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

__global__ void axpy_f64(double *y, const double *x, double a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}
// ybar = (L V - T) * inv
__global__ void ybar_kernel(double *ybar, const double *V, const float *T, double L, double inv, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        ybar[i] = (L * V[i] - (double)T[i]) * inv;
}
__global__ void scale_f32(float *y, const float *x, float a, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// C[I][J] += alpha * sum_t P(I, t) Q(J, t), P(I, t) = P[I*psi + t*pst],
// Q(J, t) = Q[J*qsj + t*qst]; 64 x 64 tiles, 16-deep K slices, 4 x 4 per thread.
template <bool P_I_CONTIG, bool Q_J_CONTIG>
__global__ void __launch_bounds__(256) sgemm_acc(float *C, int ldc, int I, int J, int T, const float *P, long psi,
                                                 long pst, const float *Q, long qsj, long qst, float alpha) {
    __shared__ float Ps[16][64 + 4], Qs[16][64 + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int I0 = blockIdx.y * 64, J0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int t0 = 0; t0 < T; t0 += 16) {
        for (int e = tid; e < 1024; e += 256) {
            int ii, tt;
            if (P_I_CONTIG) { ii = e % 64; tt = e / 64; } else { tt = e % 16; ii = e / 16; }
            const int gi = I0 + ii, gt = t0 + tt;
            Ps[tt][ii] = (gi < I && gt < T) ? P[gi * psi + gt * pst] : 0.f;
            int jj, t2;
            if (Q_J_CONTIG) { jj = e % 64; t2 = e / 64; } else { t2 = e % 16; jj = e / 16; }
            const int gj = J0 + jj, gt2 = t0 + t2;
            Qs[t2][jj] = (gj < J && gt2 < T) ? Q[gj * qsj + gt2 * qst] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Ps[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Qs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = I0 + ty * 4 + i;
        if (gi >= I) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = J0 + tx * 4 + j;
            if (gj < J) C[(size_t)gi * ldc + gj] += alpha * acc[i][j];
        }
    }
}

int grid1(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

// C (I x J) += alpha * P^T Q  with P (T x I), Q (T x J) row-major: contract rows.
void gemm_tn(float *C, int I, int J, int T, const float *P, const float *Q, float alpha, cudaStream_t s) {
    dim3 g((J + 63) / 64, (I + 63) / 64);
    sgemm_acc<true, true><<<g, 256, 0, s>>>(C, J, I, J, T, P, 1, I, Q, 1, J, alpha);
}
// C (I x J) += alpha * P Q^T  with P (I x T), Q (J x T) row-major: contract columns.
void gemm_nt(float *C, int I, int J, int T, const float *P, const float *Q, float alpha, cudaStream_t s) {
    dim3 g((J + 63) / 64, (I + 63) / 64);
    sgemm_acc<false, false><<<g, 256, 0, s>>>(C, J, I, J, T, P, T, 1, Q, T, 1, alpha);
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
    if (iters < 1 || ckpt < 1) return fail(SFISTA_EINVAL, "iters and ckpt_every must be >= 1");
    return SFISTA_OK;
}

// Forward operator A_s x (FP32, banded) into out, using the context's Z.
void As_apply(sfista_ctx *c, const float *x, float *out, cudaStream_t s) {
    const HostSetup &h = c->hs;
    ProxArgs pa{};
    launch_band_rows<float>(x, c->m, c->n, c->fA, h.A.lo, h.A.w, c->r, c->Z, s);
    launch_band_cols<float>(c->Z, c->m, c->n, c->fB, h.B.lo, h.B.w, c->r, EPI_STORE, out, pa, s);
}
void AsT_apply(sfista_ctx *c, const float *x, float *out, cudaStream_t s) {
    const HostSetup &h = c->hs;
    ProxArgs pa{};
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
    Scratch sc;
    double *segX, *segY, *xb, *sumV, *ybar, *dots, *partial, *dot2;
    float *Vf, *Wf, *Tf, *Yf, *Rf, *U, *U2, *Zs, *Zq;
    cudaError_t e;
    if ((e = sc.get(&segX, (size_t)ce * N)) || (e = sc.get(&segY, (size_t)ce * N)) || (e = sc.get(&xb, 3 * N)) ||
        (e = sc.get(&sumV, N)) || (e = sc.get(&ybar, N)) || (e = sc.get(&dots, 2 * (size_t)iters)) ||
        (e = sc.get(&partial, 512)) || (e = sc.get(&dot2, 2)) || (e = sc.get(&Vf, N)) || (e = sc.get(&Wf, N)) ||
        (e = sc.get(&Tf, N)) || (e = sc.get(&Yf, N)) || (e = sc.get(&Rf, N)) || (e = sc.get(&U, N)) ||
        (e = sc.get(&U2, N)) || (e = sc.get(&Zs, (size_t)r * N)) || (e = sc.get(&Zq, (size_t)r * N)))
        return fail(SFISTA_ENOMEM, std::string("adjoint buffers: ") + cudaGetErrorString(e));
    SF_CUDA(cudaEventRecord(c->ev_in, user));
    SF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    cudaStream_t s = c->stream;
    SF_CUDA(cudaMemcpyAsync(c->Bd, d_b, N * 4, cudaMemcpyDeviceToDevice, s));
    SF_CUDA(cudaMemsetAsync(xb, 0, 3 * N * 8, s));
    SF_CUDA(cudaMemsetAsync(sumV, 0, N * 8, s));
    launch_f32_to_f64(d_gX, xb + (size_t)(iters % 3) * N, N, s);
    const bool factors = d_gA || d_gB;
    if (d_gA) SF_CUDA(cudaMemsetAsync(d_gA, 0, (size_t)r * n * n * 4, s));
    if (d_gB) SF_CUDA(cudaMemsetAsync(d_gB, 0, (size_t)r * m * m * 4, s));
    ProxArgs pz{};
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
        for (int k = k1; k > k0; --k) {
            double *V = xb + (size_t)(k % 3) * N;
            const double *Xk = segX + (size_t)(k - k0 - 1) * N, *Yk = segY + (size_t)(k - k0 - 1) * N;
            launch_f64_to_f32(V, Vf, N, s);
            As_apply(c, Vf, Wf, s);
            AsT_apply(c, Wf, Tf, s);
            ybar_kernel<<<grid1(N), 256, 0, s>>>(ybar, V, Tf, L, inv, N);
            axpy_f64<<<grid1(N), 256, 0, s>>>(sumV, V, 1.0, N);
            launch_dots(Xk, V, N, partial, 256, dot2, s);
            SF_CUDA(cudaMemcpyAsync(dots + 2 * (size_t)(k - 1), dot2, 16, cudaMemcpyDeviceToDevice, s));
            if (factors) {
                launch_f64_to_f32(Yk, Yf, N, s);
                ProxArgs pr{};
                pr.Bd = c->Bd;
                launch_band_rows<float>(Yf, m, n, c->fA, h.A.lo, h.A.w, r, c->Z, s);
                launch_band_cols<float>(c->Z, m, n, c->fB, h.B.lo, h.B.w, r, EPI_RESIDUAL, Rf, pr, s);
                if (d_gA) {
                    for (int i = 0; i < r; ++i) {
                        const float *Bi = c->fB + (size_t)i * h.B.w * m;
                        launch_band_cols<float>(Vf, m, n, Bi, h.B.lo, h.B.w, 1, EPI_STORE, U, pz, s);
                        launch_band_cols<float>(Yf, m, n, Bi, h.B.lo, h.B.w, 1, EPI_STORE, U2, pz, s);
                        float *gAi = d_gA + (size_t)i * n * n;
                        gemm_tn(gAi, n, n, m, Rf, U, minus_inv, s);
                        gemm_tn(gAi, n, n, m, Wf, U2, minus_inv, s);
                    }
                }
                if (d_gB) {
                    launch_band_rows<float>(Rf, m, n, c->fAT, h.AT.lo, h.AT.w, r, Zs, s);   // R A_i
                    launch_band_rows<float>(Wf, m, n, c->fAT, h.AT.lo, h.AT.w, r, Zq, s);   // W A_i
                    for (int i = 0; i < r; ++i) {
                        float *gBi = d_gB + (size_t)i * m * m;
                        gemm_nt(gBi, m, m, n, Zs + (size_t)i * N, Vf, minus_inv, s);
                        gemm_nt(gBi, m, m, n, Zq + (size_t)i * N, Yf, minus_inv, s);
                    }
                }
            }
            if (k >= 2) {
                const double beta = c->beta_host[k - 2];   // beta_{k-1}
                axpy_f64<<<grid1(N), 256, 0, s>>>(xb + (size_t)((k - 1) % 3) * N, ybar, 1.0 + beta, N);
                axpy_f64<<<grid1(N), 256, 0, s>>>(xb + (size_t)((k - 2) % 3) * N, ybar, -beta, N);
            }
            SF_CUDA(cudaMemsetAsync(V, 0, N * 8, s));
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
