// C ABI of libsfista: context, setup, the Alg. 2 loop driver and the
// operator entry points.  See include/sfista.h for the contract of each call.
#include <math.h>
#include <string.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ctx.h"
#include "trace.h"
#include "epilogue.cuh"

namespace sfista {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
sfista_status fail(sfista_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

namespace {


// Y_{k0+1} = X + beta (X - Xp) in double-float, plus its operand copies.
__global__ void init_state_kernel(const float2 *X, const float2 *Xp, float2 *Y, float *Yop, void *Yhi, void *Ylo,
                                  int split_kind, size_t count, float2 beta) {
    ProxArgs pa{};
    pa.Yop = Yop;
    pa.Yhi = Yhi;
    pa.Ylo = Ylo;
    pa.split_kind = split_kind;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        const float2 y = dfp::momentum(X[i], Xp[i], beta);
        Y[i] = y;
        store_operands(pa, i, y);
    }
}

// The FP32 state of a tensor-core form at the start of a solve: X_k0 rounded
// to FP32 and Y_{k0+1} = X + beta (X - Xp) formed in FP32 exactly as the
// prox epilogue forms it, so a resumed solve continues bit for bit; then
// the operand copies of that Y.
__global__ void init_state32_kernel(const float2 *X, const float2 *Xp, float *X32, float *Y32, void *Yhi, void *Ylo,
                                    int split_kind, size_t count, float beta) {
    ProxArgs pa{};
    pa.Yhi = Yhi;
    pa.Ylo = Ylo;
    pa.split_kind = split_kind;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        const float x = dfp::to_float(X[i]), xp = dfp::to_float(Xp[i]);
        const float y = fmaf(beta, x - xp, x);
        X32[i] = x;
        Y32[i] = y;
        store_operands32(pa, i, y);
    }
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t count, cudaStream_t s) {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(count, 1));
    if (e) return e;
    return cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s);
}

}  // namespace

void launch_init_state(const float2 *X, const float2 *Xp, float2 *Y, float *Yop, void *Yhi, void *Ylo, int split_kind,
                       size_t count, double beta, cudaStream_t s) {
    init_state_kernel<<<1024, 256, 0, s>>>(X, Xp, Y, Yop, Yhi, Ylo, split_kind, count, dfp::from_double(beta));
}

namespace {

}  // namespace
}  // namespace sfista

using namespace sfista;


namespace {

void ctx_free(sfista_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gemm) gemm_destroy(c->gemm);
    if (c->fft) fftconv_destroy(c->fft);
    void *ptrs[] = {c->dA, c->dAT, c->dB, c->dBT, c->fA, c->fAT, c->fB, c->fBT, c->Bd, c->Yop, c->Z,
                    c->R, c->tmp, c->Xb[0], c->Xb[1], c->Y, c->status, c->beta, c->bar,
                    c->Xf[0], c->Xf[1], c->Yf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // namespace
sfista_status sfista::ensure_beta(sfista_ctx *c, int k_end) {
    if (k_end <= c->beta_len) return SFISTA_OK;
    int len = std::max(k_end, 2 * c->beta_len);
    momentum_table(len, &c->beta_host);
    SF_CUDA(cudaStreamSynchronize(c->stream));
    if (c->beta) cudaFree(c->beta);
    c->beta = nullptr;
    std::vector<float2> bdf(len);
    for (int i = 0; i < len; ++i) bdf[i] = dfp::from_double(c->beta_host[i]);
    SF_CUDA(cudaMalloc((void **)&c->beta, sizeof(float2) * len));
    SF_CUDA(cudaMemcpy(c->beta, bdf.data(), sizeof(float2) * len, cudaMemcpyHostToDevice));
    c->beta_len = len;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SFISTA_OK;
}
namespace {

// Forward operator with the residual epilogue, then the adjoint with the
// prox + momentum epilogue: one iteration k of Alg. 2 (Steps 1-3).
}  // namespace
ProxArgs sfista::prox_args(sfista_ctx *c, int k, double lam) {
    ProxArgs pa{};
    pa.Bd = c->Bd;
    pa.Xin = c->Xb[(k - 1) & 1];
    pa.Xout = c->Xb[k & 1];
    pa.Y = c->Y;
    if (c->Xf[0]) {
        pa.Xin32 = c->Xf[(k - 1) & 1];
        pa.Xout32 = c->Xf[k & 1];
        pa.Y32 = c->Yf;
    }
    pa.Yop = c->Yop;
    pa.beta = c->beta;
    pa.k = k;
    pa.L = c->L;
    pa.lam2 = lam * lam;
    pa.inv_den = dfp::from_double(1.0 / (c->L + lam * lam));
    pa.shrink = dfp::from_double(c->L / (c->L + lam * lam));
    pa.project = c->opts.project_nonneg;
    pa.tau = dfp::from_double(c->opts.l1 / (c->L + lam * lam));
    pa.status = c->status;
    return pa;
}
namespace {

// The context's problem as a banded descriptor (geometry and buffers; pa
// left default).
BandProb ctx_prob(const sfista_ctx *c) {
    const HostSetup &h = c->hs;
    BandProb P{};
    P.m = c->m;
    P.n = c->n;
    P.r = c->r;
    P.fA = c->fA;
    P.fB = c->fB;
    P.fAT = c->fAT;
    P.fBT = c->fBT;
    P.loA = h.A.lo;
    P.wA = h.A.w;
    P.loB = h.B.lo;
    P.wB = h.B.w;
    P.loAT = h.AT.lo;
    P.wAT = h.AT.w;
    P.loBT = h.BT.lo;
    P.wBT = h.BT.w;
    P.Z = c->Z;
    P.R = c->R;
    P.tfwd = interior_fwd(c);
    P.tadj = interior_adj(c);
    P.th = c->pth;
    return P;
}

// Stage `st` (0..3) of iteration k; see sfista_time_stages for the numbering.
void enqueue_stage(sfista_ctx *c, int st, const ProxArgs &pa) {
    const HostSetup &h = c->hs;
    if (is_fft(c->op)) {
        // Stage 0: Passes A and B of A_s Y (or A Y); 1: Pass C with the
        // residual fused with the adjoint's Pass A on it (R stays on chip);
        // 2: the adjoint's Pass B; 3: its Pass C with Step 1 + Step 3.
        switch (st) {
            case 0: fftconv_part(c->fft, 0, false, c->Yop, EPI_STORE, nullptr, pa, c->stream); break;
            case 1: fftconv_residual_adjoint(c->fft, pa, c->stream); break;
            case 2: fftconv_adjoint_columns(c->fft, c->stream); break;
            default: fftconv_part(c->fft, 1, true, nullptr, EPI_PROX, nullptr, pa, c->stream); break;
        }
    } else if (fused_apply(c)) {
        // Two launches per iteration: stage 0 = forward operator + residual,
        // stage 2 = adjoint + shrink / momentum (stages 1 and 3 are empty).
        if (st == 0)
            launch_band_op_fused(c->Yop, c->m, c->n, c->r, c->fA, h.A.lo, h.A.w, c->fB, h.B.lo, h.B.w, EPI_RESIDUAL,
                                 c->R, pa, interior_fwd(c), c->stream);
        else if (st == 2)
            launch_band_op_fused(c->R, c->m, c->n, c->r, c->fAT, h.AT.lo, h.AT.w, c->fBT, h.BT.lo, h.BT.w, EPI_PROX,
                                 nullptr, pa, interior_adj(c), c->stream);
    } else if (is_banded(c->op)) {
        switch (st) {
            case 0: launch_band_rows<float>(c->Yop, c->m, c->n, c->fA, h.A.lo, h.A.w, c->r, c->Z, c->stream,
                                            c->chunk[0]); break;
            case 1: launch_band_cols<float>(c->Z, c->m, c->n, c->fB, h.B.lo, h.B.w, c->r, EPI_RESIDUAL, c->R, pa,
                                            c->stream, c->chunk[1]); break;
            case 2: launch_band_rows<float>(c->R, c->m, c->n, c->fAT, h.AT.lo, h.AT.w, c->r, c->Z, c->stream,
                                            c->chunk[2]); break;
            default: launch_band_cols<float>(c->Z, c->m, c->n, c->fBT, h.BT.lo, h.BT.w, c->r, EPI_PROX, nullptr,
                                             pa, c->stream, c->chunk[3]); break;
        }
    } else {
        gemm_stage(c->gemm, st, pa, c->stream);
    }
}

}  // namespace
void sfista::enqueue_iteration(sfista_ctx *c, int k, double lam) {
    ProxArgs pa = prox_args(c, k, lam);
    if (c->gemm && c->opts.refine_every > 0 && k % c->opts.refine_every == 0) {
        // A refinement iteration runs all of Step 1 in FP32 on the band
        // kernels: R_k = A_s Y_k - B (rows, then columns with the residual
        // epilogue) on the FP32 value of Y_k, then G = A_s^T R_k (rows, then
        // columns with the Step 1 + Step 3 epilogue on the form's own state),
        // writing Y_{k+1} in the split operand format of the next GEMMs.
        const HostSetup &h = c->hs;
        const float *y = c->Yf;   // the FP32 state holds Y_k itself
        if (!y) {                 // double-float state: its FP32 value
            launch_df_to_f32(c->Y, c->Yop, c->N, c->stream);
            y = c->Yop;
        }
        launch_band_rows<float>(y, c->m, c->n, c->fA, h.A.lo, h.A.w, c->r, c->Z, c->stream, c->chunk[0]);
        launch_band_cols<float>(c->Z, c->m, c->n, c->fB, h.B.lo, h.B.w, c->r, EPI_RESIDUAL, c->R, pa, c->stream,
                                c->chunk[1]);
        ProxArgs pr = pa;
        gemm_state_operands(c->gemm, &pr.Yhi, &pr.Ylo, &pr.split_kind);
        pr.Yop = nullptr;
        launch_band_rows<float>(c->R, c->m, c->n, c->fAT, h.AT.lo, h.AT.w, c->r, c->Z, c->stream, c->chunk[2]);
        launch_band_cols<float>(c->Z, c->m, c->n, c->fBT, h.BT.lo, h.BT.w, c->r, EPI_PROX, nullptr, pr, c->stream,
                                c->chunk[3]);
        return;
    }
    for (int st = 0; st < 4; ++st) enqueue_stage(c, st, pa);
}
namespace {

sfista_status run_loop(sfista_ctx *c, double lam, int k0, int iters) {
    TraceRange trace_("sfista iterations");
    if (iters <= 0) return SFISTA_OK;
    if (c->op == SFISTA_OP_BANDED_PERSISTENT) {
        const HostSetup &h = c->hs;
        ProxArgs pa = prox_args(c, k0 + 1, lam);
        if (c->pfused) {
            BandProb P = ctx_prob(c);
            P.pa = pa;
            P.pa.Xin = c->Xb[0];
            P.pa.Xout = c->Xb[1];
            SF_CUDA(launch_band_solve_fused(c->pgrid, c->psmem, P, k0, iters, c->bar, c->stream));
        }
        else
            SF_CUDA(launch_persistent(c->pgrid, c->psmem, c->prows_chunk, c->pcols_chunk, c->m, c->n, c->r, c->fA,
                                      h.A, c->fB, h.B, c->fAT, h.AT, c->fBT, h.BT, c->Z, c->R, c->Xb[0], c->Xb[1], pa,
                                      k0, iters, c->bar, c->stream));
        return SFISTA_OK;
    }
    if (!c->opts.use_graph) {
        for (int k = k0 + 1; k <= k0 + iters; ++k) enqueue_iteration(c, k, lam);
        SF_CUDA(cudaGetLastError());
        return SFISTA_OK;
    }
    if (!(c->gexec && c->g_k0 == k0 && c->g_iters == iters && c->g_lam == lam)) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        TraceRange capture_("sfista graph capture");
        SF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        for (int k = k0 + 1; k <= k0 + iters; ++k) enqueue_iteration(c, k, lam);
        cudaError_t le = cudaGetLastError();
        cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(SFISTA_ECUDA, std::string("graph capture failed: ") +
                                          cudaGetErrorString(le != cudaSuccess ? le : ee));
        }
        cudaError_t ie = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            c->gexec = nullptr;
            return fail(SFISTA_ECUDA, std::string("graph instantiate failed: ") + cudaGetErrorString(ie));
        }
        c->g_k0 = k0;
        c->g_iters = iters;
        c->g_lam = lam;
    }
    SF_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    return SFISTA_OK;
}

// FP64 power iteration for lambda_max(A_s^T A_s) with the banded kernels.
sfista_status power_lipschitz(sfista_ctx *c, double tol, int maxit, double *L_out) {
    TraceRange trace_("sfista lipschitz");
    const HostSetup &h = c->hs;
    size_t N = c->N;
    double *v = nullptr, *u = nullptr, *w = nullptr, *Zd = nullptr, *partial = nullptr, *dot = nullptr;
    const int nblk = 256;
    sfista_status st = SFISTA_OK;
    double hdot[2] = {0, 0}, mu = 0, prev = 0;
    ProxArgs pa{};
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc((void **)&v, N * 8)) || (e = cudaMalloc((void **)&u, N * 8)) ||
        (e = cudaMalloc((void **)&w, N * 8)) || (e = cudaMalloc((void **)&Zd, N * 8 * c->r)) ||
        (e = cudaMalloc((void **)&partial, nblk * 2 * 8)) || (e = cudaMalloc((void **)&dot, 2 * 8))) {
        st = fail(SFISTA_ENOMEM, std::string("power iteration buffers: ") + cudaGetErrorString(e));
        goto done;
    }
    launch_seed_image(v, N, c->stream);
    launch_dots(v, v, N, partial, nblk, dot, c->stream);
    launch_scale(v, N, dot, c->stream);
    for (int it = 1; it <= maxit; ++it) {
        launch_band_rows<double>(v, c->m, c->n, c->dA, h.A.lo, h.A.w, c->r, Zd, c->stream);
        launch_band_cols<double>(Zd, c->m, c->n, c->dB, h.B.lo, h.B.w, c->r, EPI_STORE, u, pa, c->stream);
        launch_band_rows<double>(u, c->m, c->n, c->dAT, h.AT.lo, h.AT.w, c->r, Zd, c->stream);
        launch_band_cols<double>(Zd, c->m, c->n, c->dBT, h.BT.lo, h.BT.w, c->r, EPI_STORE, w, pa, c->stream);
        launch_dots(v, w, N, partial, nblk, dot, c->stream);
        launch_scale(w, N, dot, c->stream);
        std::swap(v, w);
        if ((e = cudaMemcpyAsync(hdot, dot, 16, cudaMemcpyDeviceToHost, c->stream)) ||
            (e = cudaStreamSynchronize(c->stream))) {
            st = fail(SFISTA_ECUDA, std::string("power iteration: ") + cudaGetErrorString(e));
            goto done;
        }
        mu = hdot[0];
        if (!isfinite(mu) || !(hdot[1] > 0)) {
            st = fail(SFISTA_ENUMERIC, "power iteration produced a non-finite or zero vector");
            goto done;
        }
        if (it > 1 && fabs(mu - prev) <= tol * fabs(mu)) break;
        prev = mu;
    }
    *L_out = mu;
done:
    cudaFree(v);
    cudaFree(u);
    cudaFree(w);
    cudaFree(Zd);
    cudaFree(partial);
    cudaFree(dot);
    return st;
}

// The FFT engine of a sfista_setup context: kernel K = sum_i c_i d_i^T.
sfista_status make_fft(sfista_ctx *c) {
    const HostSetup &h = c->hs;
    std::vector<double> K((size_t)h.p * h.q, 0.0);
    for (int i = 0; i < h.r; ++i)
        for (int k = 0; k < h.p; ++k)
            for (int l = 0; l < h.q; ++l) K[(size_t)k * h.q + l] += h.C[(size_t)i * h.p + k] * h.D[(size_t)i * h.q + l];
    return fftconv_create(&c->fft, K.data(), h.p, h.q, h.cr, h.cc, c->m, c->n, h.bc);
}

// lambda_max(Op^T Op) by power iteration with the context's FFT operator
// (FP32 applications, FP64 iterate and sums).  The FP32 operator leaves the
// Rayleigh quotient about 1e-7 noisy, so the stopping tolerance is at least
// 2e-7.
sfista_status power_lipschitz_fft(sfista_ctx *c, double tol, int maxit, double *L_out) {
    TraceRange trace_("sfista lipschitz (FFT operator)");
    tol = std::max(tol, 2e-7);
    size_t N = c->N;
    double *v = nullptr, *w = nullptr, *partial = nullptr, *dot = nullptr;
    const int nblk = 256;
    sfista_status st = SFISTA_OK;
    double hdot[2] = {0, 0}, mu = 0, prev = 0;
    ProxArgs pa{};
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc((void **)&v, N * 8)) || (e = cudaMalloc((void **)&w, N * 8)) ||
        (e = cudaMalloc((void **)&partial, nblk * 2 * 8)) || (e = cudaMalloc((void **)&dot, 2 * 8))) {
        st = fail(SFISTA_ENOMEM, std::string("power iteration buffers: ") + cudaGetErrorString(e));
        goto done;
    }
    launch_seed_image(v, N, c->stream);
    launch_dots(v, v, N, partial, nblk, dot, c->stream);
    launch_scale(v, N, dot, c->stream);
    for (int it = 1; it <= maxit; ++it) {
        launch_f64_to_f32(v, c->Yop, N, c->stream);
        fftconv_apply(c->fft, false, c->Yop, EPI_STORE, c->tmp, pa, c->stream);
        fftconv_apply(c->fft, true, c->tmp, EPI_STORE, c->R, pa, c->stream);
        launch_f32_to_f64(c->R, w, N, c->stream);
        launch_dots(v, w, N, partial, nblk, dot, c->stream);
        launch_scale(w, N, dot, c->stream);
        std::swap(v, w);
        if ((e = cudaMemcpyAsync(hdot, dot, 16, cudaMemcpyDeviceToHost, c->stream)) ||
            (e = cudaStreamSynchronize(c->stream))) {
            st = fail(SFISTA_ECUDA, std::string("power iteration: ") + cudaGetErrorString(e));
            goto done;
        }
        mu = hdot[0];
        if (!isfinite(mu) || !(hdot[1] > 0)) {
            st = fail(SFISTA_ENUMERIC, "power iteration produced a non-finite or zero vector");
            goto done;
        }
        if (it > 1 && fabs(mu - prev) <= tol * fabs(mu)) break;
        prev = mu;
    }
    *L_out = mu;
done:
    cudaFree(v);
    cudaFree(w);
    cudaFree(partial);
    cudaFree(dot);
    return st;
}

// Band storage (geometry of `like`: lo, w, len, r) of dense factors F
// (r x len x len, row-major); transpose = true stores F_i^T.  false if F has
// a nonzero entry outside that band.
bool band_from_dense(const double *F, const Band &like, bool transpose, Band *out) {
    const int r = like.r, len = like.len, lo = like.lo, w = like.w;
    *out = like;
    std::fill(out->band.begin(), out->band.end(), 0.0);
    for (int i = 0; i < r; ++i)
        for (int row = 0; row < len; ++row)
            for (int col = 0; col < len; ++col) {
                // entry (row, col) of the stored matrix G = F_i or F_i^T
                const double v = transpose ? F[((size_t)i * len + col) * len + row] : F[((size_t)i * len + row) * len + col];
                const int k = col - row - lo;
                if (k >= 0 && k < w)
                    out->band[((size_t)i * w + k) * len + row] = v;
                else if (v != 0.0)
                    return false;
            }
    return true;
}

// Rewrites a context's device band tables (FP64, FP32 + its Toeplitz row)
// from host band storage of unchanged geometry.
cudaError_t store_band(sfista_ctx *c, const Band &b, double *d64, float *d32, int2 *interior) {
    cudaError_t e = cudaMemcpyAsync(d64, b.band.data(), sizeof(double) * b.band.size(), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e) return e;
    std::vector<float> f(b.band.begin(), b.band.end());
    const int len = b.len, ref = len / 2, cnt = b.r * b.w;
    int i0 = 0, i1 = 0;
    band_interior(f.data(), len, cnt, &i0, &i1);
    *interior = make_int2(i0, i1);
    for (int t = 0; t < cnt; ++t) f.push_back(f[(size_t)t * len + ref]);
    e = cudaMemcpyAsync(d32, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, c->stream);
    if (e) return e;
    return cudaStreamSynchronize(c->stream);
}

sfista_status check_ctx(const sfista_ctx *c) {
    if (!c) return fail(SFISTA_EINVAL, "context is NULL");
    return SFISTA_OK;
}

// Reads and clears the device status word (synchronises the context stream).
}  // namespace
sfista_status sfista::drain_status(sfista_ctx *c) {
    unsigned s = 0;
    SF_CUDA(cudaStreamSynchronize(c->stream));
    SF_CUDA(cudaMemcpy(&s, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (s) SF_CUDA(cudaMemset(c->status, 0, sizeof(unsigned)));
    if (s & DEV_TIMEOUT) return fail(SFISTA_ETIMEOUT, "a device-side wait exceeded its bound");
    if (s & DEV_BADARG) return fail(SFISTA_EINVAL, "a kernel rejected its arguments");
    if (s & DEV_NONFINITE) return fail(SFISTA_ENUMERIC, "non-finite value in the input or the iterates");
    return SFISTA_OK;
}
namespace {

}  // namespace
sfista_status sfista::solve_core(sfista_ctx *c, const float *d_b, double lam, int k0, int iters,
                         const double *X_in, const double *Xprev_in, cudaStream_t user) {
    if (!d_b) return fail(SFISTA_EINVAL, "b is NULL");
    if (!(lam >= 0) || !isfinite(lam)) return fail(SFISTA_EINVAL, "lambda must be finite and >= 0");
    if (iters < 0 || k0 < 0) return fail(SFISTA_EINVAL, "iters and k0 must be >= 0");
    sfista_status st = ensure_beta(c, k0 + iters + 1);
    if (st) return st;
    SF_CUDA(cudaEventRecord(c->ev_in, user));
    SF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    size_t N = c->N;
    SF_CUDA(cudaMemcpyAsync(c->Bd, d_b, N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    launch_check_finite(c->Bd, N, c->status, c->stream);
    float2 *Xk = c->Xb[k0 & 1], *Xkm = c->Xb[(k0 + 1) & 1];
    if (X_in) launch_f64_to_df(X_in, Xk, N, c->stream);
    else SF_CUDA(cudaMemsetAsync(Xk, 0, N * 8, c->stream));
    if (k0 > 0 && Xprev_in) launch_f64_to_df(Xprev_in, Xkm, N, c->stream);
    else SF_CUDA(cudaMemcpyAsync(Xkm, Xk, N * 8, cudaMemcpyDeviceToDevice, c->stream));
    double beta0 = k0 > 0 ? c->beta_host[k0 - 1] : 0.0;
    void *yhi = nullptr, *ylo = nullptr;
    int split = 0;
    if (c->gemm) gemm_state_operands(c->gemm, &yhi, &ylo, &split);
    launch_init_state(Xk, Xkm, c->Y, c->Yop, yhi, ylo, split, N, beta0, c->stream);
    if (c->Xf[0])   // the FP32 state the tensor-core prox epilogue iterates on
        init_state32_kernel<<<1024, 256, 0, c->stream>>>(Xk, Xkm, c->Xf[k0 & 1], c->Yf, yhi, ylo, split, N,
                                                        (float)beta0);
    if (c->gemm) gemm_prepare_solve(c->gemm, c->Bd, c->stream);
    SF_CUDA(cudaGetLastError());
    st = run_loop(c, lam, k0, iters);
    if (st) return st;
    if (c->Xf[0] && iters > 0) {   // back into the double-float buffers: X_ke, X_{ke-1}, Y_{ke+1}
        const int ke = k0 + iters;
        launch_f32_to_df(c->Xf[ke & 1], c->Xb[ke & 1], N, c->stream);
        launch_f32_to_df(c->Xf[(ke + 1) & 1], c->Xb[(ke + 1) & 1], N, c->stream);
        launch_f32_to_df(c->Yf, c->Y, N, c->stream);
    }
    SF_CUDA(cudaGetLastError());
    return SFISTA_OK;
}
namespace {

}  // namespace
sfista_status sfista::finish_on_user(sfista_ctx *c, cudaStream_t user) {
    SF_CUDA(cudaEventRecord(c->ev_out, c->stream));
    SF_CUDA(cudaStreamWaitEvent(user, c->ev_out, 0));
    return SFISTA_OK;
}
namespace {

}  // namespace


struct sfista_batch {
    std::vector<sfista_ctx *> ctxs;
    int dev = 0;
    bool gemm = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    GemmBatch *gb = nullptr;
    BandProb *d_probs = nullptr;
    std::vector<BandProb> h_probs;
    std::vector<BandProb> sent;   // the table d_probs holds for the one-launch form (empty: unknown)
    BandItem *d_items[4] = {nullptr, nullptr, nullptr, nullptr};
    int nitems[4] = {0, 0, 0, 0};
    size_t smem = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_iters = -1;
    std::vector<double> g_lams;
    // FP32 batches whose tiles all fit as co-resident blocks: the whole batch
    // solve as one cooperative launch (fused_ok), taken while use_fused.
    bool fused_ok = false, use_fused = false;
    int2 *d_fitems = nullptr;
    int fnitems = 0;
    size_t fsmem = 0;
    unsigned *bar = nullptr;
};

namespace {

void batch_free(sfista_batch *b) {
    if (!b) return;
    DeviceGuard g(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gb) gemm_batch_destroy(b->gb);
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->d_fitems) cudaFree(b->d_fitems);
    if (b->bar) cudaFree(b->bar);
    for (int st = 0; st < 4; ++st)
        if (b->d_items[st]) cudaFree(b->d_items[st]);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

void batch_stage(sfista_batch *b, int st, int k) {
    if (b->gemm) gemm_batch_stage(b->gb, st, k, b->stream);
    else launch_band_grouped_stage(st, b->d_probs, b->d_items[st], b->nitems[st], k, b->smem, b->stream);
}

// Term chunks, work lists and shared-memory size of a banded batch.  budget 0:
// each problem's own chunks (tuned, else the default rule); otherwise every
// problem takes the largest chunks whose tiles fit in `budget` bytes, so the
// one shared-memory size of the grouped launches stays within it.
sfista_status band_batch_plan(sfista_batch *b, size_t budget) {
    const int np = (int)b->ctxs.size();
    std::vector<int> order(np);
    for (int p = 0; p < np; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)b->ctxs[x]->N * b->ctxs[x]->r > (double)b->ctxs[y]->N * b->ctxs[y]->r;
    });
    b->smem = 0;
    for (int p = 0; p < np; ++p) {
        sfista_ctx *c = b->ctxs[p];
        const HostSetup &h = c->hs;
        BandProb &P = b->h_probs[p];
        const int wmax = std::max(std::max(h.A.w, h.AT.w), std::max(h.B.w, h.BT.w));
        int rq = c->chunk[0], cq = c->chunk[1];
        if (budget) {
            rq = cq = 1;
            while (rq < c->r && band_smem_f32(true, wmax, rq + 1) <= budget) ++rq;
            while (cq < c->r && band_smem_f32(false, wmax, cq + 1) <= budget) ++cq;
        }
        size_t sm = 0;
        P.vec = c->m % 4 == 0 && c->n % 4 == 0;   // the buffers are cudaMalloc'ed (aligned)
        grouped_chunks(c->r, wmax, P.vec, rq, cq, &P.rows_chunk, &P.cols_chunk, &sm);
        b->smem = std::max(b->smem, sm);
    }
    std::vector<BandItem> items[4];
    for (int p : order) {
        const BandProb &P = b->h_probs[p];
        const int nq = (P.r + P.rows_chunk - 1) / P.rows_chunk;
        for (int q = 0; q < nq; ++q)
            for (int t = 0; t < band_rows_tiles(P.m, P.n, P.vec); ++t) items[0].push_back(BandItem{p, q, t, 0});
        for (int t = 0; t < band_cols_tiles(P.m, P.n, P.vec); ++t) items[1].push_back(BandItem{p, 0, t, 0});
    }
    items[2] = items[0];
    items[3] = items[1];
    cudaError_t e = band_grouped_prepare(b->smem);
    if (e) return fail(SFISTA_ENOTSUP, std::string("grouped banded kernels: ") + cudaGetErrorString(e));
    for (int st = 0; st < 4; ++st) {
        if (b->d_items[st]) {
            cudaFree(b->d_items[st]);
            b->d_items[st] = nullptr;
        }
        b->nitems[st] = (int)items[st].size();
        if ((e = cudaMalloc((void **)&b->d_items[st], items[st].size() * sizeof(BandItem))) ||
            (e = cudaMemcpy(b->d_items[st], items[st].data(), items[st].size() * sizeof(BandItem),
                            cudaMemcpyHostToDevice)))
            return fail(SFISTA_ENOMEM, std::string("grouped work lists: ") + cudaGetErrorString(e));
    }
    if (b->gexec) {   // captured with the old work lists
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->g_iters = -1;
    }
    return SFISTA_OK;
}

}  // namespace

extern "C" {

void sfista_default_opts(sfista_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->prec = SFISTA_FP32;
    o->op = SFISTA_OP_AUTO;
    o->project_nonneg = 0;
    o->use_graph = 1;
    o->lipschitz = 0.0;
    o->lipschitz_tol = 1e-10;
    o->lipschitz_maxit = 1000;
    o->device = -1;
    o->l1 = 0.0;
    o->refine_every = 0;
    o->tile_override = 0;
    o->gemm_bn = 0;
    o->gemm_resident_panels = 0;
}

sfista_status sfista_setup(const double *psf, int psf_rows, int psf_cols, int center_row,
                           int center_col, int img_rows, int img_cols, sfista_bc bc, int r,
                           const sfista_opts *opts, sfista_ctx **out) {
    TraceRange trace_("sfista_setup");
    if (!out) return fail(SFISTA_EINVAL, "out is NULL");
    *out = nullptr;
    sfista_opts o;
    sfista_default_opts(&o);
    if (opts) o = *opts;
    if (o.prec < SFISTA_FP32 || o.prec > SFISTA_BF16X3) return fail(SFISTA_EINVAL, "unknown precision");
    if (o.op < SFISTA_OP_AUTO || o.op > SFISTA_OP_FFT) return fail(SFISTA_EINVAL, "unknown operator form");
    if (!(o.lipschitz <= 0.0 || isfinite(o.lipschitz))) return fail(SFISTA_EINVAL, "lipschitz must be finite");
    if (!(o.l1 >= 0.0) || !isfinite(o.l1)) return fail(SFISTA_EINVAL, "l1 must be finite and >= 0");
    if (o.refine_every < 0) return fail(SFISTA_EINVAL, "refine_every must be >= 0");
    if (o.tile_override != 0 && (o.tile_override < 16 || o.tile_override > 64 || o.tile_override % 4))
        return fail(SFISTA_EINVAL, "tile_override must be 0 or a multiple of 4 from 16 to 64");
    if (o.gemm_bn != 0 && o.gemm_bn != 64 && o.gemm_bn != 128 && o.gemm_bn != 256)
        return fail(SFISTA_EINVAL, "gemm_bn must be 0, 64, 128 or 256");
    if (o.gemm_resident_panels != 0 && o.gemm_resident_panels != 1)
        return fail(SFISTA_EINVAL, "gemm_resident_panels must be 0 or 1");
    if (center_row == -1 && psf_rows > 0) center_row = (psf_rows - 1) / 2;
    if (center_col == -1 && psf_cols > 0) center_col = (psf_cols - 1) / 2;
    sfista_ctx *c = new (std::nothrow) sfista_ctx();
    if (!c) return fail(SFISTA_ENOMEM, "context allocation failed");
    sfista_status st = host_setup(psf, psf_rows, psf_cols, center_row, center_col, img_rows, img_cols,
                                  bc, r, &c->hs);
    if (st) {
        delete c;
        return st;
    }
    c->opts = o;
    c->m = img_rows;
    c->n = img_cols;
    c->r = r;
    c->N = (size_t)img_rows * img_cols;
    c->prec = o.prec;
    c->op = o.op;
    if (c->op == SFISTA_OP_AUTO) {
        // Measured on GB300: one kernel per operator application wins while the
        // halo rows it recomputes stay below ~1.5x the tile (band <= 48) and the
        // image is small enough for launch latency to dominate; otherwise the
        // two-pass form.  When every tile of the fused form also has its own
        // resident block, the whole solve runs as one launch (below).
        // Tensor-core forms default to band-aware GEMMs.
        const int wl = std::max(c->hs.B.w, c->hs.BT.w);
        const bool small = (size_t)img_rows * img_cols <= ((size_t)1 << 20) && wl <= 48;
        c->op = (c->prec == SFISTA_FP32) ? (small ? SFISTA_OP_BANDED_FUSED : SFISTA_OP_BANDED) : SFISTA_OP_GEMM_BAND;
    }
    if ((is_banded(c->op) || is_fft(c->op)) && c->prec != SFISTA_FP32) {
        delete c;
        return fail(SFISTA_ENOTSUP, "the banded and FFT operator forms run in FP32 only");
    }
    if (o.device < 0) {
        if (cudaGetDevice(&c->dev) != cudaSuccess) {
            delete c;
            return fail(SFISTA_ECUDA, "no CUDA device");
        }
    } else {
        c->dev = o.device;
    }
    DeviceGuard g(c->dev);
    auto bail = [&](sfista_status s) {
        ctx_free(c);
        return s;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)))
        return bail(fail(SFISTA_ECUDA, std::string("stream/event: ") + cudaGetErrorString(e)));
    const HostSetup &h = c->hs;
    int wmax = std::max(std::max(h.A.w, h.AT.w), std::max(h.B.w, h.BT.w));
    if ((e = band_set_smem_limits(wmax)))
        return bail(fail(SFISTA_ENOTSUP, std::string("band too wide for shared memory: ") + cudaGetErrorString(e)));
    std::vector<float> tmpf;
    // FP32 tables are followed by the row of the middle output index (r x w
    // values); `interior` is the widest range around it whose rows hold the
    // same FP32 values bit for bit (the Toeplitz interior of Sec. 2's T + H).
    auto up_band = [&](const Band &b, double **d64, float **d32, int2 *interior) -> cudaError_t {
        cudaError_t ee = upload(d64, b.band.data(), b.band.size(), c->stream);
        if (ee) return ee;
        tmpf.assign(b.band.begin(), b.band.end());
        const int len = b.len, ref = len / 2, cnt = b.r * b.w;
        int i0 = 0, i1 = 0;
        band_interior(tmpf.data(), len, cnt, &i0, &i1);
        *interior = make_int2(i0, i1);
        for (int t = 0; t < cnt; ++t) tmpf.push_back(tmpf[(size_t)t * len + ref]);
        ee = upload(d32, tmpf.data(), tmpf.size(), c->stream);
        if (ee) return ee;
        return cudaStreamSynchronize(c->stream);
    };
    if ((e = up_band(h.A, &c->dA, &c->fA, &c->interior[0])) || (e = up_band(h.AT, &c->dAT, &c->fAT, &c->interior[1])) ||
        (e = up_band(h.B, &c->dB, &c->fB, &c->interior[2])) || (e = up_band(h.BT, &c->dBT, &c->fBT, &c->interior[3])))
        return bail(fail(SFISTA_ENOMEM, std::string("factor upload: ") + cudaGetErrorString(e)));
    size_t N = c->N;
    if ((e = cudaMalloc((void **)&c->Bd, N * 4)) || (e = cudaMalloc((void **)&c->Yop, N * 4)) ||
        (e = cudaMalloc((void **)&c->Z, N * 4 * r)) || (e = cudaMalloc((void **)&c->R, N * 4)) ||
        (e = cudaMalloc((void **)&c->tmp, N * 4)) || (e = cudaMalloc((void **)&c->Xb[0], N * 8)) ||
        (e = cudaMalloc((void **)&c->Xb[1], N * 8)) || (e = cudaMalloc((void **)&c->Y, N * 8)) ||
        (e = cudaMalloc((void **)&c->status, 16)))
        return bail(fail(SFISTA_ENOMEM, std::string("state buffers: ") + cudaGetErrorString(e)));
    if ((e = cudaMemset(c->status, 0, 16))) return bail(fail(SFISTA_ECUDA, cudaGetErrorString(e)));
    if (c->op == SFISTA_OP_BANDED_FUSED &&
        !band_op_fused_prepare(c->r, std::max(h.A.w, h.AT.w), std::max(h.B.w, h.BT.w))) {
        if (o.op == SFISTA_OP_BANDED_FUSED) return bail(fail(SFISTA_ENOTSUP, "fused banded tile exceeds shared memory"));
        c->op = SFISTA_OP_BANDED;   // automatic choice falls back to the two-pass form
    }
    if (o.op == SFISTA_OP_AUTO && c->op == SFISTA_OP_BANDED_FUSED) {
        int grid = 0;
        size_t smem = 0;
        int th = 32;
        if (o.tile_override ? band_solve_fused_config_th(ctx_prob(c), c->dev, o.tile_override, &grid, &smem)
                            : band_solve_fused_config(ctx_prob(c), c->dev, &grid, &smem, &th))
            c->op = SFISTA_OP_BANDED_PERSISTENT;
    }
    if (c->op == SFISTA_OP_BANDED_PERSISTENT) {
        if ((e = cudaMalloc((void **)&c->bar, kBarrierBytes)) || (e = cudaMemset(c->bar, 0, kBarrierBytes)))
            return bail(fail(SFISTA_ENOMEM, std::string("barrier words: ") + cudaGetErrorString(e)));
        c->pfused = o.tile_override
                        ? band_solve_fused_config_th(ctx_prob(c), c->dev, o.tile_override, &c->pgrid, &c->psmem)
                        : band_solve_fused_config(ctx_prob(c), c->dev, &c->pgrid, &c->psmem, &c->pth);
        if (c->pfused && o.tile_override) c->pth = o.tile_override;
        // Single operator applications (sfista_apply, the objective, reverse
        // mode) then take the fused operator kernel as well.
        if (c->pfused && !band_op_fused_prepare(c->r, std::max(h.A.w, h.AT.w), std::max(h.B.w, h.BT.w)))
            c->pfused = 0;
        if (!c->pfused) {
            st = persistent_config(c->m, c->n, c->r, wmax, c->dev, &c->pgrid, &c->psmem, &c->prows_chunk,
                                   &c->pcols_chunk);
            if (st) return bail(st);
        }
    }
    if (c->op == SFISTA_OP_FFT) {
        st = make_fft(c);
        if (st) return bail(st);
    }
    if (c->op == SFISTA_OP_GEMM_BAND || c->op == SFISTA_OP_GEMM_DENSE) {
        st = gemm_create(&c->gemm, h, c->prec, c->op == SFISTA_OP_GEMM_DENSE, c->status, c->stream);
        if (st) return bail(st);
        // gemm_bn: every stage's N tile (256 exists for the summed stages
        // only; the stacked ones keep 128 then); 0: per stage, 64 where the
        // stage has fewer 128-column tiles than the GPU has SMs, else 128.
        for (int s4 = 0; s4 < 4; ++s4) {
            int bn = o.gemm_bn ? o.gemm_bn : gemm_default_bn(c->gemm, s4);
            if (s4 % 2 == 0 && bn == 256) bn = 128;
            gemm_set_tile(c->gemm, s4, bn, s4 % 2 == 0 ? o.gemm_resident_panels : 0);
        }
        // FP32 state for the forms whose products are far coarser than FP32
        // (BF16, BF16x3, TF32); TF32x3 keeps the double-float state, which its
        // products are accurate enough to use (1.9e-6 vs 1.7e-5 at 512^2).
        if (c->prec != SFISTA_TF32X3 &&
            ((e = cudaMalloc((void **)&c->Xf[0], N * 4)) || (e = cudaMalloc((void **)&c->Xf[1], N * 4)) ||
             (e = cudaMalloc((void **)&c->Yf, N * 4))))
            return bail(fail(SFISTA_ENOMEM, std::string("FP32 state: ") + cudaGetErrorString(e)));
    }
    if (o.lipschitz > 0.0) {
        c->L = o.lipschitz;
    } else {
        double tol = o.lipschitz_tol > 0 ? o.lipschitz_tol : 1e-10;
        int maxit = o.lipschitz_maxit > 0 ? o.lipschitz_maxit : 1000;
        st = power_lipschitz(c, tol, maxit, &c->L);
        if (st) return bail(st);
    }
    if ((e = cudaStreamSynchronize(c->stream))) return bail(fail(SFISTA_ECUDA, cudaGetErrorString(e)));
    *out = c;
    return SFISTA_OK;
}

sfista_status sfista_setup_exact(const double *psf, int psf_rows, int psf_cols, int center_row, int center_col,
                                 int img_rows, int img_cols, sfista_bc bc, const sfista_opts *opts, sfista_ctx **out) {
    TraceRange trace_("sfista_setup_exact");
    if (!out) return fail(SFISTA_EINVAL, "out is NULL");
    *out = nullptr;
    sfista_opts o;
    sfista_default_opts(&o);
    if (opts) o = *opts;
    if (o.prec != SFISTA_FP32) return fail(SFISTA_ENOTSUP, "the exact blur runs in FP32 only");
    if (o.op != SFISTA_OP_AUTO && o.op != SFISTA_OP_EXACT_FFT)
        return fail(SFISTA_EINVAL, "the exact blur has one operator form (SFISTA_OP_EXACT_FFT)");
    if (!(o.lipschitz <= 0.0 || isfinite(o.lipschitz))) return fail(SFISTA_EINVAL, "lipschitz must be finite");
    if (!(o.l1 >= 0.0) || !isfinite(o.l1)) return fail(SFISTA_EINVAL, "l1 must be finite and >= 0");
    if (!psf) return fail(SFISTA_EINVAL, "psf is NULL");
    if (psf_rows < 1 || psf_cols < 1 || img_rows < 1 || img_cols < 1 || psf_rows > img_rows || psf_cols > img_cols)
        return fail(SFISTA_EINVAL, "bad sizes (the PSF must fit in the image)");
    if (bc == SFISTA_BC_PERIODIC) return fail(SFISTA_ENOTSUP, "periodic boundary is not supported");
    if (bc != SFISTA_BC_ZERO && bc != SFISTA_BC_REFLEXIVE) return fail(SFISTA_EINVAL, "unknown boundary");
    if (center_row == -1) center_row = (psf_rows - 1) / 2;
    if (center_col == -1) center_col = (psf_cols - 1) / 2;
    if (center_row < 0 || center_row >= psf_rows || center_col < 0 || center_col >= psf_cols)
        return fail(SFISTA_EINVAL, "PSF centre outside the PSF");
    for (size_t i = 0; i < (size_t)psf_rows * psf_cols; ++i)
        if (!isfinite(psf[i])) return fail(SFISTA_EINVAL, "non-finite PSF entry");
    sfista_ctx *c = new (std::nothrow) sfista_ctx();
    if (!c) return fail(SFISTA_ENOMEM, "context allocation failed");
    c->opts = o;
    c->opts.refine_every = 0;
    c->exact = 1;
    c->m = img_rows;
    c->n = img_cols;
    c->r = 0;
    c->N = (size_t)img_rows * img_cols;
    c->prec = SFISTA_FP32;
    c->op = SFISTA_OP_EXACT_FFT;
    c->hs.m = img_rows;
    c->hs.n = img_cols;
    c->hs.p = psf_rows;
    c->hs.q = psf_cols;
    c->hs.cr = center_row;
    c->hs.cc = center_col;
    c->hs.bc = bc;
    if (o.device < 0) {
        if (cudaGetDevice(&c->dev) != cudaSuccess) {
            delete c;
            return fail(SFISTA_ECUDA, "no CUDA device");
        }
    } else {
        c->dev = o.device;
    }
    DeviceGuard g(c->dev);
    auto bail = [&](sfista_status s) {
        ctx_free(c);
        return s;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)))
        return bail(fail(SFISTA_ECUDA, std::string("stream/event: ") + cudaGetErrorString(e)));
    const size_t N = c->N;
    if ((e = cudaMalloc((void **)&c->Bd, N * 4)) || (e = cudaMalloc((void **)&c->Yop, N * 4)) ||
        (e = cudaMalloc((void **)&c->R, N * 4)) || (e = cudaMalloc((void **)&c->tmp, N * 4)) ||
        (e = cudaMalloc((void **)&c->Xb[0], N * 8)) || (e = cudaMalloc((void **)&c->Xb[1], N * 8)) ||
        (e = cudaMalloc((void **)&c->Y, N * 8)) || (e = cudaMalloc((void **)&c->status, 16)))
        return bail(fail(SFISTA_ENOMEM, std::string("state buffers: ") + cudaGetErrorString(e)));
    if ((e = cudaMemset(c->status, 0, 16))) return bail(fail(SFISTA_ECUDA, cudaGetErrorString(e)));
    sfista_status st = fftconv_create(&c->fft, psf, psf_rows, psf_cols, center_row, center_col, img_rows, img_cols, bc);
    if (st) return bail(st);
    if (o.lipschitz > 0.0) {
        c->L = o.lipschitz;
    } else {
        const double tol = o.lipschitz_tol > 0 ? o.lipschitz_tol : 1e-10;
        const int maxit = o.lipschitz_maxit > 0 ? o.lipschitz_maxit : 1000;
        st = power_lipschitz_fft(c, tol, maxit, &c->L);
        if (st) return bail(st);
    }
    if ((e = cudaStreamSynchronize(c->stream))) return bail(fail(SFISTA_ECUDA, cudaGetErrorString(e)));
    *out = c;
    return SFISTA_OK;
}

void sfista_destroy(sfista_ctx *ctx) { ctx_free(ctx); }

sfista_status sfista_set_factors(sfista_ctx *c, const double *A, const double *B) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!is_banded(c->op) || c->exact)
        return fail(SFISTA_ENOTSUP, "factors can be replaced in the banded FP32 forms only");
    DeviceGuard g(c->dev);
    HostSetup &h = c->hs;
    Band nA, nAT, nB, nBT;
    if (A && !(band_from_dense(A, h.A, false, &nA) && band_from_dense(A, h.AT, true, &nAT)))
        return fail(SFISTA_EINVAL, "A has a nonzero entry outside the band of the context's right factors");
    if (B && !(band_from_dense(B, h.B, false, &nB) && band_from_dense(B, h.BT, true, &nBT)))
        return fail(SFISTA_EINVAL, "B has a nonzero entry outside the band of the context's left factors");
    SF_CUDA(cudaStreamSynchronize(c->stream));
    cudaError_t e = cudaSuccess;
    if (A) {
        h.A = nA;
        h.AT = nAT;
        if ((e = store_band(c, h.A, c->dA, c->fA, &c->interior[0])) ||
            (e = store_band(c, h.AT, c->dAT, c->fAT, &c->interior[1])))
            return fail(SFISTA_ECUDA, std::string("factor upload: ") + cudaGetErrorString(e));
    }
    if (B) {
        h.B = nB;
        h.BT = nBT;
        if ((e = store_band(c, h.B, c->dB, c->fB, &c->interior[2])) ||
            (e = store_band(c, h.BT, c->dBT, c->fBT, &c->interior[3])))
            return fail(SFISTA_ECUDA, std::string("factor upload: ") + cudaGetErrorString(e));
    }
    if (A || B) c->custom_factors = 1;
    if (c->gexec) {   // the captured loop holds the old interior ranges
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->g_k0 = c->g_iters = -1;
    }
    return SFISTA_OK;
}

sfista_status sfista_factorize(const double *psf, int p, int q, int cr, int cc, int m, int n, sfista_bc bc, int r,
                               double *sigma, double *C, double *D, double *approx_err) {
    if (cr == -1 && p > 0) cr = (p - 1) / 2;
    if (cc == -1 && q > 0) cc = (q - 1) / 2;
    HostSetup h;
    sfista_status st = host_setup(psf, p, q, cr, cc, m, n, bc, r, &h);
    if (st) return st;
    if (sigma) std::copy(h.sigma.begin(), h.sigma.end(), sigma);
    if (C) std::copy(h.C.begin(), h.C.end(), C);
    if (D) std::copy(h.D.begin(), h.D.end(), D);
    if (approx_err) *approx_err = h.approx_err;
    return SFISTA_OK;
}

sfista_status sfista_factor_bands(const double *psf, int p, int q, int cr, int cc, int m, int n, sfista_bc bc, int r,
                                  int which, int *lo, int *w, double *band, int *interior) {
    if (which < 0 || which > 3) return fail(SFISTA_EINVAL, "which must be 0 (A), 1 (A^T), 2 (B) or 3 (B^T)");
    if (!lo || !w) return fail(SFISTA_EINVAL, "lo or w is NULL");
    if (cr == -1 && p > 0) cr = (p - 1) / 2;
    if (cc == -1 && q > 0) cc = (q - 1) / 2;
    HostSetup h;
    sfista_status st = host_setup(psf, p, q, cr, cc, m, n, bc, r, &h);
    if (st) return st;
    const Band &F = which == 0 ? h.A : which == 1 ? h.AT : which == 2 ? h.B : h.BT;
    *lo = F.lo;
    *w = F.w;
    if (band) std::copy(F.band.begin(), F.band.end(), band);
    if (interior) {
        std::vector<float> f(F.band.begin(), F.band.end());
        band_interior(f.data(), F.len, F.r * F.w, &interior[0], &interior[1]);
    }
    return SFISTA_OK;
}

sfista_status sfista_solve_device(sfista_ctx *c, const float *d_b, double lambda, int iters, float *d_x,
                                  void *stream) {
    TraceRange trace_("sfista_solve_device");
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!d_x) return fail(SFISTA_EINVAL, "x is NULL");
    DeviceGuard g(c->dev);
    cudaStream_t user = (cudaStream_t)stream;
    st = solve_core(c, d_b, lambda, 0, iters, nullptr, nullptr, user);
    if (st) return st;
    launch_df_to_f32(c->Xb[iters & 1], d_x, c->N, c->stream);
    SF_CUDA(cudaGetLastError());
    return finish_on_user(c, user);
}

sfista_status sfista_solve_state(sfista_ctx *c, const float *d_b, double lambda, int k0, int iters,
                                 double *d_X, double *d_Xprev, void *stream) {
    TraceRange trace_("sfista_solve_state");
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!d_X || !d_Xprev) return fail(SFISTA_EINVAL, "state buffers are NULL");
    DeviceGuard g(c->dev);
    cudaStream_t user = (cudaStream_t)stream;
    st = solve_core(c, d_b, lambda, k0, iters, d_X, d_Xprev, user);
    if (st) return st;
    int ke = k0 + iters;
    launch_df_to_f64(c->Xb[ke & 1], d_X, c->N, c->stream);
    launch_df_to_f64(c->Xb[(ke + 1) & 1], d_Xprev, c->N, c->stream);
    return finish_on_user(c, user);
}

sfista_status sfista_sync(sfista_ctx *c, void *stream) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    DeviceGuard g(c->dev);
    SF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return drain_status(c);
}

sfista_status sfista_solve(sfista_ctx *c, const float *b, double lambda, int iters, float *x) {
    TraceRange trace_("sfista_solve");
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!b || !x) return fail(SFISTA_EINVAL, "b or x is NULL");
    DeviceGuard g(c->dev);
    for (size_t i = 0; i < c->N; ++i)
        if (!isfinite(b[i])) return fail(SFISTA_EINVAL, "b has a non-finite entry");
    SF_CUDA(cudaMemcpyAsync(c->tmp, b, c->N * 4, cudaMemcpyHostToDevice, c->stream));
    st = solve_core(c, c->tmp, lambda, 0, iters, nullptr, nullptr, c->stream);
    if (st) return st;
    launch_df_to_f32(c->Xb[iters & 1], c->tmp, c->N, c->stream);
    SF_CUDA(cudaMemcpyAsync(x, c->tmp, c->N * 4, cudaMemcpyDeviceToHost, c->stream));
    return drain_status(c);
}

sfista_status sfista_apply(sfista_ctx *c, const float *d_x, float *d_y, int transpose, void *stream) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!d_x || !d_y) return fail(SFISTA_EINVAL, "x or y is NULL");
    DeviceGuard g(c->dev);
    cudaStream_t user = (cudaStream_t)stream;
    SF_CUDA(cudaEventRecord(c->ev_in, user));
    SF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    const HostSetup &h = c->hs;
    ProxArgs pa{};
    if (is_fft(c->op)) {
        fftconv_apply(c->fft, transpose != 0, d_x, EPI_STORE, d_y, pa, c->stream);
    } else if (fused_apply(c)) {
        const Band &F = transpose ? h.AT : h.A;
        const Band &G = transpose ? h.BT : h.B;
        launch_band_op_fused(d_x, c->m, c->n, c->r, transpose ? c->fAT : c->fA, F.lo, F.w, transpose ? c->fBT : c->fB,
                             G.lo, G.w, EPI_STORE, d_y, pa, transpose ? interior_adj(c) : interior_fwd(c), c->stream);
    } else if (is_banded(c->op)) {
        const Band &F = transpose ? h.AT : h.A;
        const Band &G = transpose ? h.BT : h.B;
        launch_band_rows<float>(d_x, c->m, c->n, transpose ? c->fAT : c->fA, F.lo, F.w, c->r, c->Z, c->stream);
        launch_band_cols<float>(c->Z, c->m, c->n, transpose ? c->fBT : c->fB, G.lo, G.w, c->r, EPI_STORE, d_y,
                                pa, c->stream);
    } else {
        st = gemm_apply(c->gemm, d_x, d_y, transpose, c->stream);
        if (st) return st;
    }
    SF_CUDA(cudaGetLastError());
    return finish_on_user(c, user);
}

sfista_status sfista_objective(sfista_ctx *c, const float *d_b, const float *d_x, double lambda, double *phi,
                               void *stream) {
    TraceRange trace_("sfista_objective");
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!d_b || !d_x || !phi) return fail(SFISTA_EINVAL, "NULL argument");
    if (!(lambda >= 0) || !isfinite(lambda)) return fail(SFISTA_EINVAL, "lambda must be finite and >= 0");
    DeviceGuard g(c->dev);
    cudaStream_t user = (cudaStream_t)stream;
    SF_CUDA(cudaEventRecord(c->ev_in, user));
    SF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
    // A_s x into the scratch image, then the two sums of squares in FP64.
    const HostSetup &h = c->hs;
    ProxArgs pa{};
    if (is_fft(c->op)) {
        fftconv_apply(c->fft, false, d_x, EPI_STORE, c->tmp, pa, c->stream);
    } else if (fused_apply(c)) {
        launch_band_op_fused(d_x, c->m, c->n, c->r, c->fA, h.A.lo, h.A.w, c->fB, h.B.lo, h.B.w, EPI_STORE, c->tmp, pa,
                             interior_fwd(c), c->stream);
    } else if (is_banded(c->op)) {
        launch_band_rows<float>(d_x, c->m, c->n, c->fA, h.A.lo, h.A.w, c->r, c->Z, c->stream);
        launch_band_cols<float>(c->Z, c->m, c->n, c->fB, h.B.lo, h.B.w, c->r, EPI_STORE, c->tmp, pa, c->stream);
    } else {
        st = gemm_apply(c->gemm, d_x, c->tmp, 0, c->stream);
        if (st) return st;
    }
    const int nblk = 256;
    double *scratch = nullptr;
    SF_CUDA(cudaMallocAsync((void **)&scratch, (nblk + 2) * sizeof(double), c->stream));
    launch_sumsq(c->tmp, d_b, c->N, scratch, nblk, scratch + nblk, c->stream);
    launch_sumsq(d_x, nullptr, c->N, scratch, nblk, scratch + nblk + 1, c->stream);
    double sums[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(sums, scratch + nblk, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(scratch, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (!e) e = cudaGetLastError();
    if (e) return fail(SFISTA_ECUDA, std::string("objective: ") + cudaGetErrorString(e));
    *phi = 0.5 * sums[0] + 0.5 * lambda * lambda * sums[1];
    return finish_on_user(c, user);
}

sfista_status sfista_info(const sfista_ctx *c, double *lipschitz, double *sigma, double *approx_err,
                          int *config) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (lipschitz) *lipschitz = c->L;
    if (sigma) std::copy(c->hs.sigma.begin(), c->hs.sigma.end(), sigma);
    if (approx_err) *approx_err = c->hs.approx_err;
    if (config) {
        config[0] = c->prec;
        config[1] = c->op;
        config[2] = c->hs.A.w;
        config[3] = c->hs.B.w;
        config[4] = c->hs.A.lo;
        config[5] = c->hs.B.lo;
        config[6] = c->hs.AT.lo;
        config[7] = c->hs.BT.lo;
    }
    return SFISTA_OK;
}

sfista_status sfista_get_profiles(const sfista_ctx *c, double *C, double *D) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (c->exact) return fail(SFISTA_ENOTSUP, "the exact-blur context has no Kronecker factors");
    if (c->custom_factors) return fail(SFISTA_ENOTSUP, "the factors were replaced: no profiles describe them");
    if (C) std::copy(c->hs.C.begin(), c->hs.C.end(), C);
    if (D) std::copy(c->hs.D.begin(), c->hs.D.end(), D);
    return SFISTA_OK;
}

sfista_status sfista_get_factors(const sfista_ctx *c, double *A, double *B) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (c->exact) return fail(SFISTA_ENOTSUP, "the exact-blur context has no Kronecker factors");
    auto dense = [](const Band &b, double *out) {
        size_t len = b.len;
        std::fill(out, out + (size_t)b.r * len * len, 0.0);
        for (int i = 0; i < b.r; ++i)
            for (int k = 0; k < b.w; ++k)
                for (size_t row = 0; row < len; ++row) {
                    long col = (long)row + b.lo + k;
                    if (col >= 0 && col < (long)len)
                        out[((size_t)i * len + row) * len + col] = b.band[((size_t)i * b.w + k) * len + row];
                }
    };
    if (A) dense(c->hs.A, A);
    if (B) dense(c->hs.B, B);
    return SFISTA_OK;
}

sfista_status sfista_blur(const double *psf, int p, int q, int cr, int cc, sfista_bc bc, const float *d_x, int m,
                          int n, float *d_y, void *stream) {
    if (!psf || !d_x || !d_y) return fail(SFISTA_EINVAL, "NULL pointer");
    if (p < 1 || q < 1 || m < 1 || n < 1 || p > m || q > n) return fail(SFISTA_EINVAL, "bad sizes");
    if (bc == SFISTA_BC_PERIODIC) return fail(SFISTA_ENOTSUP, "periodic boundary is not supported");
    if (bc != SFISTA_BC_ZERO && bc != SFISTA_BC_REFLEXIVE) return fail(SFISTA_EINVAL, "unknown boundary");
    if (cr == -1) cr = (p - 1) / 2;
    if (cc == -1) cc = (q - 1) / 2;
    if (cr < 0 || cr >= p || cc < 0 || cc >= q) return fail(SFISTA_EINVAL, "PSF centre outside the PSF");
    std::vector<float> pf((size_t)p * q);
    for (size_t i = 0; i < pf.size(); ++i) {
        if (!isfinite(psf[i])) return fail(SFISTA_EINVAL, "PSF has a non-finite entry");
        pf[i] = (float)psf[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    float *dP = nullptr;
    SF_CUDA(cudaMalloc((void **)&dP, pf.size() * 4));
    cudaError_t e = cudaMemcpyAsync(dP, pf.data(), pf.size() * 4, cudaMemcpyHostToDevice, s);
    if (!e) {
        launch_blur_exact(d_x, m, n, dP, p, q, cr, cc, bc, d_y, s);
        e = cudaGetLastError();
    }
    if (!e) e = cudaStreamSynchronize(s);
    cudaFree(dP);
    if (e) return fail(SFISTA_ECUDA, std::string("blur: ") + cudaGetErrorString(e));
    return SFISTA_OK;
}


sfista_status sfista_batch_create(sfista_ctx *const *ctxs, int nprob, sfista_batch **out) {
    if (!out) return fail(SFISTA_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || nprob < 1) return fail(SFISTA_EINVAL, "no problems");
    for (int p = 0; p < nprob; ++p) {
        if (!ctxs[p]) return fail(SFISTA_EINVAL, "a context is NULL");
        if (is_fft(ctxs[p]->op)) return fail(SFISTA_ENOTSUP, "batches take banded or tensor-core contexts only");
    }
    const bool gemm = ctxs[0]->op == SFISTA_OP_GEMM_BAND || ctxs[0]->op == SFISTA_OP_GEMM_DENSE;
    for (int p = 0; p < nprob; ++p) {
        const bool gp = ctxs[p]->op == SFISTA_OP_GEMM_BAND || ctxs[p]->op == SFISTA_OP_GEMM_DENSE;
        if (gp != gemm || ctxs[p]->prec != ctxs[0]->prec || ctxs[p]->dev != ctxs[0]->dev)
            return fail(SFISTA_EINVAL, "batched problems need one device, one precision and one operator family");
        for (int q = 0; q < p; ++q)
            if (ctxs[q] == ctxs[p]) return fail(SFISTA_EINVAL, "a context appears twice in the batch");
        if (gp && ctxs[p]->opts.refine_every > 0)
            return fail(SFISTA_ENOTSUP, "residual refinement is not available in batched solves");
    }
    sfista_batch *b = new (std::nothrow) sfista_batch();
    if (!b) return fail(SFISTA_ENOMEM, "batch allocation failed");
    b->ctxs.assign(ctxs, ctxs + nprob);
    b->dev = ctxs[0]->dev;
    b->gemm = gemm;
    DeviceGuard g(b->dev);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming))) {
        batch_free(b);
        return fail(SFISTA_ECUDA, std::string("batch stream: ") + cudaGetErrorString(e));
    }
    if (gemm) {
        std::vector<GemmPath *> paths(nprob);
        for (int p = 0; p < nprob; ++p) paths[p] = ctxs[p]->gemm;
        sfista_status st = gemm_batch_create(&b->gb, paths.data(), nprob, b->stream);
        if (st) {
            batch_free(b);
            return st;
        }
    } else {
        b->h_probs.resize(nprob);
        for (int p = 0; p < nprob; ++p) b->h_probs[p] = ctx_prob(ctxs[p]);
        if ((e = cudaMalloc((void **)&b->d_probs, nprob * sizeof(BandProb)))) {
            batch_free(b);
            return fail(SFISTA_ENOMEM, std::string("grouped banded tables: ") + cudaGetErrorString(e));
        }
        sfista_status st = band_batch_plan(b, 0);
        if (st) {
            batch_free(b);
            return st;
        }
        std::vector<int2> items;
        int th = 32;
        if (band_solve_fused_batch_config(b->h_probs.data(), nprob, b->dev, &items, &b->fsmem, &th)) {
            for (BandProb &P : b->h_probs) P.th = th;
            if ((e = cudaMalloc((void **)&b->d_fitems, items.size() * sizeof(int2))) ||
                (e = cudaMemcpy(b->d_fitems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice)) ||
                (e = cudaMalloc((void **)&b->bar, kBarrierBytes))) {
                batch_free(b);
                return fail(SFISTA_ENOMEM, std::string("one-launch batch tables: ") + cudaGetErrorString(e));
            }
            b->fnitems = (int)items.size();
            b->fused_ok = b->use_fused = true;
        }
    }
    *out = b;
    return SFISTA_OK;
}

void sfista_batch_destroy(sfista_batch *b) { batch_free(b); }

sfista_status sfista_batch_solve(sfista_batch *b, const float *const *d_b, const double *lambdas, int iters,
                                 float *const *d_x, void *stream) {
    TraceRange trace_("sfista_batch_solve");
    if (!b) return fail(SFISTA_EINVAL, "batch is NULL");
    if (!d_b || !lambdas || !d_x) return fail(SFISTA_EINVAL, "NULL argument array");
    if (iters < 0) return fail(SFISTA_EINVAL, "iters must be >= 0");
    const int np = (int)b->ctxs.size();
    for (int p = 0; p < np; ++p) {
        if (!d_b[p] || !d_x[p]) return fail(SFISTA_EINVAL, "NULL observation or output pointer");
        if (!(lambdas[p] >= 0) || !isfinite(lambdas[p])) return fail(SFISTA_EINVAL, "lambda must be finite and >= 0");
    }
    DeviceGuard g(b->dev);
    cudaStream_t user = (cudaStream_t)stream;
    for (int p = 0; p < np; ++p) {
        sfista_ctx *c = b->ctxs[p];
        sfista_status st = ensure_beta(c, iters + 1);
        if (st) return st;
    }
    SF_CUDA(cudaEventRecord(b->ev_in, user));
    SF_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    if (b->use_fused) {
        // One launch: the solver starts from X_0 = 0 itself, reads each B in
        // place (checking it for non-finite values) and writes each X_iters.
        for (int p = 0; p < np; ++p) {
            sfista_ctx *c = b->ctxs[p];
            ProxArgs pa = prox_args(c, 1, lambdas[p]);
            pa.Bd = d_b[p];
            pa.Xin = c->Xb[0];
            pa.Xout = c->Xb[1];
            b->h_probs[p].pa = pa;
            b->h_probs[p].xout = d_x[p];
        }
        // Repeated solves on the same buffers and weights reuse the table
        // already on the device (copies are stream-ordered after the solves
        // that read it).
        if (b->sent.size() != b->h_probs.size() ||
            memcmp(b->sent.data(), b->h_probs.data(), np * sizeof(BandProb))) {
            b->sent.clear();
            SF_CUDA(cudaMemcpyAsync(b->d_probs, b->h_probs.data(), np * sizeof(BandProb), cudaMemcpyHostToDevice,
                                    b->stream));
            SF_CUDA(cudaStreamSynchronize(b->stream));   // host staging array is reused on the next solve
            b->sent = b->h_probs;
        }
        if (iters > 0) {
            SF_CUDA(launch_band_solve_fused_batch(b->fnitems, b->fsmem, b->d_probs, b->d_fitems, iters, b->bar,
                                                  b->stream));
        } else {
            for (int p = 0; p < np; ++p) {
                sfista_ctx *c = b->ctxs[p];
                launch_check_finite(d_b[p], c->N, c->status, b->stream);
                SF_CUDA(cudaMemsetAsync(d_x[p], 0, c->N * sizeof(float), b->stream));
            }
        }
        SF_CUDA(cudaGetLastError());
        SF_CUDA(cudaEventRecord(b->ev_out, b->stream));
        SF_CUDA(cudaStreamWaitEvent(user, b->ev_out, 0));
        return SFISTA_OK;
    }
    std::vector<ProxArgs> pas(np);
    std::vector<const float *> bds(np);
    for (int p = 0; p < np; ++p) {
        sfista_ctx *c = b->ctxs[p];
        SF_CUDA(cudaMemcpyAsync(c->Bd, d_b[p], c->N * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
        launch_check_finite(c->Bd, c->N, c->status, b->stream);
        SF_CUDA(cudaMemsetAsync(c->Xb[0], 0, c->N * 8, b->stream));
        SF_CUDA(cudaMemsetAsync(c->Xb[1], 0, c->N * 8, b->stream));
        void *yhi = nullptr, *ylo = nullptr;
        int split = 0;
        if (c->gemm) gemm_state_operands(c->gemm, &yhi, &ylo, &split);
        launch_init_state(c->Xb[0], c->Xb[1], c->Y, c->Yop, yhi, ylo, split, c->N, 0.0, b->stream);
        if (c->Xf[0]) {   // X_0 = X_{-1} = Y_1 = 0 in the FP32 state too
            SF_CUDA(cudaMemsetAsync(c->Xf[0], 0, c->N * 4, b->stream));
            SF_CUDA(cudaMemsetAsync(c->Xf[1], 0, c->N * 4, b->stream));
            SF_CUDA(cudaMemsetAsync(c->Yf, 0, c->N * 4, b->stream));
        }
        ProxArgs pa = prox_args(c, 1, lambdas[p]);
        pa.Xin = c->Xb[0];
        pa.Xout = c->Xb[1];
        pas[p] = pa;
        bds[p] = c->Bd;
    }
    if (b->gemm) {
        sfista_status st = gemm_batch_bind(b->gb, bds.data(), pas.data(), b->stream);
        if (st) return st;
    } else {
        for (int p = 0; p < np; ++p) b->h_probs[p].pa = pas[p];
        b->sent.clear();
        SF_CUDA(cudaMemcpyAsync(b->d_probs, b->h_probs.data(), np * sizeof(BandProb), cudaMemcpyHostToDevice,
                                b->stream));
        SF_CUDA(cudaStreamSynchronize(b->stream));   // host staging array is reused on the next solve
    }
    if (iters > 0) {
        std::vector<double> lams(lambdas, lambdas + np);
        if (!(b->gexec && b->g_iters == iters && b->g_lams == lams)) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            SF_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            for (int k = 1; k <= iters; ++k)
                for (int st = 0; st < 4; ++st) batch_stage(b, st, k);
            cudaError_t le = cudaGetLastError();
            cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
            if (le || ee) {
                if (graph) cudaGraphDestroy(graph);
                return fail(SFISTA_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(le ? le : ee));
            }
            cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie) {
                b->gexec = nullptr;
                return fail(SFISTA_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(ie));
            }
            b->g_iters = iters;
            b->g_lams = lams;
        }
        SF_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    }
    for (int p = 0; p < np; ++p) {
        sfista_ctx *c = b->ctxs[p];
        if (c->Xf[0])
            SF_CUDA(cudaMemcpyAsync(d_x[p], c->Xf[iters & 1], c->N * 4, cudaMemcpyDeviceToDevice, b->stream));
        else
            launch_df_to_f32(c->Xb[iters & 1], d_x[p], c->N, b->stream);
    }
    SF_CUDA(cudaGetLastError());
    SF_CUDA(cudaEventRecord(b->ev_out, b->stream));
    SF_CUDA(cudaStreamWaitEvent(user, b->ev_out, 0));
    return SFISTA_OK;
}

sfista_status sfista_batch_sync(sfista_batch *b, void *stream) {
    if (!b) return fail(SFISTA_EINVAL, "batch is NULL");
    DeviceGuard g(b->dev);
    SF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    SF_CUDA(cudaStreamSynchronize(b->stream));
    sfista_status worst = SFISTA_OK;
    for (sfista_ctx *c : b->ctxs) {
        sfista_status st = drain_status(c);
        if (st && !worst) worst = st;
    }
    return worst;
}

sfista_status sfista_batch_tune(sfista_batch *b, int iters, sfista_tune_entry *entries, int max_entries,
                                int *n_entries) {
    TraceRange trace_("sfista_batch_tune");
    if (!b) return fail(SFISTA_EINVAL, "batch is NULL");
    if (n_entries) *n_entries = 0;
    if (iters < 1 || max_entries < 0) return fail(SFISTA_EINVAL, "iters must be >= 1 and max_entries >= 0");
    if (b->gemm && !gemm_batch_res_ok(b->gb)) return SFISTA_OK;   // one tile shape: nothing to choose
    DeviceGuard g(b->dev);
    const int np = (int)b->ctxs.size();
    std::vector<const float *> d_b(np);
    std::vector<float *> d_x(np);
    std::vector<double> lams(np, 0.0);
    for (int p = 0; p < np; ++p) {   // all-zero observations; the scratch image doubles as output
        sfista_ctx *c = b->ctxs[p];
        SF_CUDA(cudaMemsetAsync(c->tmp, 0, c->N * sizeof(float), b->stream));
        d_b[p] = c->tmp;
        d_x[p] = c->tmp;
    }
    cudaEvent_t e0, e1;
    SF_CUDA(cudaEventCreate(&e0));
    SF_CUDA(cudaEventCreate(&e1));
    if (b->gemm) {
        // Grouped tensor-core stages 0 and 2 with and without resident P
        // panels (entries: stage -1, chunk 1 = resident, 0 = streamed): the
        // first batch solve of each plan captures its graph, the second is
        // timed.
        int count = 0;
        float t[2] = {0.f, 0.f};
        sfista_status st = SFISTA_OK;
        for (int res = 1; res >= 0 && !st; --res) {
            gemm_batch_set_res(b->gb, res != 0);
            if (b->gexec) {   // captured with the other tile shape
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            if ((st = sfista_batch_solve(b, d_b.data(), lams.data(), iters, d_x.data(), b->stream))) break;
            cudaError_t e = cudaEventRecord(e0, b->stream);
            if (!e && !(st = sfista_batch_solve(b, d_b.data(), lams.data(), iters, d_x.data(), b->stream)))
                e = cudaEventRecord(e1, b->stream);
            if (st) break;
            if (!e) e = cudaEventSynchronize(e1);
            if (!e) e = cudaEventElapsedTime(&t[res], e0, e1);
            if (e) {
                st = fail(SFISTA_ECUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
                break;
            }
            t[res] /= iters;
            if (entries && count < max_entries) entries[count] = sfista_tune_entry{b->ctxs[0]->op, -1, res, t[res]};
            ++count;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st) return st;
        gemm_batch_set_res(b->gb, t[1] <= t[0]);
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        if (n_entries) *n_entries = count;
        return sfista_batch_sync(b, nullptr);
    }
    const size_t kb = 1024;
    const size_t budgets[] = {0, 24 * kb, 32 * kb, 48 * kb, 64 * kb, 80 * kb, 96 * kb, 128 * kb, 160 * kb, 227 * kb};
    std::vector<std::vector<int>> seen;
    int count = 0;
    float best = -1.f;
    size_t best_budget = 0;
    bool best_fused = false;
    sfista_status st = SFISTA_OK;
    if (b->fused_ok) {   // the one-launch solve of the whole batch
        b->use_fused = true;
        float ms = 0.f;
        cudaError_t e = cudaSuccess;
        if (!(st = sfista_batch_solve(b, d_b.data(), lams.data(), 2, d_x.data(), b->stream))) {
            e = cudaEventRecord(e0, b->stream);
            if (!e && !(st = sfista_batch_solve(b, d_b.data(), lams.data(), iters, d_x.data(), b->stream)))
                e = cudaEventRecord(e1, b->stream);
            if (!st && !e) e = cudaEventSynchronize(e1);
            if (!st && !e) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (!st && e) st = fail(SFISTA_ECUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
        if (!st) {
            ms /= iters;
            if (entries && count < max_entries) entries[count] = sfista_tune_entry{SFISTA_OP_BANDED_PERSISTENT, -1, 0, ms};
            ++count;
            best = ms;
            best_fused = true;
        }
        b->use_fused = false;
    }
    for (size_t bud : budgets) {
        if (st) break;
        if ((st = band_batch_plan(b, bud))) break;
        std::vector<int> sig;
        for (const BandProb &P : b->h_probs) sig.push_back(P.rows_chunk), sig.push_back(P.cols_chunk);
        if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
        seen.push_back(sig);
        // The first solve captures the graph of this plan; the second is timed.
        if ((st = sfista_batch_solve(b, d_b.data(), lams.data(), iters, d_x.data(), b->stream))) break;
        cudaError_t e = cudaEventRecord(e0, b->stream);
        if (!e && !(st = sfista_batch_solve(b, d_b.data(), lams.data(), iters, d_x.data(), b->stream)))
            e = cudaEventRecord(e1, b->stream);
        if (st) break;
        float ms = 0.f;
        if (!e) e = cudaEventSynchronize(e1);
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e) {
            st = fail(SFISTA_ECUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
            break;
        }
        ms /= iters;
        if (entries && count < max_entries) entries[count] = sfista_tune_entry{SFISTA_OP_BANDED, -1, (int)(bud / kb), ms};
        ++count;
        if (best < 0.f || ms < best) best = ms, best_budget = bud, best_fused = false;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    b->use_fused = best_fused;
    if (!best_fused && (st = band_batch_plan(b, best_budget))) return st;
    if (n_entries) *n_entries = count;
    return sfista_batch_sync(b, nullptr);
}

sfista_status sfista_solve_batched(sfista_ctx *const *ctxs, const float *const *d_b, const double *lambdas,
                                   int nprob, int iters, float *const *d_x, void *stream) {
    sfista_batch *b = nullptr;
    sfista_status st = sfista_batch_create(ctxs, nprob, &b);
    if (st) return st;
    st = sfista_batch_solve(b, d_b, lambdas, iters, d_x, stream);
    if (!st) st = sfista_batch_sync(b, stream);
    batch_free(b);
    return st;
}

sfista_status sfista_time_stages(sfista_ctx *c, const float *d_b, double lambda, int reps, float *ms) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (!ms || reps < 1) return fail(SFISTA_EINVAL, "ms is NULL or reps < 1");
    DeviceGuard g(c->dev);
    st = ensure_beta(c, reps + 1);
    if (st) return st;
    st = solve_core(c, d_b, lambda, 0, 0, nullptr, nullptr, c->stream);
    if (st) return st;
    cudaEvent_t ev[5];
    for (int i = 0; i < 5; ++i) SF_CUDA(cudaEventCreate(&ev[i]));
    double acc[4] = {0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    if (c->op == SFISTA_OP_BANDED_PERSISTENT) {
        // One persistent launch covers all four stages: report its mean time
        // per iteration in slot 0.
        e = cudaEventRecord(ev[0], c->stream);
        if (!e) {
            sfista_status rs = run_loop(c, lambda, 0, reps);
            if (rs) {
                for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
                return rs;
            }
            e = cudaEventRecord(ev[1], c->stream);
        }
        if (!e) e = cudaEventSynchronize(ev[1]);
        float t = 0;
        if (!e) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
        if (e) return fail(SFISTA_ECUDA, std::string("stage timing: ") + cudaGetErrorString(e));
        ms[0] = t / reps;
        ms[1] = ms[2] = ms[3] = 0.0f;
        return drain_status(c);
    }
    for (int k = 1; k <= reps && !e; ++k) {
        ProxArgs pa = prox_args(c, k, lambda);
        e = cudaEventRecord(ev[0], c->stream);
        for (int s4 = 0; s4 < 4 && !e; ++s4) {
            enqueue_stage(c, s4, pa);
            e = cudaEventRecord(ev[s4 + 1], c->stream);
        }
        if (!e) e = cudaEventSynchronize(ev[4]);
        for (int s4 = 0; s4 < 4 && !e; ++s4) {
            float t = 0;
            e = cudaEventElapsedTime(&t, ev[s4], ev[s4 + 1]);
            acc[s4] += t;
        }
    }
    for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
    if (e) return fail(SFISTA_ECUDA, std::string("stage timing: ") + cudaGetErrorString(e));
    for (int s4 = 0; s4 < 4; ++s4) ms[s4] = (float)(acc[s4] / reps);
    return drain_status(c);
}

namespace {

// Mean time (ms) of stages [s0, s1] of Alg. 2, repeated `reps` times after two
// untimed repetitions, launched back to back on the context's stream.
sfista_status time_stage_range(sfista_ctx *c, int s0, int s1, int reps, float *ms) {
    cudaEvent_t e0, e1;
    SF_CUDA(cudaEventCreate(&e0));
    SF_CUDA(cudaEventCreate(&e1));
    cudaError_t e = cudaSuccess;
    for (int k = 1; k <= reps + 2 && !e; ++k) {
        if (k == 3) e = cudaEventRecord(e0, c->stream);
        const ProxArgs pa = prox_args(c, k, 0.0);
        for (int st = s0; st <= s1; ++st) enqueue_stage(c, st, pa);
    }
    if (!e) e = cudaEventRecord(e1, c->stream);
    if (!e) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (!e) e = cudaEventElapsedTime(&t, e0, e1);
    if (!e) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return fail(SFISTA_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
    *ms = t / reps;
    return SFISTA_OK;
}

// Mean time per iteration of the iteration loop exactly as a solve runs it
// (run_loop: a CUDA graph of `iters` iterations when the context uses graphs,
// or the one-launch solver), over `iters` iterations after one untimed run
// of the same loop.  Forms with several launches per iteration are timed
// with the launch cost a solve has, not with that of separate launches.
sfista_status time_loop(sfista_ctx *c, int iters, float *ms) {
    if (c->gexec) {   // a graph captured for another configuration
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->g_k0 = c->g_iters = -1;
    }
    cudaEvent_t e0, e1;
    SF_CUDA(cudaEventCreate(&e0));
    SF_CUDA(cudaEventCreate(&e1));
    sfista_status st = run_loop(c, 0.0, 0, iters);
    cudaError_t e = cudaSuccess;
    if (!st) e = cudaEventRecord(e0, c->stream);
    if (!st && !e) st = run_loop(c, 0.0, 0, iters);
    if (!st && !e) e = cudaEventRecord(e1, c->stream);
    if (!st && !e) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (!st && !e) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (e) return fail(SFISTA_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
    *ms = t / iters;
    return SFISTA_OK;
}

}  // namespace

sfista_status sfista_tune(sfista_ctx *c, int iters, sfista_tune_entry *entries, int max_entries, int *n_entries) {
    TraceRange trace_("sfista_tune");
    sfista_status st = check_ctx(c);
    if (st) return st;
    if (c->exact) return fail(SFISTA_ENOTSUP, "the exact-blur context has a single operator form");
    if (n_entries) *n_entries = 0;
    if (iters < 1 || max_entries < 0) return fail(SFISTA_EINVAL, "iters must be >= 1 and max_entries >= 0");
    DeviceGuard g(c->dev);
    st = ensure_beta(c, std::max(iters, 40) + 3);   // the longest timed loop (one-launch solver: >= 40 its)
    if (st) return st;
    // All-zero observation and state (c->tmp is scratch).
    SF_CUDA(cudaMemsetAsync(c->tmp, 0, c->N * sizeof(float), c->stream));
    st = solve_core(c, c->tmp, 0.0, 0, 0, nullptr, nullptr, c->stream);
    if (st) return st;
    int count = 0;
    auto log = [&](int op, int stage, int chunk, float ms) {
        if (entries && count < max_entries) entries[count] = sfista_tune_entry{op, stage, chunk, ms};
        ++count;
    };
    const HostSetup &h = c->hs;
    const bool auto_op = c->opts.op == SFISTA_OP_AUTO;
    if (c->prec == SFISTA_FP32 && (auto_op || c->op != SFISTA_OP_BANDED_PERSISTENT)) {
        const int chosen = c->op;
        if (c->op == SFISTA_OP_BANDED || auto_op) {
            // Two-pass form: the term chunk of each stage, timed alone.
            c->op = SFISTA_OP_BANDED;
            const int widths[4] = {h.A.w, h.B.w, h.AT.w, h.BT.w};
            for (int s4 = 0; s4 < 4; ++s4) {
                const bool rows = s4 % 2 == 0;
                const int lim = rows ? band_rows_chunk_limit(c->r, widths[s4]) : band_cols_chunk_limit(c->r, widths[s4]);
                float best = 0.f;
                int best_ch = 0;
                for (int ch = 1; ch <= lim; ++ch) {
                    c->chunk[s4] = ch;
                    float t = 0.f;
                    st = time_stage_range(c, s4, s4, iters, &t);
                    if (st) return st;
                    log(SFISTA_OP_BANDED, s4, ch, t);
                    if (best_ch == 0 || t < best) best = t, best_ch = ch;
                }
                c->chunk[s4] = best_ch;
            }
            float t_two = 0.f;
            st = time_loop(c, iters, &t_two);
            if (st) return st;
            log(SFISTA_OP_BANDED, -1, 0, t_two);
            c->op = SFISTA_OP_BANDED;
            float t_best = t_two;
            if (auto_op && band_op_fused_prepare(c->r, std::max(h.A.w, h.AT.w), std::max(h.B.w, h.BT.w))) {
                float t_fused = 0.f;
                c->op = SFISTA_OP_BANDED_FUSED;
                st = time_loop(c, iters, &t_fused);
                if (st) return st;
                log(SFISTA_OP_BANDED_FUSED, -1, 0, t_fused);
                c->op = t_fused < t_two ? SFISTA_OP_BANDED_FUSED : SFISTA_OP_BANDED;
                t_best = std::min(t_fused, t_two);
                // The one-launch fused solver, when every tile has a resident
                // block: every tile height th from 32 down to 16 that fits is
                // timed (entries report th in `chunk`), or only the requested one.
                const int best_op = c->op;
                int best_th = 0, best_grid = 0;
                size_t best_smem = 0;
                for (int th = 64; th >= 16; th -= 4) {
                    if (c->opts.tile_override && th != c->opts.tile_override) continue;
                    int grid = 0;
                    size_t smem = 0;
                    if (!band_solve_fused_config_th(ctx_prob(c), c->dev, th, &grid, &smem)) continue;
                    if (!c->bar) {
                        SF_CUDA(cudaMalloc((void **)&c->bar, kBarrierBytes));
                        SF_CUDA(cudaMemset(c->bar, 0, kBarrierBytes));
                    }
                    c->op = SFISTA_OP_BANDED_PERSISTENT;
                    c->pfused = 1;   // band_op_fused_prepare succeeded above
                    c->pgrid = grid;
                    c->psmem = smem;
                    c->pth = th;
                    float t_one = 0.f;
                    st = time_loop(c, std::max(iters, 40), &t_one);
                    if (st) return st;
                    log(SFISTA_OP_BANDED_PERSISTENT, -1, th, t_one);
                    if (t_one < t_best) {
                        t_best = t_one;
                        best_th = th;
                        best_grid = grid;
                        best_smem = smem;
                    }
                }
                if (best_th) {
                    c->op = SFISTA_OP_BANDED_PERSISTENT;
                    c->pfused = 1;
                    c->pgrid = best_grid;
                    c->psmem = best_smem;
                    c->pth = best_th;
                } else {
                    c->op = best_op;
                }
            }
            if (auto_op) {
                // The FFT form: its cost does not grow with the PSF width or r,
                // so it wins for wide PSFs.  Skipped when its transforms do not fit.
                const int best_op = c->op;
                bool have = c->fft != nullptr;
                if (!have) {
                    have = make_fft(c) == SFISTA_OK;
                    set_error("");
                }
                if (have) {
                    float t_fft = 0.f;
                    c->op = SFISTA_OP_FFT;
                    st = time_loop(c, iters, &t_fft);
                    if (st) return st;
                    log(SFISTA_OP_FFT, -1, 0, t_fft);
                    if (!(t_fft < t_best)) c->op = best_op;
                }
            }
        } else {
            c->op = chosen;
        }
    } else if (c->gemm && auto_op) {
        float t_band = 0.f, t_dense = 0.f;
        c->op = SFISTA_OP_GEMM_BAND;
        gemm_set_dense(c->gemm, false);
        st = time_loop(c, iters, &t_band);
        if (st) return st;
        log(SFISTA_OP_GEMM_BAND, -1, 0, t_band);
        c->op = SFISTA_OP_GEMM_DENSE;
        gemm_set_dense(c->gemm, true);
        st = time_loop(c, iters, &t_dense);
        if (st) return st;
        log(SFISTA_OP_GEMM_DENSE, -1, 0, t_dense);
        const bool dense = t_dense < t_band;
        c->op = dense ? SFISTA_OP_GEMM_DENSE : SFISTA_OP_GEMM_BAND;
        gemm_set_dense(c->gemm, dense);
    }
    if (c->gemm) {
        // Tile shape of each tensor-core stage in the chosen K mode, timed
        // alone: the N tile width (entries report it in `chunk`) of the
        // summed stages 1 and 3 (64, 128 or 256) and of the stacked stages 0
        // and 2 (64 or 128, each streamed or, chunk + 1, with the resident
        // factor panel).
        for (int s4 = 0; s4 < 4; ++s4) {
            int bn[4], res[4];
            const int nopt = gemm_tile_options(c->gemm, s4, bn, res);
            if (nopt < 2) continue;
            float best = 0.f;
            int bi = -1;
            for (int o = 0; o < nopt; ++o) {
                gemm_set_tile(c->gemm, s4, bn[o], res[o]);
                float t = 0.f;
                st = time_stage_range(c, s4, s4, iters, &t);
                if (st) return st;
                log(c->op, s4, s4 % 2 == 0 ? bn[o] + res[o] : bn[o], t);
                if (bi < 0 || t < best) best = t, bi = o;
            }
            gemm_set_tile(c->gemm, s4, bn[bi], res[bi]);
        }
    }
    if (c->gexec) {   // the cached loop graph holds the old configuration
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->g_k0 = c->g_iters = -1;
    }
    SF_CUDA(cudaStreamSynchronize(c->stream));
    st = drain_status(c);
    SF_CUDA(cudaMemset(c->status, 0, 16));
    if (n_entries) *n_entries = count;
    return st;
}

sfista_status sfista_selftest_wait_timeout(sfista_ctx *c) {
    sfista_status st = check_ctx(c);
    if (st) return st;
    DeviceGuard g(c->dev);
    SF_CUDA(cudaStreamSynchronize(c->stream));
    st = drain_status(c);   // start from a clean status word
    if (st) return st;
    launch_wait_timeout_selftest(c->status, c->stream);
    SF_CUDA(cudaGetLastError());
    return drain_status(c);
}

const char *sfista_strerror(sfista_status s) {
    switch (s) {
        case SFISTA_OK: return "ok";
        case SFISTA_EINVAL: return "invalid argument";
        case SFISTA_ENOMEM: return "out of memory";
        case SFISTA_ECUDA: return "CUDA error";
        case SFISTA_ENOTSUP: return "not supported";
        case SFISTA_ENUMERIC: return "non-finite value";
        case SFISTA_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *sfista_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
