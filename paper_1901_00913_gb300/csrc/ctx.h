// Library-internal definition of the solver context (shared by the C ABI
// translation units).  Not part of the public interface.
#pragma once

#include <vector>

#include "fftconv.h"
#include "gemm.h"
#include "internal.h"

namespace sfista {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace sfista

struct sfista_ctx {
    using HostSetup = sfista::HostSetup;
    using GemmPath = sfista::GemmPath;
    int dev = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    HostSetup hs;
    sfista_opts opts;
    int prec = SFISTA_FP32, op = SFISTA_OP_BANDED;
    double L = 0.0;
    int m = 0, n = 0, r = 0;
    size_t N = 0;
    // Band storage on the device: FP64 (power iteration) and FP32 (operator).
    double *dA = nullptr, *dAT = nullptr, *dB = nullptr, *dBT = nullptr;
    float *fA = nullptr, *fAT = nullptr, *fB = nullptr, *fBT = nullptr;
    // Interior ranges [x, y) of A, A^T, B, B^T: the band rows equal (bit for
    // bit, FP32) to the Toeplitz row stored after each FP32 table.
    int2 interior[4] = {};
    // Iteration state.
    float *Bd = nullptr, *Yop = nullptr, *Z = nullptr, *R = nullptr, *tmp = nullptr;
    float2 *Xb[2] = {nullptr, nullptr}, *Y = nullptr;   // double-float FISTA state
    // Tensor-core forms: the FP32 state their prox epilogue iterates on,
    // converted from / to Xb and Y at the start / end of each solve.
    float *Xf[2] = {nullptr, nullptr}, *Yf = nullptr;
    unsigned *status = nullptr;
    float2 *beta = nullptr;        // double-float momentum table
    int beta_len = 0;
    std::vector<double> beta_host;
    // Tensor-core path (operand panels, intermediates, tensor maps).
    GemmPath *gemm = nullptr;
    // FFT form (SFISTA_OP_FFT, or the exact blur of a sfista_setup_exact
    // context: exact = 1, no band storage).
    sfista::FftConv *fft = nullptr;
    int exact = 0;
    int custom_factors = 0;   // sfista_set_factors replaced the setup's factors
    // Terms per block of the two-pass banded stages 0..3 (0: default rule);
    // set by the autotuner.
    int chunk[4] = {0, 0, 0, 0};
    // Persistent solver launch shape and its grid-barrier words; pfused: the
    // one-launch fused solver (every tile resident), else the two-pass one.
    int pgrid = 0, prows_chunk = 1, pcols_chunk = 1, pfused = 0, pth = 32;   // pth: one-launch tile height
    size_t psmem = 0;
    unsigned *bar = nullptr;
    // Cached CUDA graph of the iteration loop.
    cudaGraphExec_t gexec = nullptr;
    int g_k0 = -1, g_iters = -1;
    double g_lam = -1.0;
};

namespace sfista {

// Single operator applications take the fused kernel (one launch each): the
// fused form, and the one-launch solver that is built on it.
inline bool fused_apply(const sfista_ctx *c) {
    return c->op == SFISTA_OP_BANDED_FUSED || (c->op == SFISTA_OP_BANDED_PERSISTENT && c->pfused);
}

// Interior ranges (f0, f1, g0, g1) of the forward (A, B) and adjoint
// (A^T, B^T) band pairs, as the fused kernels take them.
inline int4 interior_fwd(const sfista_ctx *c) {
    return make_int4(c->interior[0].x, c->interior[0].y, c->interior[2].x, c->interior[2].y);
}
inline int4 interior_adj(const sfista_ctx *c) {
    return make_int4(c->interior[1].x, c->interior[1].y, c->interior[3].x, c->interior[3].y);
}

// Helpers of capi.cu used by the other C-ABI translation units.
ProxArgs prox_args(sfista_ctx *c, int k, double lam);
sfista_status ensure_beta(sfista_ctx *c, int k_end);
void enqueue_iteration(sfista_ctx *c, int k, double lam);
sfista_status solve_core(sfista_ctx *c, const float *d_b, double lam, int k0, int iters, const double *X_in,
                         const double *Xprev_in, cudaStream_t user);
sfista_status drain_status(sfista_ctx *c);
sfista_status finish_on_user(sfista_ctx *c, cudaStream_t user);
void launch_init_state(const float2 *X, const float2 *Xp, float2 *Y, float *Yop, void *Yhi, void *Ylo, int split_kind,
                       size_t count, double beta, cudaStream_t s);

}  // namespace sfista
