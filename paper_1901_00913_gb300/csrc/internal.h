// Library-internal declarations shared by the host setup, the kernels and the
// C ABI of libsfista.  Nothing here is part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sfista.h"

namespace sfista {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
sfista_status fail(sfista_status s, const std::string &msg);
#define SF_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return ::sfista::fail(SFISTA_ECUDA, std::string(#call) + ": " +    \
                                                    cudaGetErrorString(e_));   \
    } while (0)

// Device status word bits (OR-reduced by kernels, read by sfista_sync).
enum : unsigned {
    DEV_NONFINITE = 1u,
    DEV_TIMEOUT = 2u,
    DEV_BADARG = 4u,
};

// ------------------------------------------------------------------ host setup (FP64)
// Band storage of one family of r banded n x n factors F_i:
//   F_i[row][row + lo + k] = band[(i * w + k) * len + row],  k in [0, w)
// (transposed so that consecutive rows are contiguous).  Entries whose column
// falls outside [0, len) are stored as zero.
struct Band {
    int len = 0, r = 0, lo = 0, w = 0;
    std::vector<double> band;   // r * w * len
};

struct HostSetup {
    int m = 0, n = 0, p = 0, q = 0, cr = 0, cc = 0, bc = 0, r = 0;
    std::vector<double> sigma;  // min(p, q) singular values of P_bar
    double approx_err = 0.0;    // sqrt(sum_{k > r} sigma_k^2)
    std::vector<double> C;      // r x p column profiles (left factors B_k)
    std::vector<double> D;      // r x q row profiles (right factors A_k)
    Band A, AT, B, BT;          // right factor, its transpose, left factor, its transpose
};

// Sec. 2 / Theorem 1 in FP64; returns SFISTA_OK or an error (message set).
sfista_status host_setup(const double *psf, int p, int q, int cr, int cc, int m,
                         int n, int bc, int r, HostSetup *out);

// beta_k = (t_k - 1) / t_{k+1} for k = 1..iters (index k-1), t_1 = 1 (Alg. 2, Step 2).
void momentum_table(int k_end, std::vector<double> *beta);
// Widest run [*i0, *i1) of rows around len / 2 of an FP32 band table
// (cnt = r * w values per row, stored tbl[t * len + row]) whose values equal
// row len / 2 bit for bit: the Toeplitz interior of the factor family.
void band_interior(const float *tbl, int len, int cnt, int *i0, int *i1);

// ------------------------------------------------------------------ device kernels
// Banded operator passes (compact band storage), T = float or double.
// rows:  Z[i][a][c] = sum_k In[a][c + lo + k] * Fb[i][k][c]        (i < r)
// cols:  acc[a][c]  = sum_i sum_k Gb[i][k][a] * Z[i][a + lo + k][c]
enum EpiKind : int { EPI_STORE = 0, EPI_RESIDUAL = 1, EPI_PROX = 2 };

struct ProxArgs {
    const float *Bd;     // EPI_RESIDUAL: observed image
    // FISTA state as double-float pairs (hi, lo), 8 bytes per pixel.
    const float2 *Xin;   // EPI_PROX: X_{k-1}
    float2 *Xout;        // EPI_PROX: X_k (a different buffer, ping-pong)
    float2 *Y;           // EPI_PROX: Y_k in, Y_{k+1} out (in place)
    float *Yop;          // EPI_PROX: FP32 copy of Y_{k+1} (operand of the next GEMM/pass)
    void *Yhi, *Ylo;     // EPI_PROX: optional split copies (bf16 or tf32-in-fp32), may be NULL
    int split_kind;      // 0 none, 1 bf16 hi/lo, 2 tf32 hi/lo (fp32 storage)
    const float2 *beta;  // momentum table (double-float), beta[k-1] for iteration k
    int k;               // iteration index (1-based)
    double L, lam2;      // Lipschitz constant and lambda^2
    float2 inv_den;      // 1 / (L + lambda^2), double-float
    float2 shrink;       // L / (L + lambda^2), double-float
    int project;         // max(X, 0) after the shrink
    float2 tau;          // mu / (L + lambda^2), double-float: soft threshold of the l1 term (0: none)
    unsigned *status;    // device status word
    // Tensor-core forms: FP32 state (X_{k-1} in, X_k out, Y in place) that
    // their EPI_PROX epilogue uses instead of Xin / Xout / Y; NULL otherwise.
    const float *Xin32;
    float *Xout32, *Y32;
};

// chunk: terms staged per block (0: the default rule, a shared-memory budget);
// a chunk that does not fit falls back to the default.
template <typename T>
void launch_band_rows(const T *In, int m, int n, const T *Fb, int lo, int w, int r, T *Z,
                      cudaStream_t s, int chunk = 0);
template <typename T>
void launch_band_cols(const T *Z, int m, int n, const T *Gb, int lo, int w, int r,
                      EpiKind epi, T *Out, const ProxArgs &pa, cudaStream_t s, int chunk = 0);

// Out + i * m * n = G_i In for every term i (FP32, terms not summed).
void launch_band_cols_each(const float *In, int m, int n, const float *Gb, int lo, int w, int r, float *Out,
                           cudaStream_t s);

size_t band_rows_smem(int w, size_t elem);
size_t band_cols_smem(int w, size_t elem);
// Largest FP32 term chunk of a rows (cols) block of band width w that fits in
// shared memory, at most r.
int band_rows_chunk_limit(int r, int w);
int band_cols_chunk_limit(int r, int w);
// Shared memory of an FP32 rows (cols) block staging `chunk` terms of width w.
size_t band_smem_f32(bool rows, int w, int chunk);
cudaError_t band_set_smem_limits(int w);

// Persistent cooperative solver (kernels_persistent.cu).
sfista_status persistent_config(int m, int n, int r, int wmax, int dev, int *grid, size_t *smem, int *rows_chunk,
                                int *cols_chunk);
cudaError_t launch_persistent(int grid, size_t smem, int rows_chunk, int cols_chunk, int m, int n, int r, const float *fA, const Band &A,
                              const float *fB, const Band &B, const float *fAT, const Band &AT, const float *fBT,
                              const Band &BT, float *Z, float *R, float2 *Xb0, float2 *Xb1, const ProxArgs &pa,
                              int k0, int iters, unsigned *bar, cudaStream_t s);

// Bytes of grid-barrier words the persistent solvers use.
constexpr size_t kBarrierBytes = 1024;

// Grouped (batched) banded FP32 execution: one launch per stage over the
// tiles of many problems of any size, rank and band.
struct BandProb {
    int m, n, r, rows_chunk, cols_chunk;
    int vec;       // 1: the 16-byte FP32 routines with 64-row tiles (m, n multiples of 4), 0: 32-row scalar ones
    const float *fA, *fB, *fAT, *fBT;
    int loA, wA, loB, wB, loAT, wAT, loBT, wBT;
    float *Z, *R;
    ProxArgs pa;   // Bd, Y, Yop, beta, constants, status; Xin / Xout = state buffers 0 / 1
    float *xout;   // one-launch batch: the FP32 result X_iters, written by the solver itself
    int4 tfwd, tadj;   // interior ranges (f0, f1, g0, g1) of (A, B) and (A^T, B^T); see launch_band_op_fused
    int th;            // one-launch solver: output rows per tile (multiple of 4, <= 64; <= 32 in batches)
};
struct BandItem {
    int prob, q, tile, pad;   // rows pass: q = term chunk; cols pass: q = 0
};

// The whole solve in one cooperative launch of the fused operator kernel
// (kernels_fused.cu), when every th x 32 output tile has a resident block:
// for one problem, or for a batch (one block per tile of every problem).
// The configs pick the tile height th (set it in the descriptors' th).
// The descriptor's pa.Xin / pa.Xout are the state buffers 0 / 1.
bool band_solve_fused_config(const BandProb &prob, int dev, int *grid, size_t *smem, int *th);
// The same for a given tile height th (a multiple of 4 from 16 to 64); false
// when those tiles do not all fit as co-resident blocks.
bool band_solve_fused_config_th(const BandProb &prob, int dev, int th, int *grid, size_t *smem);
cudaError_t launch_band_solve_fused(int grid, size_t smem, const BandProb &prob, int k0, int iters, unsigned *bar,
                                    cudaStream_t s);
bool band_solve_fused_batch_config(const BandProb *probs, int np, int dev, std::vector<int2> *items, size_t *smem,
                                   int *th);
cudaError_t launch_band_solve_fused_batch(int nitems, size_t smem, const BandProb *d_probs, const int2 *d_items,
                                          int iters, unsigned *bar, cudaStream_t s);
void persistent_chunks(int r, int wmax, int *rows_chunk, int *cols_chunk, size_t *smem);
// Term chunks of the grouped batch kernels: the requested ones (> 0, e.g.
// from the autotuner) when they fit, else the persistent solver's rule.
void grouped_chunks(int r, int wmax, bool vec, int rows_req, int cols_req, int *rows_chunk, int *cols_chunk,
                    size_t *smem);
cudaError_t band_grouped_prepare(size_t smem);
void launch_band_grouped_stage(int st, const BandProb *probs, const BandItem *items, int nitems, int k, size_t smem,
                               cudaStream_t s);
int band_rows_tiles(int m, int n, bool vec);
int band_cols_tiles(int m, int n, bool vec);

// One kernel per banded operator application (kernels_fused.cu).  tr =
// (f0, f1, g0, g1): the output columns of Fb and rows of Gb whose band rows
// equal the Toeplitz row stored after the table (empty range: none stored).
size_t band_op_fused_smem(int r, int wF, int wG);
bool band_op_fused_prepare(int r, int wF, int wG);
void launch_band_op_fused(const float *In, int m, int n, int r, const float *Fb, int loF, int wF, const float *Gb,
                          int loG, int wG, EpiKind epi, float *Out, const ProxArgs &pa, int4 tr, cudaStream_t s);

inline bool is_banded(int op) {
    return op == SFISTA_OP_BANDED || op == SFISTA_OP_BANDED_PERSISTENT || op == SFISTA_OP_BANDED_FUSED;
}
// The FFT engine (fftconv.h): the Kronecker operator, or the exact blur.
inline bool is_fft(int op) { return op == SFISTA_OP_FFT || op == SFISTA_OP_EXACT_FFT; }

// Small helpers.
void launch_fill_f64(double *p, size_t count, double v, cudaStream_t s);
void launch_f64_to_f32(const double *in, float *out, size_t count, cudaStream_t s);
// Double-float state conversions.
void launch_df_to_f32(const float2 *in, float *out, size_t count, cudaStream_t s);
void launch_f32_to_df(const float *in, float2 *out, size_t count, cudaStream_t s);
void launch_df_to_f64(const float2 *in, double *out, size_t count, cudaStream_t s);
void launch_f64_to_df(const double *in, float2 *out, size_t count, cudaStream_t s);
void launch_f32_to_f64(const float *in, double *out, size_t count, cudaStream_t s);
void launch_split(const float *in, void *hi, void *lo, size_t count, int kind,
                  cudaStream_t s);
void launch_check_finite(const float *in, size_t count, unsigned *status, cudaStream_t s);
void launch_seed_image(double *v, size_t count, cudaStream_t s);
// dot[0] = <u, v>, dot[1] = <v, v>  (FP64, deterministic two-pass reduction)
void launch_dots(const double *u, const double *v, size_t count, double *partial,
                 int nblk, double *dot, cudaStream_t s);
void launch_scale(double *v, size_t count, const double *dot, cudaStream_t s);
// *out = sum_i (a_i - b_i)^2 (b may be NULL) in FP64; partial holds nblk doubles.
void launch_sumsq(const float *a, const float *b, size_t count, double *partial, int nblk, double *out,
                  cudaStream_t s);
void launch_blur_exact(const float *X, int m, int n, const float *P, int p, int q,
                       int cr, int cc, int bc, float *Y, cudaStream_t s);
// Dense factor panels from band storage: F[i][row][col] for col in [0, cols).
// kind: 0 fp32, 1 bf16 hi/lo, 2 tf32 hi/lo (fp32 storage), 3 fp64.
void launch_densify(const double *band, int r, int len, int lo, int w, int cols,
                    int kind, void *hi, void *lo_out, size_t ld, cudaStream_t s);

}  // namespace sfista
