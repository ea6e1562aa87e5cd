// FFT form of the operator (fftconv.cu): the boundary-extended image
// convolved with a 2-D kernel (the rank-r kernel sum_i c_i d_i^T of the
// Kronecker approximation, or the PSF itself for the exact blur) through
// mixed-radix FFTs in shared memory.  Library-internal.
#pragma once

#include "internal.h"

namespace sfista {

constexpr int kFftMaxStages = 14;
constexpr int kFftMaxLen = 8192;   // longest line transform (one line, its twiddles and positions: 160 KB of shared memory)

// DIF stage plan of one line length N = prod R[j]; stage j has stride M[j]
// and its twiddles at tw[j] in the plan's table ((R - 1) * M values).
struct FftLine {
    int N, ns;
    int R[kFftMaxStages], M[kFftMaxStages], tw[kFftMaxStages];
};

// Device view (passed to the kernels by value).
struct FftConvDev {
    int m, n, bc;
    int offr, offc;           // extension rows above / columns left: p - 1 - cr, q - 1 - cc
    int ext_rows, ext_cols;   // m + p - 1, n + q - 1
    int H2;                   // N2 / 2 + 1 stored frequencies along rows
    int sr1, sr2;             // rows of S1, S2: ext_rows, m rounded up to whole 8-row tiles
    FftLine l1, l2;           // column transforms (length N1 >= ext_rows), row transforms (N2 >= ext_cols)
    const float2 *tw1, *tw2;  // twiddle tables (N - 1 values each)
    const int *pos2;          // pos2[f]: DIF position of row frequency f
    const float2 *K;          // kernel spectrum / (N1 N2): H2 x N1, the column frequency in DIF order
    float2 *S1, *S2;          // half spectra in 8-row tiles: (row, f) at ((row / 8) * H2 + f) * 8 + row % 8
};

struct FftConv {
    FftConvDev d{};
    int lpc_a = 1, lpc_b = 1, lpc_c = 1;   // lines per block of the three passes
    bool big1 = false, big2 = false;        // the column (l1) / row (l2) plan has radix-9 or radix-16 stages
};

// K: p x q kernel (FP64, row-major) with centre (cr, cc), for m x n images.
sfista_status fftconv_create(FftConv **out, const double *K, int p, int q, int cr, int cc, int m, int n, int bc);
void fftconv_destroy(FftConv *f);
// Out = A In (adj = false) or A^T In (adj = true) with the epilogue: part 0 =
// Passes A and B (In read), part 1 = Pass C with the epilogue (Out written).
void fftconv_part(const FftConv *f, int part, bool adj, const float *In, EpiKind epi, float *Out, const ProxArgs &pa,
                  cudaStream_t s);
// Pass C of the forward operator with the residual R = A Y - B, fused with
// Pass A of the adjoint on R (R is not written to global memory): after it,
// fftconv_adjoint_columns and fftconv_part(1, adj = true, ...) complete the
// adjoint product.
void fftconv_residual_adjoint(const FftConv *f, const ProxArgs &pa, cudaStream_t s);
// Pass B of the adjoint (column transforms with the conjugate kernel spectrum).
void fftconv_adjoint_columns(const FftConv *f, cudaStream_t s);
void fftconv_apply(const FftConv *f, bool adj, const float *In, EpiKind epi, float *Out, const ProxArgs &pa,
                   cudaStream_t s);
// Device bytes the engine holds (spectra and kernel spectrum).
size_t fftconv_bytes(const FftConv *f);

}  // namespace sfista
