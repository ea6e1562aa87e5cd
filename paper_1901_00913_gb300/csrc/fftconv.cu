// FFT form of the operator: the boundary-extended image convolved with a 2-D
// kernel through mixed-radix FFTs in shared memory.
//
// Why one 2-D convolution.  A right factor A_i = toep(d_i) [+ hank(d_i)]
// applies the row profile d_i to the zero or reflected extension of each row,
// and a left factor B_i does the same along columns with c_i (Sec. 2; the
// Hankel part is exactly the reflection).  The extension acts on each axis
// separately, so
//   (sum_i B_i X A_i^T)[a][b] = sum_{k,l} K[k][l] Xext[a - k + cr][b - l + cc],
//   K = sum_i c_i d_i^T,
// one 2-D convolution of the extended image with the rank-r kernel K.  The
// exact blur of Eq. (1.1) has the same form with K = P (the PSF itself), so
// the same engine applies A for vector FISTA on the unapproximated blur
// (Alg. 1).  The paper's structured products transform every term's factor
// separately (1-D FFTs per term); here the r terms are summed in the kernel,
// so the cost does not grow with r.
//
// Index conventions (rows; columns alike with n, q, cc).  offr = p - 1 - cr
// extension rows lie above row 0; the extended image has m + p - 1 rows,
// row s holding source row ext(s - offr) (zero or half-sample reflection, as
// the Hankel part of Sec. 2 encodes).  With N1 >= m + p - 1 (no wrap-around):
//   forward:  y = h (*) E, h[u mod N1] = K[u + p - 1] for u in [-(p-1), 0],
//             output rows a in [0, m) are y[a];
//   adjoint:  u = g (*) R0 with g[s] = K[p - 1 - s] (conj(h^) in frequency),
//             R0 the input zero-padded, output row a sums u[s] over the s with
//             ext(s - offr) = a (the transpose of the extension: a fold).
// (*) is circular convolution of length N1, done as pointwise products of
// spectra.
//
// Three passes per application (Pass A and Pass C along rows, Pass B along
// columns), each one kernel:
//   A  two real rows packed as one complex line (real, imaginary part), the
//      extension gathered on load, a decimation-in-frequency FFT, then the
//      half spectra of the two rows unpacked (Hermitian symmetry) to S1.
//   B  per frequency column f of S1: DIF FFT along the rows, product with the
//      kernel spectrum (conjugated for the adjoint), inverse DIT FFT, the
//      output rows (forward) or the fold (adjoint) to S2.
//   C  two rows' half spectra packed into one complex line (Y_a + i Y_{a+1}),
//      inverse DIT FFT, real and imaginary parts are the two output rows;
//      column fold for the adjoint; then the epilogue (store, residual, or
//      Step 1 shrink + Step 3 momentum of Alg. 2 on the double-float state).
// The DIF FFT leaves its output in digit-reversed order and the inverse DIT
// FFT with the stages reversed reads exactly that order, so no reordering
// pass is needed: the kernel spectrum is stored in the same scrambled order
// (Pass B), and Pass A / C address frequency f at its scrambled position.
// Twiddles and kernel spectra are computed in FP64 on the host; all device
// arithmetic is FP32.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "epilogue.cuh"
#include "fftconv.h"

namespace sfista {
namespace {

constexpr int kThreads = 256;

// The passes' dynamic shared memory, addressed by element offsets (32-bit
// index arithmetic on a shared-space array).
extern __shared__ __align__(16) float2 fft_sm[];

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// -i * a (forward) or +i * a (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of R points, v[u] = sum_k v[k] w^(u k), w = exp(-+2 pi i / R)
// (minus: forward, plus: INV; no scaling).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]);

template <>
__device__ __forceinline__ void dft<2, false>(float2 (&v)[2]) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft<2, true>(float2 (&v)[2]) {
    dft<2, false>(v);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 (&v)[4]) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = rot<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}
template <>
__device__ __forceinline__ void dft<4, false>(float2 (&v)[4]) {
    dft4<false>(v);
}
template <>
__device__ __forceinline__ void dft<4, true>(float2 (&v)[4]) {
    dft4<true>(v);
}

// R = 3: w = c -+ i s with c = cos(2 pi / 3) = -1/2, s = sin(2 pi / 3) = sqrt(3)/2.
template <bool INV>
__device__ __forceinline__ void dft3(float2 (&v)[3]) {
    const float s3 = 0.86602540378443864676f;
    const float2 t = cadd(v[1], v[2]);
    const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    const float2 d = csub(v[1], v[2]);
    const float2 j = rot<INV>(make_float2(s3 * d.x, s3 * d.y));   // -+ i s (v1 - v2)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, j);
    v[2] = csub(m, j);
}
template <>
__device__ __forceinline__ void dft<3, false>(float2 (&v)[3]) {
    dft3<false>(v);
}
template <>
__device__ __forceinline__ void dft<3, true>(float2 (&v)[3]) {
    dft3<true>(v);
}

// R = 5 with c1 = cos(2 pi / 5), c2 = cos(4 pi / 5), s1 = sin(2 pi / 5),
// s2 = sin(4 pi / 5):  y1,4 = v0 + c1 t1 + c2 t2 -+ i (s1 d1 + s2 d2),
// y2,3 = v0 + c2 t1 + c1 t2 -+ i (s2 d1 - s1 d2), t = sums, d = differences
// of the mirrored pairs (1, 4) and (2, 3).
template <bool INV>
__device__ __forceinline__ void dft5(float2 (&v)[5]) {
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    const float2 b1 = rot<INV>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    const float2 b2 = rot<INV>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}
template <>
__device__ __forceinline__ void dft<5, false>(float2 (&v)[5]) {
    dft5<false>(v);
}
template <>
__device__ __forceinline__ void dft<5, true>(float2 (&v)[5]) {
    dft5<true>(v);
}

// R = 8 as two 4-point DFTs of the even and odd points combined with
// w8^u = exp(-+2 pi i u / 8), u < 4.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    const float h = 0.70710678118654752440f;
    const float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                          : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    const float2 o2 = rot<INV>(o[2]);
    const float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                          : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2 (&v)[8]) {
    dft8<false>(v);
}
template <>
__device__ __forceinline__ void dft<8, true>(float2 (&v)[8]) {
    dft8<true>(v);
}

// a * exp(-+i theta) with c = cos(theta), sn = sin(theta) (minus: forward,
// plus: INV).
template <bool INV>
__device__ __forceinline__ float2 twc(float2 a, float c, float sn) {
    return INV ? make_float2(a.x * c - a.y * sn, a.y * c + a.x * sn)
               : make_float2(a.x * c + a.y * sn, a.y * c - a.x * sn);
}

// R = n1 n2 in two levels (Cooley-Tukey on the register array): with
// v[n2 k2 + k1] (k2 < n1, k1 < n2),
//   X[u1 + n1 u2] = sum_k1 w_R^(k1 u1) w_n2^(k1 u2) sum_k2 v[n2 k2 + k1] w_n1^(k2 u1),
// i.e. n2 DFTs of n1 points, the internal twiddles w_R^(k1 u1), then n1
// DFTs of n2 points.  R = 16 = 4 x 4: w16^k = cos(2 pi k / 16) -+ i sin(.).
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;   // k = 1 (k = 3: swapped)
    const float h = 0.70710678118654752440f;                                   // k = 2, 6
    float2 y[4][4];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a[4] = {v[k1], v[4 + k1], v[8 + k1], v[12 + k1]};
        dft4<INV>(a);
#pragma unroll
        for (int u1 = 0; u1 < 4; ++u1) y[k1][u1] = a[u1];
    }
    // w16^(k1 u1), k1 u1 in {1, 2, 3, 4, 6, 9}
    y[1][1] = twc<INV>(y[1][1], c1, s1);
    y[1][2] = twc<INV>(y[1][2], h, h);
    y[1][3] = twc<INV>(y[1][3], s1, c1);
    y[2][1] = twc<INV>(y[2][1], h, h);
    y[2][2] = rot<INV>(y[2][2]);
    y[2][3] = twc<INV>(y[2][3], -h, h);
    y[3][1] = twc<INV>(y[3][1], s1, c1);
    y[3][2] = twc<INV>(y[3][2], -h, h);
    y[3][3] = twc<INV>(y[3][3], -c1, -s1);
#pragma unroll
    for (int u1 = 0; u1 < 4; ++u1) {
        float2 b[4] = {y[0][u1], y[1][u1], y[2][u1], y[3][u1]};
        dft4<INV>(b);
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) v[u1 + 4 * u2] = b[u2];
    }
}
template <>
__device__ __forceinline__ void dft<16, false>(float2 (&v)[16]) {
    dft16<false>(v);
}
template <>
__device__ __forceinline__ void dft<16, true>(float2 (&v)[16]) {
    dft16<true>(v);
}

// R = 9 = 3 x 3 the same way; w9^k = cos(2 pi k / 9) -+ i sin(.), k in {1, 2, 4}.
template <bool INV>
__device__ __forceinline__ void dft9(float2 (&v)[9]) {
    float2 y[3][3];
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        float2 a[3] = {v[k1], v[3 + k1], v[6 + k1]};
        dft3<INV>(a);
#pragma unroll
        for (int u1 = 0; u1 < 3; ++u1) y[k1][u1] = a[u1];
    }
    y[1][1] = twc<INV>(y[1][1], 0.76604444311897803520f, 0.64278760968653932632f);
    y[1][2] = twc<INV>(y[1][2], 0.17364817766693034885f, 0.98480775301220805936f);
    y[2][1] = twc<INV>(y[2][1], 0.17364817766693034885f, 0.98480775301220805936f);
    y[2][2] = twc<INV>(y[2][2], -0.93969262078590838405f, 0.34202014332566873304f);
#pragma unroll
    for (int u1 = 0; u1 < 3; ++u1) {
        float2 b[3] = {y[0][u1], y[1][u1], y[2][u1]};
        dft3<INV>(b);
#pragma unroll
        for (int u2 = 0; u2 < 3; ++u2) v[u1 + 3 * u2] = b[u2];
    }
}
template <>
__device__ __forceinline__ void dft<9, false>(float2 (&v)[9]) {
    dft9<false>(v);
}
template <>
__device__ __forceinline__ void dft<9, true>(float2 (&v)[9]) {
    dft9<true>(v);
}

// One butterfly of a stage: the R points x[k * M], k < R, with the stage's
// twiddles w[u - 1] = w_L^(u q), u >= 1, already loaded.
// DIF (forward): DFT, then the twiddles on outputs u >= 1.
// DIT inverse: conjugate twiddles on inputs u >= 1, then the inverse DFT.
template <int R, bool INV>
__device__ __forceinline__ void bfly(int x, int M, const float2 (&w)[R > 1 ? R - 1 : 1]) {
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = fft_sm[x + k * M];
    if (INV) {
#pragma unroll
        for (int u = 1; u < R; ++u) v[u] = cmulc(v[u], w[u - 1]);
        dft<R, true>(v);
    } else {
        dft<R, false>(v);
#pragma unroll
        for (int u = 1; u < R; ++u) v[u] = cmul(v[u], w[u - 1]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) fft_sm[x + k * M] = v[k];
}

// One stage of radix R over LINES transforms at buf + line * ls: a thread
// takes butterfly positions (b, q) of the stage and applies each to every
// line, so the position arithmetic and the twiddle loads are shared by the
// lines (and the lines' butterflies are independent work for the pipeline).
template <int R, bool INV, int LINES>
__device__ __forceinline__ void fft_stage(int buf, int ls, int N, int M, int t) {
    const int L = R * M, per = N / R, T = blockDim.x;
    // position bf = b * M + q of the thread's butterflies bf = tid, tid + T, ...:
    // divided once, then advanced by (T / M, T % M) with a carry
    const int db = T / M, dq = T - db * M;
    int b = threadIdx.x / M, q = threadIdx.x - b * M;
    for (int bf = threadIdx.x; bf < per; bf += T, b += db, q += dq) {
        if (q >= M) {
            q -= M;
            ++b;
        }
        float2 w[R - 1];
#pragma unroll
        for (int u = 1; u < R; ++u) w[u - 1] = fft_sm[t + (u - 1) * M + q];
        const int x = buf + b * L + q;
#pragma unroll
        for (int line = 0; line < LINES; ++line) bfly<R, INV>(x + line * ls, M, w);
    }
}

template <int R, bool INV>
__device__ __forceinline__ void fft_stage_lines(int buf, int lines, int ls, int N, int M, int t) {
    switch (lines) {
        case 1: fft_stage<R, INV, 1>(buf, ls, N, M, t); break;
        case 2: fft_stage<R, INV, 2>(buf, ls, N, M, t); break;
        default: fft_stage<R, INV, 4>(buf, ls, N, M, t); break;
    }
}

// All stages of `lines` in-place transforms of length P.N held in shared
// memory at buf + line * ls, the whole block cooperating; tw: the plan's
// twiddle table in shared memory.  Forward: DIF, natural order in,
// digit-reversed out.  INV: DIT with the stages in reverse order,
// digit-reversed in, natural out, unscaled.
template <bool INV, bool BIG>
__device__ void fft_lines(int buf, int lines, int ls, const FftLine &P, int tw) {
    for (int jj = 0; jj < P.ns; ++jj) {
        const int j = INV ? P.ns - 1 - jj : jj;
        const int M = P.M[j];
        const int t = tw + P.tw[j];
        switch (P.R[j]) {
            case 2: fft_stage_lines<2, INV>(buf, lines, ls, P.N, M, t); break;
            case 3: fft_stage_lines<3, INV>(buf, lines, ls, P.N, M, t); break;
            case 4: fft_stage_lines<4, INV>(buf, lines, ls, P.N, M, t); break;
            case 5: fft_stage_lines<5, INV>(buf, lines, ls, P.N, M, t); break;
            case 9:
                if constexpr (BIG) fft_stage_lines<9, INV>(buf, lines, ls, P.N, M, t);
                break;
            case 16:
                if constexpr (BIG) fft_stage_lines<16, INV>(buf, lines, ls, P.N, M, t);
                break;
            default: fft_stage_lines<8, INV>(buf, lines, ls, P.N, M, t); break;
        }
        __syncthreads();
    }
}

// Source index of extended index t on an axis of len pixels, or -1 (zero
// boundary outside, or beyond one reflection).
__device__ __forceinline__ int ext_src(int t, int len, int bc) {
    if (t >= 0 && t < len) return t;
    if (!bc) return -1;
    t = t < 0 ? -1 - t : 2 * len - 1 - t;
    return (t >= 0 && t < len) ? t : -1;
}

// Loop over [0, total) with the block's threads in batches of kBatch items
// per thread: every item's global loads (load(it)) are issued before any of
// them is used (use(it, value)), so a thread keeps kBatch loads in flight
// instead of waiting for each.
constexpr int kBatch = 8;
template <typename T, typename Load, typename Use>
__device__ __forceinline__ void batched(int total, Load load, Use use) {
    for (int base = threadIdx.x; base < total; base += kBatch * blockDim.x) {
        T v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int it = base + u * blockDim.x;
            if (it < total) v[u] = load(it);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int it = base + u * blockDim.x;
            if (it < total) use(it, v[u]);
        }
    }
}

// Half spectra are stored in tiles of 8 image rows: element (row s, frequency
// f) at ((s / 8) * H2 + f) * 8 + s % 8.  A Pass A / Pass C block (up to 8
// rows) then writes / reads one contiguous run per tile, and a Pass B block
// (neighbouring frequencies) reads and writes 8 * lines contiguous values
// per tile.
__device__ __forceinline__ size_t tile_index(int s, int f, int H2) {
    return ((size_t)(s >> 3) * H2 + f) * 8 + (s & 7);
}

// Shared layout of a pass (element offsets into fft_sm): `lines` line
// buffers of N + 1 values (the odd stride spreads the lanes of a stage over
// the banks) from 0, the twiddle table (N - 1 values) at tw, then (Passes A
// and C) the position table (N ints) at int offset pos.
struct PassSmem {
    int tw, pos;
};
__device__ __forceinline__ PassSmem pass_smem(int lines, int N) {
    PassSmem p;
    p.tw = lines * (N + 1);
    p.pos = 2 * (p.tw + N - 1);
    return p;
}
__device__ __forceinline__ int *fft_pos() { return reinterpret_cast<int *>(fft_sm); }

// Copies a plan's twiddle table and, if pos_g is non-NULL, its DIF position
// table into shared memory.
__device__ __forceinline__ void stage_tables(const FftLine &P, const float2 *__restrict__ tw_g,
                                             const int *__restrict__ pos_g, const PassSmem &sm) {
    for (int i = threadIdx.x; i < P.N - 1; i += blockDim.x) fft_sm[sm.tw + i] = __ldg(tw_g + i);
    if (pos_g)
        for (int i = threadIdx.x; i < P.N; i += blockDim.x) fft_pos()[sm.pos + i] = __ldg(pos_g + i);
}

// Loop over LPC lines x `cols` columns, columns strided over the block's
// threads in batches of kBatch per thread: each batch's global loads
// (load(line, col)) are issued before any is used (use(line, col, value)).
template <int LPC, typename T, typename Load, typename Use>
__device__ __forceinline__ void batched_lines(int cols, Load load, Use use) {
    for (int base = threadIdx.x; base < cols; base += kBatch * blockDim.x) {
#pragma unroll
        for (int j = 0; j < LPC; ++j) {
            T v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int t = base + u * blockDim.x;
                if (t < cols) v[u] = load(j, t);
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int t = base + u * blockDim.x;
                if (t < cols) use(j, t, v[u]);
            }
        }
    }
}

// Pass A: rows (extended rows for the forward operator) -> half spectra S1
// (8-row tiles).  LPC: complex lines (row pairs) per block.
template <bool ADJ, int LPC, bool BIG>
__global__ void __launch_bounds__(kThreads) fft_pass_a(FftConvDev P, const float *__restrict__ In) {
    const int N = P.l2.N, ls = N + 1;
    const PassSmem sm = pass_smem(LPC, N);
    stage_tables(P.l2, P.tw2, P.pos2, sm);
    const int rows = ADJ ? P.m : P.ext_rows;
    const int s0 = 2 * blockIdx.x * LPC;   // first row of the block
    batched_lines<LPC, float2>(
        N,
        [&](int j, int t) {
            const int s = s0 + 2 * j;
            float2 v = make_float2(0.f, 0.f);
            if (ADJ) {
                if (t < P.n) {
                    if (s < rows) v.x = __ldcg(In + (size_t)s * P.n + t);
                    if (s + 1 < rows) v.y = __ldcg(In + (size_t)(s + 1) * P.n + t);
                }
            } else if (t < P.ext_cols) {
                const int b = ext_src(t - P.offc, P.n, P.bc);
                if (b >= 0) {
                    const int a0 = s < rows ? ext_src(s - P.offr, P.m, P.bc) : -1;
                    const int a1 = s + 1 < rows ? ext_src(s + 1 - P.offr, P.m, P.bc) : -1;
                    if (a0 >= 0) v.x = __ldcg(In + (size_t)a0 * P.n + b);
                    if (a1 >= 0) v.y = __ldcg(In + (size_t)a1 * P.n + b);
                }
            }
            return v;
        },
        [&](int j, int t, float2 v) { fft_sm[j * ls + t] = v; });
    __syncthreads();
    fft_lines<false, BIG>(0, LPC, ls, P.l2, sm.tw);
    // Z = FFT(a + i b): A[f] = (Z[f] + conj Z[N-f]) / 2, B[f] = (Z[f] - conj Z[N-f]) / (2i);
    // the two rows' values at f leave as one 16-byte store, neighbouring
    // threads taking neighbouring row pairs of the same f (one contiguous run
    // per tile of 8 rows).
    const int *pos = fft_pos() + sm.pos;
    for (int it = threadIdx.x; it < LPC * P.H2; it += blockDim.x) {
        const int f = it / LPC, j = it - f * LPC;
        const int s = s0 + 2 * j;
        if (s >= rows) continue;
        const float2 z1 = fft_sm[j * ls + pos[f]];
        const float2 z2 = fft_sm[j * ls + pos[f == 0 ? 0 : N - f]];
        const float4 v = make_float4(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y), 0.5f * (z1.y + z2.y),
                                     0.5f * (z2.x - z1.x));
        *reinterpret_cast<float4 *>(P.S1 + tile_index(s, f, P.H2)) = v;   // s even: 16-byte aligned
    }
}

// Pass B: frequency lines of S1 -> kernel product along the rows -> S2.
// LPC: neighbouring frequencies per block.
template <bool ADJ, int LPC, bool BIG>
__global__ void __launch_bounds__(kThreads) fft_pass_b(FftConvDev P) {
    const int N = P.l1.N, ls = N + 1;
    const PassSmem sm = pass_smem(LPC, N);
    stage_tables(P.l1, P.tw1, nullptr, sm);
    const int rows_in = ADJ ? P.m : P.ext_rows;
    const int f0 = blockIdx.x * LPC;
    constexpr int run = 8 * LPC;   // contiguous values per 8-row tile: LPC frequencies x 8 rows
    const int Nt = (N + 7) & ~7;
    batched<float2>(
        LPC * Nt,
        [&](int it) {
            const int sb = it / run, rem = it - sb * run;
            const int j = rem >> 3, s = sb * 8 + (rem & 7);
            const int f = f0 + j;
            return (s < rows_in && f < P.H2) ? __ldcg(P.S1 + tile_index(s, f, P.H2)) : make_float2(0.f, 0.f);
        },
        [&](int it, float2 v) {
            const int sb = it / run, rem = it - sb * run;
            const int s = sb * 8 + (rem & 7);
            if (s < N) fft_sm[(rem >> 3) * ls + s] = v;
        });
    __syncthreads();
    fft_lines<false, BIG>(0, LPC, ls, P.l1, sm.tw);
    batched_lines<LPC, float2>(
        N,
        [&](int j, int t) { return f0 + j < P.H2 ? __ldg(P.K + (size_t)(f0 + j) * N + t) : make_float2(0.f, 0.f); },
        [&](int j, int t, float2 k) {
            float2 &x = fft_sm[j * ls + t];
            x = ADJ ? cmulc(x, k) : cmul(x, k);
        });
    __syncthreads();
    fft_lines<true, BIG>(0, LPC, ls, P.l1, sm.tw);
    const int mt = (P.m + 7) & ~7;
    for (int it = threadIdx.x; it < LPC * mt; it += blockDim.x) {
        const int ab = it / run, rem = it - ab * run;
        const int j = rem >> 3, a = ab * 8 + (rem & 7);
        const int f = f0 + j;
        if (f >= P.H2 || a >= P.m) continue;
        const float2 *u = fft_sm + j * ls;
        float2 v;
        if (ADJ) {
            // extended rows s with ext(s - offr) = a: s = a + offr, and for the
            // reflective boundary offr - 1 - a and 2m - 1 - a + offr
            v = u[a + P.offr];
            if (P.bc) {
                const int s1 = P.offr - 1 - a, s2 = 2 * P.m - 1 - a + P.offr;
                if (s1 >= 0) v = cadd(v, u[s1]);
                if (s2 < P.ext_rows) v = cadd(v, u[s2]);
            }
        } else {
            v = u[a];
        }
        P.S2[tile_index(a, f, P.H2)] = v;
    }
}

// Pass C: two rows' half spectra -> one inverse FFT -> the two output rows,
// then the epilogue.  LPC: row pairs per block.
template <bool ADJ, int EPI, int LPC, bool BIG>
__global__ void __launch_bounds__(kThreads) fft_pass_c(FftConvDev P, float *__restrict__ Out, ProxArgs pa) {
    const int N = P.l2.N, ls = N + 1;
    const PassSmem sm = pass_smem(LPC, N);
    stage_tables(P.l2, P.tw2, P.pos2, sm);
    __syncthreads();
    const int a0 = 2 * blockIdx.x * LPC;
    const int *pos = fft_pos() + sm.pos;
    batched<float4>(
        LPC * N,
        [&](int it) {
            const int f = it / LPC, j = it - f * LPC;   // neighbouring threads: neighbouring row pairs
            const int a = a0 + 2 * j;
            const int g = f >= P.H2 ? N - f : f;
            return a < P.m ? __ldcg(reinterpret_cast<const float4 *>(P.S2 + tile_index(a, g, P.H2)))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        },
        [&](int it, float4 y) {
            const int f = it / LPC, j = it - f * LPC;
            if (f >= P.H2) {   // Y[f] = conj Y[N - f] for a real row
                y.y = -y.y;
                y.w = -y.w;
            }
            // Y_a + i Y_{a+1}; row a + 1 past the image reads the zero padding of S2
            fft_sm[j * ls + pos[f]] = make_float2(y.x - y.w, y.y + y.z);
        });
    __syncthreads();
    fft_lines<true, BIG>(0, LPC, ls, P.l2, sm.tw);
    // Output pixels of each of the block's 2 LPC rows, kEpi per thread at a
    // time (their state / observation loads issued together).
    const int n = P.n;
    constexpr int kEpi = 4;
#pragma unroll 1
    for (int rr = 0; rr < 2 * LPC; ++rr) {
        const int a = a0 + rr;
        if (a >= P.m) break;
        const float2 *ub = fft_sm + (rr >> 1) * ls;
        for (int base = threadIdx.x; base < n; base += kEpi * blockDim.x) {
            float g[kEpi];
            size_t idx[kEpi];
            bool ok[kEpi];
#pragma unroll
            for (int u = 0; u < kEpi; ++u) {
                const int b = base + u * blockDim.x;
                ok[u] = b < n;
                idx[u] = (size_t)a * n + b;
                g[u] = 0.f;
                if (!ok[u]) continue;
                float2 w;
                if (ADJ) {
                    w = ub[b + P.offc];
                    if (P.bc) {
                        const int t1 = P.offc - 1 - b, t2 = 2 * n - 1 - b + P.offc;
                        if (t1 >= 0) w = cadd(w, ub[t1]);
                        if (t2 < P.ext_cols) w = cadd(w, ub[t2]);
                    }
                } else {
                    w = ub[b];
                }
                g[u] = (rr & 1) ? w.y : w.x;
            }
            if (EPI == EPI_STORE) {
#pragma unroll
                for (int u = 0; u < kEpi; ++u)
                    if (ok[u]) Out[idx[u]] = g[u];
            } else if (EPI == EPI_RESIDUAL) {
                float bv[kEpi];
#pragma unroll
                for (int u = 0; u < kEpi; ++u) bv[u] = ok[u] ? __ldcg(pa.Bd + idx[u]) : 0.f;
#pragma unroll
                for (int u = 0; u < kEpi; ++u)
                    if (ok[u]) Out[idx[u]] = g[u] - bv[u];
            } else {
                prox_momentum_n<kEpi>(pa, idx, g, ok);
            }
        }
    }
}

// Pass C of the forward operator with the residual, fused with Pass A of
// the adjoint: the inverse row transforms give (A Y)_a + i (A Y)_{a+1}, the
// residual R = A Y - B of the two rows replaces them in the same line buffer
// (columns n .. N - 1, and a row past the image, set to zero as Pass A's
// zero padding would), and the forward row transform of R and the Hermitian
// unpacking into the half spectra S1 follow without R leaving shared memory.
// Pass B of the adjoint then reads S1.  Same row pairs, line plan, twiddles
// and positions as the two passes it replaces.
template <int LPC, bool BIG>
__global__ void __launch_bounds__(kThreads) fft_pass_ca(FftConvDev P, ProxArgs pa) {
    const int N = P.l2.N, ls = N + 1;
    const PassSmem sm = pass_smem(LPC, N);
    stage_tables(P.l2, P.tw2, P.pos2, sm);
    __syncthreads();
    const int a0 = 2 * blockIdx.x * LPC;
    const int *pos = fft_pos() + sm.pos;
    batched<float4>(
        LPC * N,
        [&](int it) {
            const int f = it / LPC, j = it - f * LPC;
            const int a = a0 + 2 * j;
            const int g = f >= P.H2 ? N - f : f;
            return a < P.m ? __ldcg(reinterpret_cast<const float4 *>(P.S2 + tile_index(a, g, P.H2)))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        },
        [&](int it, float4 y) {
            const int f = it / LPC, j = it - f * LPC;
            if (f >= P.H2) {
                y.y = -y.y;
                y.w = -y.w;
            }
            fft_sm[j * ls + pos[f]] = make_float2(y.x - y.w, y.y + y.z);
        });
    __syncthreads();
    fft_lines<true, BIG>(0, LPC, ls, P.l2, sm.tw);
    // Residual of each row, in place: row 2j + 0 in the real part of line j,
    // row 2j + 1 in the imaginary part.  Each thread reads and rewrites only
    // its own elements, one component per row.
    const int n = P.n;
    constexpr int kEpi = 4;
#pragma unroll 1
    for (int rr = 0; rr < 2 * LPC; ++rr) {
        const int a = a0 + rr;
        float2 *ub = fft_sm + (rr >> 1) * ls;
        for (int base = threadIdx.x; base < N; base += kEpi * blockDim.x) {
            float bv[kEpi];
#pragma unroll
            for (int u = 0; u < kEpi; ++u) {
                const int b = base + u * blockDim.x;
                bv[u] = (a < P.m && b < n) ? __ldcg(pa.Bd + (size_t)a * n + b) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kEpi; ++u) {
                const int b = base + u * blockDim.x;
                if (b >= N) continue;
                float &c = (rr & 1) ? ub[b].y : ub[b].x;
                c = (a < P.m && b < n) ? c - bv[u] : 0.f;   // zero padding past the row and past the image
            }
        }
    }
    __syncthreads();
    fft_lines<false, BIG>(0, LPC, ls, P.l2, sm.tw);
    for (int it = threadIdx.x; it < LPC * P.H2; it += blockDim.x) {
        const int f = it / LPC, j = it - f * LPC;
        const int s2 = a0 + 2 * j;
        if (s2 >= P.m) continue;
        const float2 z1 = fft_sm[j * ls + pos[f]];
        const float2 z2 = fft_sm[j * ls + pos[f == 0 ? 0 : N - f]];
        const float4 v = make_float4(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y), 0.5f * (z1.y + z2.y),
                                     0.5f * (z2.x - z1.x));
        *reinterpret_cast<float4 *>(P.S1 + tile_index(s2, f, P.H2)) = v;
    }
}

// Kernel instances by lines per block (1, 2, 4) and by whether the line's
// plan has radix-9 / radix-16 stages (BIG: those butterflies need about
// twice the registers, so plans without them use instances without them
// and keep their occupancy).
template <bool ADJ, bool BIG>
void launch_a2(int lpc, int grid, size_t smem, cudaStream_t s, const FftConvDev &d, const float *In) {
    if (lpc == 4) fft_pass_a<ADJ, 4, BIG><<<grid, kThreads, smem, s>>>(d, In);
    else if (lpc == 2) fft_pass_a<ADJ, 2, BIG><<<grid, kThreads, smem, s>>>(d, In);
    else fft_pass_a<ADJ, 1, BIG><<<grid, kThreads, smem, s>>>(d, In);
}
template <bool ADJ>
void launch_a(int lpc, bool big, int grid, size_t smem, cudaStream_t s, const FftConvDev &d, const float *In) {
    if (big) launch_a2<ADJ, true>(lpc, grid, smem, s, d, In);
    else launch_a2<ADJ, false>(lpc, grid, smem, s, d, In);
}
template <bool ADJ, bool BIG>
void launch_b2(int lpc, int grid, size_t smem, cudaStream_t s, const FftConvDev &d) {
    if (lpc == 4) fft_pass_b<ADJ, 4, BIG><<<grid, kThreads, smem, s>>>(d);
    else if (lpc == 2) fft_pass_b<ADJ, 2, BIG><<<grid, kThreads, smem, s>>>(d);
    else fft_pass_b<ADJ, 1, BIG><<<grid, kThreads, smem, s>>>(d);
}
template <bool ADJ>
void launch_b(int lpc, bool big, int grid, size_t smem, cudaStream_t s, const FftConvDev &d) {
    if (big) launch_b2<ADJ, true>(lpc, grid, smem, s, d);
    else launch_b2<ADJ, false>(lpc, grid, smem, s, d);
}
template <bool ADJ, int EPI, bool BIG>
void launch_c2(int lpc, int grid, size_t smem, cudaStream_t s, const FftConvDev &d, float *Out, const ProxArgs &pa) {
    if (lpc == 4) fft_pass_c<ADJ, EPI, 4, BIG><<<grid, kThreads, smem, s>>>(d, Out, pa);
    else if (lpc == 2) fft_pass_c<ADJ, EPI, 2, BIG><<<grid, kThreads, smem, s>>>(d, Out, pa);
    else fft_pass_c<ADJ, EPI, 1, BIG><<<grid, kThreads, smem, s>>>(d, Out, pa);
}
template <bool BIG>
void launch_ca2(int lpc, int grid, size_t smem, cudaStream_t s, const FftConvDev &d, const ProxArgs &pa) {
    if (lpc == 4) fft_pass_ca<4, BIG><<<grid, kThreads, smem, s>>>(d, pa);
    else if (lpc == 2) fft_pass_ca<2, BIG><<<grid, kThreads, smem, s>>>(d, pa);
    else fft_pass_ca<1, BIG><<<grid, kThreads, smem, s>>>(d, pa);
}
template <bool ADJ, int EPI>
void launch_c(int lpc, bool big, int grid, size_t smem, cudaStream_t s, const FftConvDev &d, float *Out,
              const ProxArgs &pa) {
    if (big) launch_c2<ADJ, EPI, true>(lpc, grid, smem, s, d, Out, pa);
    else launch_c2<ADJ, EPI, false>(lpc, grid, smem, s, d, Out, pa);
}

// ------------------------------------------------------------------ host plan
// Smallest even N >= need of the form 2^a 3^b 5^c.
int smooth_len(int need) {
    long best = -1;
    for (long a = 2; a < 4L * need; a *= 2)
        for (long b = a; b < 4L * need; b *= 3)
            for (long c = b; c < 4L * need; c *= 5)
                if (c >= need && (best < 0 || c < best)) best = c;
    return (int)best;
}

// DIF stages of length N.  Long lines (N / R >= 128: a butterfly for
// every thread of a block's half) take the factors 2 as radix 16
// (in-register 4 x 4) and the factors 3 as radix 9 (3 x 3): fewer stages,
// each one pass over the line in shared memory and one block barrier.
// Otherwise, and for what remains, the factors 2 as radix 8 and 4 (a single
// 2 only when the power of two is odd and below 8, or after the 8s), then
// 3s, then 5s.  (Measured: 2160-point lines 16, 9, 3, 5 against 4, 4, 3, 3,
// 3, 5: 6 % faster per solve; 640-point lines 16, 8, 5 against 8, 4, 4, 5:
// 2 % slower, as a radix-16 stage has only 40 butterflies there.)
bool line_plan(int N, FftLine *P, std::vector<double2> *tw) {
    std::vector<int> rad;
    int r = N, n2 = 0;
    while (r % 2 == 0) {
        r /= 2;
        ++n2;
    }
    while (n2 >= 4 && N / 16 >= 128) {
        rad.push_back(16);
        n2 -= 4;
    }
    while (n2 >= 3 && n2 != 4) {
        rad.push_back(8);
        n2 -= 3;
    }
    while (n2 >= 2) {
        rad.push_back(4);
        n2 -= 2;
    }
    if (n2 == 1) rad.push_back(2);
    while (r % 9 == 0 && N / 9 >= 128) {
        rad.push_back(9);
        r /= 9;
    }
    while (r % 3 == 0) {
        rad.push_back(3);
        r /= 3;
    }
    while (r % 5 == 0) {
        rad.push_back(5);
        r /= 5;
    }
    if (r != 1 || (int)rad.size() > kFftMaxStages) return false;
    P->N = N;
    P->ns = (int)rad.size();
    tw->clear();
    int L = N;
    for (int j = 0; j < P->ns; ++j) {
        const int R = rad[j], M = L / R;
        P->R[j] = R;
        P->M[j] = M;
        P->tw[j] = (int)tw->size();
        for (int u = 1; u < R; ++u)
            for (int q = 0; q < M; ++q) {
                const double ang = -2.0 * M_PI * (double)u * q / L;
                tw->push_back(make_double2(std::cos(ang), std::sin(ang)));
            }
        L = M;
    }
    return true;
}

// pos[f]: the position at which the DIF stages leave frequency f.  Position
// p = sum_j u_j M_j (u_j the butterfly output of stage j) holds frequency
// f = sum_j u_j R_1 ... R_{j-1}.
std::vector<int> dif_positions(const FftLine &P) {
    std::vector<int> pos(P.N);
    for (int p = 0; p < P.N; ++p) {
        int rem = p, f = 0, w = 1;
        for (int j = 0; j < P.ns; ++j) {
            const int u = rem / P.M[j];
            rem -= u * P.M[j];
            f += u * w;
            w *= P.R[j];
        }
        pos[f] = p;
    }
    return pos;
}

template <typename T>
cudaError_t upload_vec(T **dst, const std::vector<T> &v) {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e) return e;
    return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Shared memory of a pass block: `lines` buffers of N + 1 values, the
// twiddle table (N - 1 values) and, for Passes A and C, the position table.
size_t pass_smem_bytes(int lines, int N, bool with_pos) {
    return sizeof(float2) * ((size_t)lines * (N + 1) + (N - 1)) + (with_pos ? sizeof(int) * N : 0);
}

// Lines per block (row pairs in Passes A and C, frequencies in Pass B): 4
// when that still gives a block per SM, else 2, else 1.  More lines per
// block share each butterfly's position arithmetic and twiddle loads and
// make longer contiguous runs in the 8-row tiles of the spectra (64 / 256
// bytes at 4 lines).  A block stays within `budget` bytes of shared memory.
int pick_lpc(long lines, int N, int sms, bool with_pos, size_t budget) {
    const int cand[3] = {4, 2, 1};
    for (int lpc : cand) {
        if (lpc > 1 && pass_smem_bytes(lpc, N, with_pos) > budget) continue;
        if (lpc == 1 || (lines + lpc - 1) / lpc >= (long)sms) return lpc;
    }
    return 1;
}

// The attribute is per kernel, not per launch: every FFT kernel is allowed
// the device's per-block maximum once, so a later, smaller plan never lowers
// an earlier one's limit.
template <typename K>
cudaError_t allow_smem(K kernel, int limit) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
}
template <int LPC, bool BIG>
cudaError_t allow_smem_lpc(int limit) {
    cudaError_t e;
    if ((e = allow_smem(fft_pass_a<false, LPC, BIG>, limit)) || (e = allow_smem(fft_pass_a<true, LPC, BIG>, limit)) ||
        (e = allow_smem(fft_pass_b<false, LPC, BIG>, limit)) || (e = allow_smem(fft_pass_b<true, LPC, BIG>, limit)) ||
        (e = allow_smem(fft_pass_c<false, EPI_STORE, LPC, BIG>, limit)) ||
        (e = allow_smem(fft_pass_c<false, EPI_RESIDUAL, LPC, BIG>, limit)) ||
        (e = allow_smem(fft_pass_c<true, EPI_STORE, LPC, BIG>, limit)) ||
        (e = allow_smem(fft_pass_c<true, EPI_PROX, LPC, BIG>, limit)) ||
        (e = allow_smem(fft_pass_ca<LPC, BIG>, limit)))
        return e;
    return cudaSuccess;
}
cudaError_t allow_smem_all(size_t sa, size_t sb, size_t sc, int limit) {
    if (sa > (size_t)limit || sb > (size_t)limit || sc > (size_t)limit) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = allow_smem_lpc<1, false>(limit)) || (e = allow_smem_lpc<2, false>(limit)) ||
        (e = allow_smem_lpc<4, false>(limit)) || (e = allow_smem_lpc<1, true>(limit)) ||
        (e = allow_smem_lpc<2, true>(limit)) || (e = allow_smem_lpc<4, true>(limit)))
        return e;
    return cudaSuccess;
}

}  // namespace

sfista_status fftconv_create(FftConv **out, const double *K, int p, int q, int cr, int cc, int m, int n, int bc) {
    *out = nullptr;
    if (p < 1 || q < 1 || p > m || q > n || cr < 0 || cr >= p || cc < 0 || cc >= q)
        return fail(SFISTA_EINVAL, "FFT form: kernel larger than the image or centre outside it");
    FftConv *f = new (std::nothrow) FftConv();
    if (!f) return fail(SFISTA_ENOMEM, "FFT form: host allocation");
    FftConvDev &d = f->d;
    d.m = m;
    d.n = n;
    d.bc = bc;
    d.offr = p - 1 - cr;
    d.offc = q - 1 - cc;
    d.ext_rows = m + p - 1;
    d.ext_cols = n + q - 1;
    const int N1 = smooth_len(d.ext_rows), N2 = smooth_len(d.ext_cols);
    if (N1 <= 0 || N2 <= 0 || N1 > kFftMaxLen || N2 > kFftMaxLen) {
        delete f;
        return fail(SFISTA_ENOTSUP, "FFT form: image plus kernel exceeds the longest transform (" +
                                        std::to_string(kFftMaxLen) + ")");
    }
    std::vector<double2> tw1, tw2;
    if (!line_plan(N1, &d.l1, &tw1) || !line_plan(N2, &d.l2, &tw2)) {
        delete f;
        return fail(SFISTA_ENOTSUP, "FFT form: no radix plan");
    }
    d.H2 = N2 / 2 + 1;
    d.sr1 = (d.ext_rows + 7) & ~7;   // rows rounded up to whole 8-row tiles
    d.sr2 = (m + 7) & ~7;
    const std::vector<int> pos1 = dif_positions(d.l1), pos2 = dif_positions(d.l2);
    // Kernel spectrum of h[s1][s2] = K[s1' + p - 1][s2' + q - 1] at s = s' mod N,
    // s' in [-(p-1), 0] x [-(q-1), 0]; scaled by 1 / (N1 N2) and stored
    // column-frequency-major with the row frequency at its DIF position:
    // Kd[f2][pos1[f1]], f2 < H2 (Pass B reads one contiguous line per f2).
    std::vector<std::complex<double>> root1(N1), root2(N2);
    for (int t = 0; t < N1; ++t) root1[t] = std::polar(1.0, -2.0 * M_PI * t / N1);
    for (int t = 0; t < N2; ++t) root2[t] = std::polar(1.0, -2.0 * M_PI * t / N2);
    const int H2 = d.H2;
    std::vector<std::complex<double>> F2((size_t)p * H2);
    for (int k = 0; k < p; ++k)
        for (int f2 = 0; f2 < H2; ++f2) {
            std::complex<double> acc = 0.0;
            for (int l = 0; l < q; ++l) {
                const long s2 = ((long)l - (q - 1) + N2) % N2;
                acc += K[(size_t)k * q + l] * root2[(size_t)((f2 * s2) % N2)];
            }
            F2[(size_t)k * H2 + f2] = acc;
        }
    std::vector<float2> Kd((size_t)N1 * H2);
    const double scale = 1.0 / ((double)N1 * N2);
    std::vector<std::complex<double>> col(p);
    for (int f1 = 0; f1 < N1; ++f1) {
        for (int k = 0; k < p; ++k) col[k] = root1[(size_t)((f1 * (((long)k - (p - 1) + N1) % N1)) % N1)];
        for (int f2 = 0; f2 < H2; ++f2) {
            std::complex<double> acc = 0.0;
            for (int k = 0; k < p; ++k) acc += F2[(size_t)k * H2 + f2] * col[k];
            acc *= scale;
            Kd[(size_t)f2 * N1 + pos1[f1]] = make_float2((float)acc.real(), (float)acc.imag());
        }
    }
    auto to_f2 = [](const std::vector<double2> &v) {
        std::vector<float2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
        return o;
    };
    cudaError_t e;
    if ((e = upload_vec((float2 **)&d.tw1, to_f2(tw1))) || (e = upload_vec((float2 **)&d.tw2, to_f2(tw2))) ||
        (e = upload_vec((int **)&d.pos2, pos2)) || (e = upload_vec((float2 **)&d.K, Kd)) ||
        (e = cudaMalloc((void **)&d.S1, sizeof(float2) * (size_t)H2 * d.sr1)) ||
        (e = cudaMalloc((void **)&d.S2, sizeof(float2) * (size_t)H2 * d.sr2)) ||
        // the padding rows (an odd row count) are read as zeros by Passes B and C
        (e = cudaMemset(d.S1, 0, sizeof(float2) * (size_t)H2 * d.sr1)) ||
        (e = cudaMemset(d.S2, 0, sizeof(float2) * (size_t)H2 * d.sr2))) {
        fftconv_destroy(f);
        return fail(SFISTA_ENOMEM, std::string("FFT form buffers: ") + cudaGetErrorString(e));
    }
    int dev = 0, sms = 152, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t budget = 110 * 1024;
    auto has_big = [](const FftLine &P) {
        for (int j = 0; j < P.ns; ++j)
            if (P.R[j] == 9 || P.R[j] == 16) return true;
        return false;
    };
    f->big1 = has_big(d.l1);
    f->big2 = has_big(d.l2);
    f->lpc_a = pick_lpc((d.ext_rows + 1) / 2, N2, sms, true, budget);
    f->lpc_b = pick_lpc(H2, N1, sms, false, budget);
    f->lpc_c = pick_lpc((m + 1) / 2, N2, sms, true, budget);
    const size_t sa = pass_smem_bytes(f->lpc_a, N2, true), sb = pass_smem_bytes(f->lpc_b, N1, false),
                 sc = pass_smem_bytes(f->lpc_c, N2, true);
    if ((e = allow_smem_all(sa, sb, sc, optin))) {
        fftconv_destroy(f);
        return fail(SFISTA_ENOTSUP, std::string("FFT form shared memory: ") + cudaGetErrorString(e));
    }
    *out = f;
    return SFISTA_OK;
}

void fftconv_destroy(FftConv *f) {
    if (!f) return;
    FftConvDev &d = f->d;
    for (void *p : {(void *)d.tw1, (void *)d.tw2, (void *)d.pos2, (void *)d.K, (void *)d.S1, (void *)d.S2})
        if (p) cudaFree(p);
    delete f;
}

void fftconv_part(const FftConv *f, int part, bool adj, const float *In, EpiKind epi, float *Out, const ProxArgs &pa,
                  cudaStream_t s) {
    const FftConvDev &d = f->d;
    if (part == 0) {
        // Pass A reads the input rows (the operator's input), Pass B the spectra.
        const int rows = adj ? d.m : d.ext_rows;
        const int ga = (int)(((rows + 1) / 2 + f->lpc_a - 1) / f->lpc_a);
        const size_t sa = pass_smem_bytes(f->lpc_a, d.l2.N, true);
        if (adj)
            launch_a<true>(f->lpc_a, f->big2, ga, sa, s, d, In);
        else
            launch_a<false>(f->lpc_a, f->big2, ga, sa, s, d, In);
        const int gb = (d.H2 + f->lpc_b - 1) / f->lpc_b;
        const size_t sb = pass_smem_bytes(f->lpc_b, d.l1.N, false);
        if (adj)
            launch_b<true>(f->lpc_b, f->big1, gb, sb, s, d);
        else
            launch_b<false>(f->lpc_b, f->big1, gb, sb, s, d);
        return;
    }
    const int gc = ((d.m + 1) / 2 + f->lpc_c - 1) / f->lpc_c;
    const size_t sc = pass_smem_bytes(f->lpc_c, d.l2.N, true);
    if (adj) {
        if (epi == EPI_PROX)
            launch_c<true, EPI_PROX>(f->lpc_c, f->big2, gc, sc, s, d, Out, pa);
        else
            launch_c<true, EPI_STORE>(f->lpc_c, f->big2, gc, sc, s, d, Out, pa);
    } else {
        if (epi == EPI_RESIDUAL)
            launch_c<false, EPI_RESIDUAL>(f->lpc_c, f->big2, gc, sc, s, d, Out, pa);
        else
            launch_c<false, EPI_STORE>(f->lpc_c, f->big2, gc, sc, s, d, Out, pa);
    }
}

void fftconv_residual_adjoint(const FftConv *f, const ProxArgs &pa, cudaStream_t s) {
    const FftConvDev &d = f->d;
    const int gc = ((d.m + 1) / 2 + f->lpc_c - 1) / f->lpc_c;
    const size_t sc = pass_smem_bytes(f->lpc_c, d.l2.N, true);
    if (f->big2) launch_ca2<true>(f->lpc_c, gc, sc, s, d, pa);
    else launch_ca2<false>(f->lpc_c, gc, sc, s, d, pa);
}

void fftconv_adjoint_columns(const FftConv *f, cudaStream_t s) {
    const FftConvDev &d = f->d;
    const int gb = (d.H2 + f->lpc_b - 1) / f->lpc_b;
    const size_t sb = pass_smem_bytes(f->lpc_b, d.l1.N, false);
    launch_b<true>(f->lpc_b, f->big1, gb, sb, s, d);
}

void fftconv_apply(const FftConv *f, bool adj, const float *In, EpiKind epi, float *Out, const ProxArgs &pa,
                   cudaStream_t s) {
    fftconv_part(f, 0, adj, In, epi, Out, pa, s);
    fftconv_part(f, 1, adj, In, epi, Out, pa, s);
}

size_t fftconv_bytes(const FftConv *f) {
    const FftConvDev &d = f->d;
    return sizeof(float2) * ((size_t)d.sr1 * d.H2 + (size_t)d.sr2 * d.H2 + (size_t)d.l1.N * d.H2);
}

}  // namespace sfista
