// One kernel per operator application of the banded FP32 operator:
//   Out[a][c] = sum_i sum_k G_i[a][a + loG + k] * Z_i[a + loG + k][c],
//   Z_i[e][c] = sum_k In[e][c + loF + k] * F_i[c][c + loF + k],
// i.e. sum_i B_i (In A_i^T) with (F, G) = (A, B), or sum_i B_i^T (In A_i) with
// (F, G) = (A^T, B^T), followed by the epilogue (store, residual, or Step 1
// shrink + Step 3 momentum).  A block computes a 32 x 32 output tile: it
// stages the input tile with its halo in both directions and all band tiles
// (cp.async, one load phase), computes the intermediate rows Z_i for the
// rows the column pass needs into shared memory, then runs the column pass.
// Z never goes to global memory and an iteration of Alg. 2 is two launches.
//
// Tap padding.  Both passes step through the taps four at a time with
// 16-byte shared loads.  The input tile is staged from the 4-aligned column
// c0 + loF - off (off = loF mod 4), so the row-pass coefficients are placed
// `off` taps late and the tap count is rounded up to a multiple of 4 with
// zero coefficients (wF4 taps); the column pass rounds wG up the same way
// (wG4).  Zero taps add exact zeros, in the same order, so every output is
// the sum the unpadded loop forms.
//
// Shared layout (floats):
//   In [rows][sp]        staged input, rows = (32 + wG4) rounded up to 32,
//                        sp = 4 * odd >= 32 + wF4
//   F  [r][wF4][32]      row-pass coefficients of this column tile
//   tF [r][wF4]          the row that interior columns share (below)
//   G  [r][wG4][32]      column-pass coefficients of this row tile
//   tG [r][wG4]          the row that interior rows share
//   Zt [r][32][zsp]      Z transposed (column-major per term), zsp = 4 * odd
// Odd multiples of four floats make the 16-byte accesses of 8 consecutive
// lanes (rows of In, columns of Zt) land in distinct banks.
//
// Row pass: lane l owns Z rows e and e + 32 of a 64-row group, warp w
// columns 4w .. 4w+3; one broadcast coefficient load feeds 8 FMAs and the
// input window advances by one 16-byte load per 4 taps and row.
// Column pass: lane l owns column l, warp w output rows 4w .. 4w+3; per 4
// taps one 16-byte Zt load (4 consecutive rows of the lane's column) and
// four broadcast coefficient loads.
// The row pass repeats the halo rows' work ((32 + wG4) / 32 times the
// two-pass count); at small and medium sizes the launch and load latency
// saved outweighs it.
//
// Interior rows.  Away from the image edges a factor is Toeplitz (Sec. 2:
// the Hankel part and the boundary only touch the first and last rows), so
// every output column of the row pass in [f0, f1), and every output row of
// the column pass in [g0, g1), has the same coefficients as one reference
// row (the host checks the FP32 values bit for bit and stores that row after
// the band table).  A warp whose four columns (rows) are all interior reads
// one 16-byte Toeplitz load per term and 4 taps instead of one per tap: the
// same coefficient values in the same order, so the result is unchanged.
//
// The same tile routines also run the whole solve in one cooperative launch
// (band_solve_fused, end of this file) when every tile has its own resident
// block, for one problem or a batch.
#include <algorithm>
#include <vector>

#include "band_items.cuh"
#include "epilogue.cuh"
#include "internal.h"

namespace sfista {
namespace {

using band::NT;
using band::TA;
using band::TC;

struct FusedGeom {
    int off;         // loF mod 4: leading zero taps of the row pass
    int wF4, wG4;    // padded tap counts (multiples of 4)
    int zs;          // Z rows the column pass reads: TA + wG4
    int th;          // output rows of a tile (a multiple of 4, <= gt; the column tile stays 32 wide)
    int gt;          // rows of the column-pass coefficient tile (32, or 64 for the 512-thread solver)
    int rows;        // staged input rows: zs rounded up to 32
    int sp, zsp;     // row strides of In and Zt
    size_t off_f, off_g, off_z, total;   // float offsets / size
};

__host__ __device__ inline FusedGeom fused_geom(int r, int loF, int wF, int wG, int th = TA, int gt = TA) {
    FusedGeom g;
    g.off = ((loF % 4) + 4) % 4;
    g.wF4 = (wF + g.off + 3) & ~3;
    g.wG4 = (wG + 3) & ~3;
    g.th = th;
    g.gt = gt;
    g.zs = th + g.wG4;
    g.rows = (g.zs + 31) & ~31;
    g.sp = 4 * (((TC + g.wF4) / 4) | 1);
    g.zsp = 4 * ((g.zs / 4) | 1);
    g.off_f = (size_t)g.rows * g.sp;
    g.off_g = g.off_f + (size_t)r * g.wF4 * (TC + 1);   // F tile, then its Toeplitz row
    g.off_z = g.off_g + (size_t)r * g.wG4 * (gt + 1);
    g.total = g.off_z + (size_t)r * TC * g.zsp;
    return g;
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Pixels (a + j, c), j = 0..3, of a thread's epilogue: linear index and bounds.
__device__ __forceinline__ void epi_index(int m, int n, int a, int c, size_t *idx, bool *ok) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ok[j] = c < n && a + j < m;
        idx[j] = (size_t)(a + j) * n + c;
    }
}

// Four taps (k .. k+3) of the row pass for K terms: (a0, a1) and (b0, b1) are
// the lanes' input windows of the two rows at columns cb + k .. cb + k + 7.
// TOEP: fk is the Toeplitz row at tap k (one coefficient for all 4 columns).
__device__ __forceinline__ float comp(const float4 &v, int t) {
    return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

template <int K, bool TWO, bool TOEP>
__device__ __forceinline__ void rows_taps4(const float4 &a0, const float4 &a1, const float4 &b0, const float4 &b1,
                                           const float *fk, int wF4, float (&acc)[TWO ? 2 : 1][K][4]) {
    const float xw[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float yw[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    float4 tq[K];
    if (TOEP) {
#pragma unroll
        for (int q = 0; q < K; ++q) tq[q] = lds4(fk + q * wF4);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            float4 f;
            if (TOEP) {
                const float v = comp(tq[q], t);
                f = make_float4(v, v, v, v);
            } else {
                f = lds4(fk + (q * wF4 + t) * TC);
            }
            acc[0][q][0] = fmaf(xw[t], f.x, acc[0][q][0]);
            acc[0][q][1] = fmaf(xw[t + 1], f.y, acc[0][q][1]);
            acc[0][q][2] = fmaf(xw[t + 2], f.z, acc[0][q][2]);
            acc[0][q][3] = fmaf(xw[t + 3], f.w, acc[0][q][3]);
            if (TWO) {
                acc[TWO ? 1 : 0][q][0] = fmaf(yw[t], f.x, acc[TWO ? 1 : 0][q][0]);
                acc[TWO ? 1 : 0][q][1] = fmaf(yw[t + 1], f.y, acc[TWO ? 1 : 0][q][1]);
                acc[TWO ? 1 : 0][q][2] = fmaf(yw[t + 2], f.z, acc[TWO ? 1 : 0][q][2]);
                acc[TWO ? 1 : 0][q][3] = fmaf(yw[t + 3], f.w, acc[TWO ? 1 : 0][q][3]);
            }
        }
    }
}

// Row pass for K terms on one (TWO: two) rows per lane.  xa: the lane's first
// input row at column cb; fr: coefficients at column cb of the first term;
// zt: Zt entry (first term, column cb, row e).  The tap loop takes two steps
// of 4 per trip so the windows alternate between two register sets.
template <int K, bool TWO, bool TOEP>
__device__ __forceinline__ void rows_pass(const float *xa, int sp, const float *fr, int wF4, float *zt, int zsp,
                                          bool sta, bool stb) {
    constexpr int ts = TOEP ? 1 : TC;   // tap stride of the coefficients
    float acc[TWO ? 2 : 1][K][4];
#pragma unroll
    for (int h = 0; h < (TWO ? 2 : 1); ++h)
#pragma unroll
        for (int q = 0; q < K; ++q) acc[h][q][0] = acc[h][q][1] = acc[h][q][2] = acc[h][q][3] = 0.f;
    const float *xb = xa + 32 * sp;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a0 = lds4(xa), b0 = TWO ? lds4(xb) : zero;
    int k = 0;
#pragma unroll 1
    for (; k + 8 <= wF4; k += 8) {
        const float4 a1 = lds4(xa + k + 4), b1 = TWO ? lds4(xb + k + 4) : zero;
        rows_taps4<K, TWO, TOEP>(a0, a1, b0, b1, fr + k * ts, wF4, acc);
        a0 = lds4(xa + k + 8);
        b0 = TWO ? lds4(xb + k + 8) : zero;
        rows_taps4<K, TWO, TOEP>(a1, a0, b1, b0, fr + (k + 4) * ts, wF4, acc);
    }
    if (k < wF4) {
        const float4 a1 = lds4(xa + k + 4), b1 = TWO ? lds4(xb + k + 4) : zero;
        rows_taps4<K, TWO, TOEP>(a0, a1, b0, b1, fr + k * ts, wF4, acc);
    }
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (sta) zt[(q * TC + j) * zsp] = acc[0][q][j];
            if (TWO && stb) zt[(q * TC + j) * zsp + 32] = acc[TWO ? 1 : 0][q][j];
        }
}

// Four taps (k .. k+3) of one term of the column pass: (w0, w1) is the Z
// window of rows rb + k .. rb + k + 7 in the lane's column.
// TOEP: gk is the Toeplitz row at tap k (one coefficient for all 4 rows).
template <bool TOEP, int GT>
__device__ __forceinline__ void cols_taps4(const float4 &w0, const float4 &w1, const float *gk, float (&a)[4]) {
    const float z[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    float4 tg;
    if (TOEP) tg = lds4(gk);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float4 g;
        if (TOEP) {
            const float v = comp(tg, t);
            g = make_float4(v, v, v, v);
        } else {
            g = lds4(gk + t * GT);
        }
        a[0] = fmaf(g.x, z[t], a[0]);
        a[1] = fmaf(g.y, z[t + 1], a[1]);
        a[2] = fmaf(g.z, z[t + 2], a[2]);
        a[3] = fmaf(g.w, z[t + 3], a[3]);
    }
}

// Column pass for K terms.  zc: Zt entry (first term, the lane's column,
// row rb); gr: coefficients of rows rb .. rb+3 of the first term.  Each
// term's chain is summed into acc at the end, terms in order.  Two steps
// of 4 taps per trip, as in the row pass.
template <int K, bool TOEP, int GT>
__device__ __forceinline__ void cols_pass(const float *zc, int zsp, const float *gr, int wG4, float *acc) {
    constexpr int ts = TOEP ? 1 : GT;   // tap stride of the coefficients
    float a[K][4];
    float4 w0[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        a[q][0] = a[q][1] = a[q][2] = a[q][3] = 0.f;
        w0[q] = lds4(zc + q * TC * zsp);
    }
    int k = 0;
#pragma unroll 1
    for (; k + 8 <= wG4; k += 8) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float *zq = zc + q * TC * zsp;
            const float4 w1 = lds4(zq + k + 4);
            cols_taps4<TOEP, GT>(w0[q], w1, gr + (q * wG4 + k) * ts, a[q]);
            w0[q] = lds4(zq + k + 8);
            cols_taps4<TOEP, GT>(w1, w0[q], gr + (q * wG4 + k + 4) * ts, a[q]);
        }
    }
    if (k < wG4) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float4 w1 = lds4(zc + q * TC * zsp + k + 4);
            cols_taps4<TOEP, GT>(w0[q], w1, gr + (q * wG4 + k) * ts, a[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
        acc[0] += a[q][0];
        acc[1] += a[q][1];
        acc[2] += a[q][2];
        acc[3] += a[q][3];
    }
}

// Loads of a thread's epilogue operands: the observed image (residual) or
// the state Y_k, X_{k-1} and beta_{k-1} (Step 1 + Step 3).
template <int EPI>
__device__ __forceinline__ void epi_load(const ProxArgs &pa, int m, int n, int a, int c, float *bv, float2 *y,
                                         float2 *xp, float2 &beta) {
    size_t idx[4];
    bool ok[4];
    epi_index(m, n, a, c, idx, ok);
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = EPI == EPI_RESIDUAL && ok[j] ? __ldcg(pa.Bd + idx[j]) : 0.f;
    if (EPI == EPI_PROX) {
        prox_load_n<4>(pa, idx, ok, y, xp);
        beta = pa.beta[pa.k - 1];
    }
}

// Band tiles of the block's output tile (a0, c0): the row-pass coefficients of
// its 32 columns and the column-pass coefficients of its 32 rows, every term.
// VEC: 16-byte copies (n, m multiples of 4, buffers 16-byte aligned);
// otherwise element-wise copies into the same layout.
// tr = (f0, f1, g0, g1): the interior ranges; a non-empty range means the
// band table is followed by its Toeplitz row (r x w values), which is then
// staged after the tile with the same tap padding.
template <bool VEC, int NTH = NT, int GT = TA>
__device__ __forceinline__ void stage_bands(const FusedGeom &geo, int r, const float *__restrict__ Fb, int wF,
                                            const float *__restrict__ Gb, int wG, int m, int n, int a0, int c0,
                                            float *Fs, float *Gs, int4 tr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tr.x < tr.y) {
        const float *tf = Fb + (size_t)r * wF * n;
        for (int i = tid; i < r * geo.wF4; i += NTH) {
            const int q = i / geo.wF4, k = i % geo.wF4 - geo.off;
            Fs[(size_t)r * geo.wF4 * TC + i] = k >= 0 && k < wF ? tf[q * wF + k] : 0.f;
        }
    }
    if (tr.z < tr.w) {
        const float *tg = Gb + (size_t)r * wG * m;
        for (int i = tid; i < r * geo.wG4; i += NTH) {
            const int q = i / geo.wG4, k = i % geo.wG4;
            Gs[(size_t)r * geo.wG4 * GT + i] = k < wG ? tg[q * wG + k] : 0.f;
        }
    }
    if (VEC) {
        // F rows: 32 columns = 8 chunks of 4; G rows: GT rows = GT / 4 chunks.
        const int tr = tid >> 3, j = tid & 7;
        constexpr int JG = GT / 4;
        const int trg = tid / JG, jg = tid % JG;
        const int fb = c0 + 4 * j < n ? 16 : 0, gb = a0 + 4 * jg < m ? 16 : 0;
        for (int q = 0; q < r; ++q) {
            for (int kp = tr; kp < geo.wF4; kp += NTH / 8) {
                const int k = kp - geo.off;
                const bool ok = k >= 0 && k < wF;
                band::stage16(Fs + (q * geo.wF4 + kp) * TC + 4 * j,
                              Fb + (size_t)(q * wF + (ok ? k : 0)) * n + c0 + 4 * j, ok ? fb : 0, Fb);
            }
            for (int kp = trg; kp < geo.wG4; kp += NTH / JG) {
                const bool ok = kp < wG;
                band::stage16(Gs + (q * geo.wG4 + kp) * GT + 4 * jg,
                              Gb + (size_t)(q * wG + (ok ? kp : 0)) * m + a0 + 4 * jg, ok ? gb : 0, Gb);
            }
        }
    } else {
        static_assert(VEC || GT == 32, "the element-wise staging covers 32-row coefficient tiles");
        const bool cin = c0 + lane < n, rin = a0 + lane < m;
        for (int q = 0; q < r; ++q) {
            for (int kp = warp; kp < geo.wF4; kp += NTH / 32) {
                const int k = kp - geo.off;
                const bool ok = k >= 0 && k < wF;
                band::stage<float, false>(Fs + (q * geo.wF4 + kp) * TC + lane,
                                          Fb + (size_t)(q * wF + (ok ? k : 0)) * n + c0 + lane, ok && cin, Fb);
            }
            for (int kp = warp; kp < geo.wG4; kp += NTH / 32) {
                const bool ok = kp < wG;
                band::stage<float, false>(Gs + (q * geo.wG4 + kp) * GT + lane,
                                          Gb + (size_t)(q * wG + (ok ? kp : 0)) * m + a0 + lane, ok && rin, Gb);
            }
        }
    }
}

// Input tile with its halo: rows e0 .. e0 + zs - 1 (the rest of the 32-row
// groups zero), columns from the 4-aligned colbase, zero outside the image.
template <bool VEC, int NTH = NT>
__device__ __forceinline__ void stage_input(const FusedGeom &geo, const float *__restrict__ In, int m, int n, int e0,
                                            int colbase, float *Ins) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int width = TC + geo.wF4;   // staged columns
    if (VEC) {
        const int nch = width >> 2;
        const int lsh = nch <= 8 ? 3 : (nch <= 16 ? 4 : 5);   // threads per staged row: 1 << lsh
        const int tr = tid >> lsh, tc = tid & ((1 << lsh) - 1);
        for (int e = tr; e < geo.rows; e += NTH >> lsh) {
            const int ge = e0 + e;
            const bool rok = e < geo.zs && ge >= 0 && ge < m;
            for (int t = tc; t < nch; t += 1 << lsh) {
                const int gcol = colbase + 4 * t;
                const bool ok = rok && gcol >= 0 && gcol < n;
                band::stage16(Ins + e * geo.sp + 4 * t, In + (size_t)(ok ? ge : 0) * n + (ok ? gcol : 0), ok ? 16 : 0,
                              In);
            }
        }
    } else {
        for (int e = warp; e < geo.rows; e += NTH / 32) {
            const int ge = e0 + e;
            const bool rok = e < geo.zs && ge >= 0 && ge < m;
            for (int s = lane; s < width; s += 32) {
                const int gcol = colbase + s;
                const bool ok = rok && gcol >= 0 && gcol < n;
                band::stage<float, false>(Ins + e * geo.sp + s, In + (size_t)(ok ? ge : 0) * n + (ok ? gcol : 0), ok,
                                          In);
            }
        }
    }
}

// Both passes on the staged tile (the caller has waited for the copies and
// synchronised): Z_i for rows [0, zs) into Zt, then the column pass added
// into acc (rows rb .. rb + 3 of the lane's column, terms summed in order).
template <bool TOEP>
__device__ __forceinline__ void rows_group(const FusedGeom &geo, int r, const float *xa, const float *fbase, int cb,
                                           float *zcol, int e, bool two) {
    for (int tb = 0; tb < r; tb += 4) {
        const float *fr = TOEP ? fbase + tb * geo.wF4 : fbase + tb * geo.wF4 * TC + cb;
        float *zt = zcol + (size_t)tb * TC * geo.zsp;
        const bool sta = e < geo.zs, stb = e + 32 < geo.zs;
        switch (min(4, r - tb) + (two ? 4 : 0)) {
            case 1: rows_pass<1, false, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            case 2: rows_pass<2, false, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            case 3: rows_pass<3, false, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            case 4: rows_pass<4, false, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            case 5: rows_pass<1, true, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            case 6: rows_pass<2, true, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            case 7: rows_pass<3, true, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
            default: rows_pass<4, true, TOEP>(xa, geo.sp, fr, geo.wF4, zt, geo.zsp, sta, stb); break;
        }
    }
}

template <bool TOEP, int GT>
__device__ __forceinline__ void cols_group(const FusedGeom &geo, int r, const float *zcol, const float *gbase, int rb,
                                           float *acc) {
    for (int tb = 0; tb < r; tb += 4) {
        const float *zc = zcol + (size_t)tb * TC * geo.zsp;
        const float *gr = TOEP ? gbase + tb * geo.wG4 : gbase + tb * geo.wG4 * GT + rb;
        switch (min(4, r - tb)) {
            case 1: cols_pass<1, TOEP, GT>(zc, geo.zsp, gr, geo.wG4, acc); break;
            case 2: cols_pass<2, TOEP, GT>(zc, geo.zsp, gr, geo.wG4, acc); break;
            case 3: cols_pass<3, TOEP, GT>(zc, geo.zsp, gr, geo.wG4, acc); break;
            default: cols_pass<4, TOEP, GT>(zc, geo.zsp, gr, geo.wG4, acc); break;
        }
    }
}

// rel = the interior ranges relative to the tile origin (columns c - c0 for
// the row pass, rows a - a0 for the column pass).
// NTH = 512 (the one-launch solver's 16-warp blocks): warps w and w + 8 take
// the same four columns in the row pass, alternate 64-row groups each; the
// column pass gives warp w output rows 4w .. 4w + 3 (up to 64 rows).
template <int NTH, int GT>
__device__ __forceinline__ void fused_passes(const FusedGeom &geo, int r, const float *Ins, const float *Fs,
                                             const float *Gs, float *Zs, float *acc, int4 rel) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cb = (warp & 7) * 4, half = NTH == 512 ? warp >> 3 : 0;
    const bool toep_f = cb >= rel.x && cb + 4 <= rel.y;   // warp-uniform
    const float *tF = Fs + (size_t)r * geo.wF4 * TC;
    for (int rbase = 64 * half; rbase < geo.zs; rbase += 64 * (NTH / 256)) {
        const int e = rbase + lane;
        const bool two = rbase + 32 < geo.zs;
        const float *xa = Ins + e * geo.sp + cb;
        float *zcol = Zs + (size_t)cb * geo.zsp + e;
        if (toep_f)
            rows_group<true>(geo, r, xa, tF, cb, zcol, e, two);
        else
            rows_group<false>(geo, r, xa, Fs, cb, zcol, e, two);
    }
    __syncthreads();
    const int rb = warp * 4;
    if (rb >= geo.th) return;   // rows beyond a shorter tile: nothing to sum
    const float *zcol = Zs + (size_t)lane * geo.zsp + rb;
    if (rb >= rel.z && rb + 4 <= rel.w)
        cols_group<true, GT>(geo, r, zcol, Gs + (size_t)r * geo.wG4 * GT, rb, acc);
    else
        cols_group<false, GT>(geo, r, zcol, Gs, rb, acc);
}

// Interior ranges (global) -> relative to the tile at (a0, c0).
__device__ __forceinline__ int4 tile_rel(int4 tr, int a0, int c0) {
    return make_int4(tr.x - c0, tr.y - c0, tr.z - a0, tr.w - a0);
}

// PRE: the epilogue's operands are loaded at the start of the block, before
// the programmatic wait, so their latency overlaps the staging and both
// passes.  None of them is written by the preceding kernel, and every kernel
// of the chain triggers its successor only after its own wait, so the kernel
// that wrote them has completed.  It holds about 30-50 more registers (two
// blocks per SM instead of three); the host takes it when every tile is
// resident at two blocks per SM.
template <int EPI, bool VEC, bool PRE>
__global__ void __launch_bounds__(NT, PRE ? 2 : 0) band_op_fused_kernel(const float *__restrict__ In, int m, int n, int r,
                                                           const float *__restrict__ Fb, int loF, int wF,
                                                           const float *__restrict__ Gb, int loG, int wG,
                                                           float *__restrict__ Out, ProxArgs pa, int4 tr) {
    extern __shared__ __align__(16) float sm[];
    const FusedGeom geo = fused_geom(r, loF, wF, wG);
    float *Ins = sm, *Fs = sm + geo.off_f, *Gs = sm + geo.off_g, *Zs = sm + geo.off_z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a0 = blockIdx.y * TA, c0 = blockIdx.x * TC;
    const int e0 = a0 + loG;                   // first staged row
    const int colbase = c0 + loF - geo.off;    // first staged column (4-aligned)
    const int rb = warp * 4, gc = c0 + lane;   // epilogue: rows a0 + rb .. + 3 of column gc
    float bv[4];
    float2 yv[4], xv[4], beta = make_float2(0.f, 0.f);
    if (PRE) epi_load<EPI>(pa, m, n, a0 + rb, gc, bv, yv, xv, beta);
    // Constant band tiles first, then (after the previous kernel) the input tile.
    stage_bands<VEC>(geo, r, Fb, wF, Gb, wG, m, n, a0, c0, Fs, Gs, tr);
    band::pdl_wait();
    stage_input<VEC>(geo, In, m, n, e0, colbase, Ins);
    band::stage_wait<false>();
    __syncthreads();
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    fused_passes<NT, TA>(geo, r, Ins, Fs, Gs, Zs, acc, tile_rel(tr, a0, c0));
    if (!PRE) epi_load<EPI>(pa, m, n, a0 + rb, gc, bv, yv, xv, beta);
    size_t idx[4];
    bool ok[4];
    epi_index(m, n, a0 + rb, gc, idx, ok);
    if (EPI == EPI_PROX) {
        prox_apply_n<4>(pa, idx, acc, ok, yv, xv, beta);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) Out[idx[j]] = EPI == EPI_STORE ? acc[j] : acc[j] - bv[j];
    }
    band::pdl_trigger();
}

// ---------------------------------------------------------------------------
// The whole solve in one cooperative launch, when every output tile has its
// own resident block (tiles <= co-resident blocks), for one problem or for a
// batch of problems of any size, PSF and rank (one block per tile of every
// problem; each block copies its problem's descriptor, a BandProb, into
// shared memory).  Tiles are th x 32 (th = P.th, a multiple of 4 up to 32,
// picked on the host); warps whose four rows lie past th sit out the column
// pass and the epilogue.  Each block keeps, for the whole solve,
//   - the band tiles of both operator applications (A, B and A^T, B^T) in
//     shared memory (staged once),
//   - the double-float state (Y_k, X_{k-1}) of its epilogue pixels in
//     registers (the epilogue's pixel -> thread map is the same in every
//     iteration),
// and per iteration runs the forward application with the residual
// epilogue and the adjoint application with Step 1 + Step 3.  Only R and
// the FP32 operand copy of Y_{k+1} go through global memory (other blocks
// read them as halo); X and Y are written once at the end.  Data that
// another block wrote in this launch is read with 16-byte cp.async.cg
// copies (L2, not the non-coherent L1).
// A grid barrier separates the phases (it orders the halo reads of R and of
// the operand copy of Y after their writes, and their next overwrite after
// the reads).  Its wait is bounded (about one second); a block that gives up
// records DEV_TIMEOUT and returns.
// The descriptor's pa.Xin / pa.Xout are the problem's state buffers 0 / 1:
// X_{k0} is read from buffer k0 & 1, X_{k0+iters} and X_{k0+iters-1} are
// written to buffers (k0+iters) & 1 and (k0+iters-1) & 1.

constexpr int kBarWords = 8;
constexpr long long kSpinCycles = 2000000000LL;   // about one second

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `nth` (1, 2, ...): every block adds one to counter
// blockIdx % kBarWords, and warp 0 polls the kBarWords counters (one lane
// each) until their sum reaches nth * gridDim.x (compared modulo 2^32).  The poll is bounded; a
// block that gives up records DEV_TIMEOUT and returns false.
// Ordering: the block barrier puts every thread's earlier writes before
// thread 0's release add, a release is cumulative over what precedes it, and
// a poller's acquire load that reads the count synchronises with the adds it
// counts; the block barrier after the poll extends that to the whole block.
__device__ bool fused_grid_sync(unsigned *bar, unsigned nth, unsigned *status, int *abort_sh) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0)
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 32 * (blockIdx.x % kBarWords))
                         : "memory");
        __syncwarp();
        const unsigned target = nth * gridDim.x;
        const long long t0 = clock64();
        for (;;) {
            const unsigned v = lane < kBarWords ? ld_acquire(bar + 32 * lane) : 0u;
            // The counters and the target wrap modulo 2^32 on long solves; the
            // sum never runs more than gridDim.x ahead of or behind the target,
            // so the signed difference orders them correctly.
            if ((int)(__reduce_add_sync(0xffffffffu, v) - target) >= 0) break;
            if (clock64() - t0 > kSpinCycles) {
                if (lane == 0) {
                    atomicOr(status, DEV_TIMEOUT);
                    *abort_sh = 1;
                }
                break;
            }
        }
    }
    __syncthreads();
    return *abort_sh == 0;
}

struct SolveLayout {
    FusedGeom gf, gt;            // forward (A, B) and adjoint (A^T, B^T) geometry
    size_t off_ff, off_gf, off_ft, off_gt, off_z, total;   // float offsets / size
};

// th <= 32: 256-thread blocks with 32-row coefficient tiles; th > 32: the
// 512-thread blocks with 64-row tiles.
__host__ __device__ inline int solve_gt(int th) { return th > TA ? 2 * TA : TA; }

__host__ __device__ inline SolveLayout solve_layout(int r, int loA, int wA, int wB, int loAT, int wAT, int wBT,
                                                    int th) {
    SolveLayout L;
    const int gt = solve_gt(th);
    L.gf = fused_geom(r, loA, wA, wB, th, gt);
    L.gt = fused_geom(r, loAT, wAT, wBT, th, gt);
    const size_t in = (size_t)max(L.gf.rows * L.gf.sp, L.gt.rows * L.gt.sp);
    L.off_ff = in;   // each table followed by its Toeplitz row
    L.off_gf = L.off_ff + (size_t)r * L.gf.wF4 * (TC + 1);
    L.off_ft = L.off_gf + (size_t)r * L.gf.wG4 * (gt + 1);
    L.off_gt = L.off_ft + (size_t)r * L.gt.wF4 * (TC + 1);
    L.off_z = L.off_gt + (size_t)r * L.gt.wG4 * (gt + 1);
    L.total = L.off_z + (size_t)r * TC * max(L.gf.zsp, L.gt.zsp);
    return L;
}

// One operator application of the one-launch solver on this block's tile;
// the geometry and shared-memory offsets come from shared memory (read
// again in every phase, so they do not hold registers across the loop).
template <int NTH, int GT>
__device__ __forceinline__ void solve_phase(const FusedGeom &g, const float *In, int m, int n, int r, int lo_rows,
                                            int lo_cols, size_t off_f, size_t off_g, size_t off_z, float *sm, int a0,
                                            int c0, float *acc, int4 tr) {
    stage_input<true, NTH>(g, In, m, n, a0 + lo_rows, c0 + lo_cols - g.off, sm);
    band::stage_wait<false>();
    __syncthreads();
    fused_passes<NTH, GT>(g, r, sm, sm + off_f, sm + off_g, sm + off_z, acc, tile_rel(tr, a0, c0));
}

// NTH = 256 threads (tiles up to 32 rows, two blocks per SM) or 512 (tiles
// of 36 to 64 rows, one block per SM: fewer halo rows per output row in the
// row pass); GT = the coefficient tile's rows (32 or 64).
template <bool BATCH, int NTH, int GT>
__global__ void __launch_bounds__(NTH, NTH == 256 ? 2 : 1)
    band_solve_fused(BandProb one, const BandProb *__restrict__ probs, const int2 *__restrict__ items, int k0,
                     int iters, unsigned *bar) {
    extern __shared__ __align__(16) float sm[];
    __shared__ BandProb P;
    __shared__ SolveLayout Ls;
    __shared__ int tile_sh, abort_sh;
    if (threadIdx.x == 0) {
        abort_sh = 0;
        if (BATCH) {
            const int2 it = items[blockIdx.x];
            P = probs[it.x];
            tile_sh = it.y;
        } else {
            P = one;
            tile_sh = blockIdx.x;
        }
        Ls = solve_layout(P.r, P.loA, P.wA, P.wB, P.loAT, P.wAT, P.wBT, P.th);
    }
    __syncthreads();
    const int m = P.m, n = P.n, r = P.r;
    const int tiles_c = (n + TC - 1) / TC;
    const int a0 = (tile_sh / tiles_c) * P.th, c0 = (tile_sh % tiles_c) * TC;
    const int mt = min(m, a0 + P.th);   // the tile's rows end here
    {
        const SolveLayout L = Ls;
        stage_bands<true, NTH, GT>(L.gf, r, P.fA, P.wA, P.fB, P.wB, m, n, a0, c0, sm + L.off_ff, sm + L.off_gf,
                                   P.tfwd);
        stage_bands<true, NTH, GT>(L.gt, r, P.fAT, P.wAT, P.fBT, P.wBT, m, n, a0, c0, sm + L.off_ft, sm + L.off_gt,
                                   P.tadj);
    }
    const int rb = (threadIdx.x >> 5) * 4, gc = c0 + (threadIdx.x & 31);   // epilogue pixels
    float2 *const Xb0 = const_cast<float2 *>(P.pa.Xin), *const Xb1 = P.pa.Xout;
    float2 y[4], xp[4];
    if (BATCH) {   // a batch starts from X_0 = X_{-1} = 0, so Y_1 = 0
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = xp[j] = make_float2(0.f, 0.f);
    } else {
        ProxArgs pa = P.pa;
        pa.Xin = (k0 & 1) ? Xb1 : Xb0;
        size_t idx[4];
        bool ok[4];
        epi_index(mt, n, a0 + rb, gc, idx, ok);
        prox_load_n<4>(pa, idx, ok, y, xp);
    }
    const int kend = k0 + iters;
    unsigned nth = 0;
    for (int k = k0 + 1; k <= kend; ++k) {
        {   // Forward operator + residual: R = A_s Y_k - B.
            size_t idx[4];
            bool ok[4];
            epi_index(mt, n, a0 + rb, gc, idx, ok);
            float bv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = ok[j] ? __ldcg(P.pa.Bd + idx[j]) : 0.f;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            // A batch's first iteration applies A_s to Y_1 = 0: every sum is
            // +0, so R = -B exactly and the passes are skipped (B is checked
            // for non-finite values here instead of by a separate kernel).
            if (BATCH && k == 1) {
                bool bad = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) bad |= ok[j] && !isfinite(bv[j]);
                if (bad) atomicOr(P.pa.status, DEV_NONFINITE);
            } else {
                solve_phase<NTH, GT>(Ls.gf, P.pa.Yop, m, n, r, P.loB, P.loA, Ls.off_ff, Ls.off_gf, Ls.off_z, sm, a0, c0,
                            acc, P.tfwd);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ok[j]) P.R[idx[j]] = acc[j] - bv[j];
        }
        if (!fused_grid_sync(bar, ++nth, P.pa.status, &abort_sh)) return;
        {   // Adjoint + Step 1 shrink + Step 3 momentum.
            const float2 beta = P.pa.beta[k - 1];
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            solve_phase<NTH, GT>(Ls.gt, P.R, m, n, r, P.loBT, P.loAT, Ls.off_ft, Ls.off_gt, Ls.off_z, sm, a0, c0, acc,
                        P.tadj);
            size_t idx[4];
            bool ok[4];
            epi_index(mt, n, a0 + rb, gc, idx, ok);
            float2 *Xlast = ((k - 1) & 1) ? Xb1 : Xb0;   // X_{k-1}: kept for a resumed solve
            bool bad = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!ok[j]) continue;
                float2 x;
                const float2 yn = prox_step(P.pa, y[j], xp[j], acc[j], beta, &x, &bad);
                store_operands(P.pa, idx[j], yn);
                if (!BATCH && k == kend) Xlast[idx[j]] = xp[j];
                xp[j] = x;
                y[j] = yn;
            }
            if (bad) atomicOr(P.pa.status, DEV_NONFINITE);
        }
        if (!fused_grid_sync(bar, ++nth, P.pa.status, &abort_sh)) return;
    }
    size_t idx[4];
    bool ok[4];
    epi_index(mt, n, a0 + rb, gc, idx, ok);
    if (BATCH) {   // the FP32 result, straight into the caller's output
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) P.xout[idx[j]] = dfp::to_float(xp[j]);
        return;
    }
    float2 *Xout = (kend & 1) ? Xb1 : Xb0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (ok[j]) {
            Xout[idx[j]] = xp[j];
            P.pa.Y[idx[j]] = y[j];
        }
}

constexpr size_t kFusedSmemMax = 227 * 1024;

template <int EPI>
void launch_epi(const cudaLaunchConfig_t &cfg, bool vec, bool pre, const float *In, int m, int n, int r,
                const float *Fb, int loF, int wF, const float *Gb, int loG, int wG, float *Out, const ProxArgs &pa,
                int4 tr) {
    if constexpr (EPI != EPI_STORE) {
        if (vec && pre)
            return (void)cudaLaunchKernelEx(&cfg, band_op_fused_kernel<EPI, true, true>, In, m, n, r, Fb, loF, wF, Gb,
                                            loG, wG, Out, pa, tr);
    }
    if (vec)
        cudaLaunchKernelEx(&cfg, band_op_fused_kernel<EPI, true, false>, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out,
                           pa, tr);
    else
        cudaLaunchKernelEx(&cfg, band_op_fused_kernel<EPI, false, false>, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out,
                           pa, tr);
}

int fused_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    }
    return sms;
}

}  // namespace

// Largest shared-memory size over the four possible column offsets.
size_t band_op_fused_smem(int r, int wF, int wG) { return sizeof(float) * fused_geom(r, 3, wF, wG).total; }

// Sets the kernels' shared-memory limit; false if one tile does not fit.
bool band_op_fused_prepare(int r, int wF, int wG) {
    const size_t sm = band_op_fused_smem(r, wF, wG);
    if (sm > kFusedSmemMax) return false;
    for (auto k : {band_op_fused_kernel<EPI_STORE, true, false>, band_op_fused_kernel<EPI_RESIDUAL, true, false>,
                   band_op_fused_kernel<EPI_PROX, true, false>, band_op_fused_kernel<EPI_RESIDUAL, true, true>,
                   band_op_fused_kernel<EPI_PROX, true, true>, band_op_fused_kernel<EPI_STORE, false, false>,
                   band_op_fused_kernel<EPI_RESIDUAL, false, false>, band_op_fused_kernel<EPI_PROX, false, false>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax) != cudaSuccess)
            return false;
    return true;
}

void launch_band_op_fused(const float *In, int m, int n, int r, const float *Fb, int loF, int wF, const float *Gb,
                          int loG, int wG, EpiKind epi, float *Out, const ProxArgs &pa, int4 tr, cudaStream_t s) {
    const bool vec = (n % 4) == 0 && (m % 4) == 0 && ((uintptr_t)In % 16) == 0 && ((uintptr_t)Fb % 16) == 0 &&
                     ((uintptr_t)Gb % 16) == 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((n + TC - 1) / TC, (m + TA - 1) / TA);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sizeof(float) * fused_geom(r, loF, wF, wG).total;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool pre = (long)cfg.gridDim.x * cfg.gridDim.y <= 2L * fused_sm_count();
    if (epi == EPI_STORE)
        launch_epi<EPI_STORE>(cfg, vec, pre, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out, pa, tr);
    else if (epi == EPI_RESIDUAL)
        launch_epi<EPI_RESIDUAL>(cfg, vec, pre, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out, pa, tr);
    else
        launch_epi<EPI_PROX>(cfg, vec, pre, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out, pa, tr);
}

namespace {

// The most dynamic shared memory a block of `kernel` may take: the device's
// opt-in maximum less the kernel's static shared memory.
int max_dynamic_smem(const void *kernel, int dev) {
    cudaFuncAttributes fa{};
    int optin = 0;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return optin - (int)fa.sharedSizeBytes;
}

// The solver instance for tiles th rows high: 256 threads up to 32 rows,
// 512 threads (single problems) above.
template <bool BATCH>
const void *solver_kernel(int th) {
    if (!BATCH && th > TA) return (const void *)band_solve_fused<false, 512, 2 * TA>;
    return (const void *)band_solve_fused<BATCH, NT, TA>;
}
inline int solver_threads(int th) { return th > TA ? 512 : NT; }

// Shared memory and co-residency of the one-launch solver over `np`
// problems with tiles `th` rows high; false when a tile does not fit, the
// 16-byte path does not apply or the tiles outnumber the co-resident blocks.
template <bool BATCH>
bool solve_fused_fits(const BandProb *probs, int np, int dev, int th, long *tiles, size_t *smem, int *sms) {
    if (BATCH && th > TA) return false;
    const void *kernel = solver_kernel<BATCH>(th);
    *tiles = 0;
    *smem = 0;
    for (int p = 0; p < np; ++p) {
        const BandProb &P = probs[p];
        if (P.m % 4 || P.n % 4) return false;
        *smem = std::max(*smem, sizeof(float) * solve_layout(P.r, P.loA, P.wA, P.wB, P.loAT, P.wAT, P.wBT, th).total);
        *tiles += (long)((P.m + th - 1) / th) * ((P.n + TC - 1) / TC);
    }
    // The attribute is per kernel, not per launch: allow the largest size, so
    // that a later, smaller configuration never lowers an earlier one's limit.
    const int lim = max_dynamic_smem(kernel, dev);
    if (*smem > (size_t)lim) return false;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) return false;
    int per_sm = 0, coop = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, solver_threads(th), *smem) != cudaSuccess ||
        cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
        return false;
    return coop && per_sm >= 1 && *tiles <= (long)per_sm * *sms;
}

// Tile height of the one-launch solver: the candidate (64, 60, ..., 36 rows
// on 512-thread blocks for single problems; 32, 28, ..., 16 on 256-thread
// blocks) whose busiest SM has the least pass work, counted as
//   ceil(tiles / SMs) * W + 0.01 * W * tiles,  W = lane_rows(th + wG4) * wF4 + th * wG4
// where the row pass covers th + wG4 staged rows in groups of 64 (two rows
// per lane; a last group of at most 32 rows takes one) and the column pass
// th rows, both 32 columns wide (widest bands of the problems).  Shorter
// tiles spread a problem over more SMs (at 512^2, 28-row tiles put two
// blocks on every SM instead of two on 104 and one on 48).  Ties keep the
// taller tile.  Taller tiles repeat fewer halo rows in the row pass (at
// 512^2, 60-row tiles on 144 blocks: 1.34 executed per algorithmic flop
// against 1.70 for 28-row tiles).  false when no candidate fits.
template <bool BATCH>
bool solve_fused_pick(const BandProb *probs, int np, int dev, int *th, long *tiles, size_t *smem) {
    int wF4 = 0, wG4 = 0;
    for (int p = 0; p < np; ++p) {
        const BandProb &P = probs[p];
        const FusedGeom gf = fused_geom(P.r, P.loA, P.wA, P.wB), gt = fused_geom(P.r, P.loAT, P.wAT, P.wBT);
        wF4 = std::max(wF4, std::max(gf.wF4, gt.wF4));
        wG4 = std::max(wG4, std::max(gf.wG4, gt.wG4));
    }
    double best = -1.0;
    for (int t = BATCH ? TA : 2 * TA; t >= 16; t -= 4) {
        long nt = 0;
        size_t sm = 0;
        int sms = 1;
        if (!solve_fused_fits<BATCH>(probs, np, dev, t, &nt, &sm, &sms)) continue;
        const int zs = t + wG4, rest = zs % 64;
        const int lane_rows = 64 * (zs / 64) + (rest == 0 ? 0 : (rest <= 32 ? 32 : 64));
        const double work = (double)lane_rows * wF4 + (double)t * wG4;
        // plus a fixed cost per block (its staging and its arrivals at the grid
        // barrier) of 1 % of a tile's work: among candidates of nearly equal
        // work the one with fewer blocks wins (measured at 512^2: 64-row tiles
        // on 128 blocks 14.4 us per iteration, 60-row tiles on 144 blocks 15.0 us)
        const double cost = (double)((nt + sms - 1) / sms) * work + 0.01 * work * (double)nt;
        if (best < 0.0 || cost < best) {
            best = cost;
            *th = t;
            *tiles = nt;
            *smem = sm;
        }
    }
    return best >= 0.0;
}

}  // namespace

bool band_solve_fused_config(const BandProb &prob, int dev, int *grid, size_t *smem, int *th) {
    long tiles = 0;
    if (!solve_fused_pick<false>(&prob, 1, dev, th, &tiles, smem)) return false;
    *grid = (int)tiles;
    return true;
}

bool band_solve_fused_config_th(const BandProb &prob, int dev, int th, int *grid, size_t *smem) {
    if (th < 16 || th > 2 * TA || th % 4) return false;
    long tiles = 0;
    int sms = 0;
    if (!solve_fused_fits<false>(&prob, 1, dev, th, &tiles, smem, &sms)) return false;
    *grid = (int)tiles;
    return true;
}

cudaError_t launch_band_solve_fused(int grid, size_t smem, const BandProb &prob, int k0, int iters, unsigned *bar,
                                    cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, kBarrierBytes, s);
    if (e) return e;
    BandProb one = prob;
    const BandProb *probs = nullptr;
    const int2 *items = nullptr;
    void *args[] = {&one, &probs, &items, &k0, &iters, &bar};
    return cudaLaunchCooperativeKernel(solver_kernel<false>(prob.th), dim3(grid), dim3(solver_threads(prob.th)), args,
                                       smem, s);
}

bool band_solve_fused_batch_config(const BandProb *probs, int np, int dev, std::vector<int2> *items, size_t *smem,
                                   int *th) {
    long tiles = 0;
    if (!solve_fused_pick<true>(probs, np, dev, th, &tiles, smem)) return false;
    items->clear();
    for (int p = 0; p < np; ++p) {
        const int t = ((probs[p].m + *th - 1) / *th) * ((probs[p].n + TC - 1) / TC);
        for (int i = 0; i < t; ++i) items->push_back(make_int2(p, i));
    }
    return true;
}

cudaError_t launch_band_solve_fused_batch(int nitems, size_t smem, const BandProb *d_probs, const int2 *d_items,
                                          int iters, unsigned *bar, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, kBarrierBytes, s);
    if (e) return e;
    BandProb one{};
    int k0 = 0;
    void *args[] = {&one, &d_probs, &d_items, &k0, &iters, &bar};
    return cudaLaunchCooperativeKernel(solver_kernel<true>(TA), dim3(nitems), dim3(NT), args, smem, s);
}

}  // namespace sfista
