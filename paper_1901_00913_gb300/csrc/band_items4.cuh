// FP32 tile routines of the two-pass banded operator with 16-byte accesses, on
// RT x 32 output tiles with RT = 64 (large images) or 32 (small ones, where
// 64-row tiles would leave SMs idle); the standalone columns pass also has a
// 128-row form with two columns per thread (end of this file).  The
// standalone and grouped kernels take them when m and n are multiples of 4
// and the buffers 16-byte aligned (decided on the host, which also sizes the
// grid); otherwise the 32-row scalar routines of band_items.cuh run.  One
// block has 256 threads (8 warps).
//
// Tap padding.  Both passes step through the taps four at a time.  The rows
// pass stages its input tile from the 4-aligned column c0 + lo - off
// (off = lo mod 4), so its coefficients sit `off` taps late; both passes pad
// the tap count to a multiple of 4 with zero coefficients.  Zero taps add
// exact zeros in the loop's order, so every sum equals the unpadded one.
//
// rows item: lane l owns row a0 + l (and a0 + 32 + l when RT = 64), warp w
//            columns c0 + 4w .. c0 + 4w + 3; one broadcast 16-byte coefficient
//            load feeds 4 FMAs per row, and each row's input window advances
//            by one 16-byte load per 4 taps (row stride 4 x odd floats:
//            conflict-free).
// cols item: lane l owns column c0 + l, warp w rows a0 + (RT/8) w .. + RT/8 - 1;
//            per tap RT/32 broadcast 16-byte coefficient loads and one Z value
//            (a window of RT/8 + 4 registers refilled by 4 loads per 4 taps);
//            terms are summed in order, then the epilogue of band_items.cuh.
#pragma once

#include "band_items.cuh"

namespace sfista {
namespace band4 {

using band::NT;
using band::TC;

__host__ __device__ inline int rows_taps(int w, int off) { return (w + off + 3) & ~3; }
__host__ __device__ inline int cols_taps(int w) { return (w + 3) & ~3; }
__host__ __device__ inline int rows_span(int w4) { return 4 * (((TC + w4) / 4) | 1); }

// Shared memory in bytes for RT-row tiles (rows: for the worst column offset).
__host__ __device__ inline size_t rows_smem(int rt, int w, int nt) {
    const int w4 = rows_taps(w, 3);
    return sizeof(float) * ((size_t)rt * rows_span(w4) + (size_t)nt * w4 * TC);
}
__host__ __device__ inline size_t cols_smem(int rt, int w, int chunk) {
    const int w4 = cols_taps(w);
    return sizeof(float) * (size_t)chunk * ((size_t)(rt + w4) * TC + (size_t)w4 * rt);
}
__host__ __device__ inline int tiles(int rt, int m, int n) { return ((m + rt - 1) / rt) * ((n + TC - 1) / TC); }

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Four taps (k .. k+3) of K terms for the lane's H rows: (a0, a1), (b0, b1)
// are the rows' input windows at columns cb + k .. cb + k + 7.
template <int K, int H>
__device__ __forceinline__ void rows_taps4(const float4 &a0, const float4 &a1, const float4 &b0, const float4 &b1,
                                           const float *fk, int w4, float (&acc)[2][K][4]) {
    const float xw[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float yw[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float4 f = lds4(fk + (q * w4 + u) * TC);
            acc[0][q][0] = fmaf(xw[u], f.x, acc[0][q][0]);
            acc[0][q][1] = fmaf(xw[u + 1], f.y, acc[0][q][1]);
            acc[0][q][2] = fmaf(xw[u + 2], f.z, acc[0][q][2]);
            acc[0][q][3] = fmaf(xw[u + 3], f.w, acc[0][q][3]);
            if (H == 2) {
                acc[1][q][0] = fmaf(yw[u], f.x, acc[1][q][0]);
                acc[1][q][1] = fmaf(yw[u + 1], f.y, acc[1][q][1]);
                acc[1][q][2] = fmaf(yw[u + 2], f.z, acc[1][q][2]);
                acc[1][q][3] = fmaf(yw[u + 3], f.w, acc[1][q][3]);
            }
        }
    }
}

// K terms of the rows pass for the lane's H rows (xa: first row at column
// cb; the second, for H = 2, 32 rows below).  Two steps of 4 taps per trip,
// the windows alternating between two register sets.
template <int K, int H>
__device__ __forceinline__ void rows_terms(const float *xa, int sp, const float *fr, int w4, float *__restrict__ Z,
                                           int m, int n, int t, int ga, int c) {
    float acc[2][K][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < K; ++q) acc[h][q][0] = acc[h][q][1] = acc[h][q][2] = acc[h][q][3] = 0.f;
    const float *xb = xa + 32 * sp;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a0 = lds4(xa), b0 = H == 2 ? lds4(xb) : zero;
    int k = 0;
#pragma unroll 1
    for (; k + 8 <= w4; k += 8) {
        const float4 a1 = lds4(xa + k + 4), b1 = H == 2 ? lds4(xb + k + 4) : zero;
        rows_taps4<K, H>(a0, a1, b0, b1, fr + k * TC, w4, acc);
        a0 = lds4(xa + k + 8);
        b0 = H == 2 ? lds4(xb + k + 8) : zero;
        rows_taps4<K, H>(a1, a0, b1, b0, fr + (k + 4) * TC, w4, acc);
    }
    if (k < w4) {
        const float4 a1 = lds4(xa + k + 4), b1 = H == 2 ? lds4(xb + k + 4) : zero;
        rows_taps4<K, H>(a0, a1, b0, b1, fr + k * TC, w4, acc);
    }
    if (c < n) {   // n is a multiple of 4: the lane's 4 columns are all inside or all outside
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int row = ga + 32 * h;
            if (row >= m) break;
#pragma unroll
            for (int q = 0; q < K; ++q)
                *reinterpret_cast<float4 *>(Z + ((size_t)(t + q) * m + row) * n + c) =
                    make_float4(acc[h][q][0], acc[h][q][1], acc[h][q][2], acc[h][q][3]);
        }
    }
}

// Z_i for the terms [t0, t0 + nt) of the RT x 32 tile at (a0, c0).
template <int RT>
__device__ __forceinline__ void rows_item(const float *__restrict__ In, int m, int n, const float *__restrict__ Fb,
                                          int lo, int w, int t0, int nt, int a0, int c0, float *__restrict__ Z,
                                          float *sm) {
    constexpr int TA = RT, H = RT / 32;
    const int off = ((lo % 4) + 4) % 4, w4 = rows_taps(w, off), sp = rows_span(w4);
    float *Ins = sm;               // TA x sp
    float *Fs = sm + TA * sp;      // nt x w4 x TC
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int j = tid & 7, tr = tid >> 3;
        const int fb = c0 + 4 * j < n ? 16 : 0;
        for (int q = 0; q < nt; ++q)
            for (int kp = tr; kp < w4; kp += NT / 8) {
                const int k = kp - off;
                const bool ok = k >= 0 && k < w;
                band::stage16(Fs + (q * w4 + kp) * TC + 4 * j,
                              Fb + ((size_t)(t0 + q) * w + (ok ? k : 0)) * n + c0 + 4 * j, ok ? fb : 0, Fb);
            }
    }
    band::pdl_wait();
    {
        const int colbase = c0 + lo - off, nch = (TC + w4) >> 2;
        const int lsh = nch <= 16 ? 4 : 5;   // threads per staged row: 1 << lsh
        const int tr = tid >> lsh, tc = tid & ((1 << lsh) - 1);
        for (int e = tr; e < TA; e += NT >> lsh) {
            const int ga = a0 + e;
            for (int t = tc; t < nch; t += 1 << lsh) {
                const int gcol = colbase + 4 * t;
                const bool ok = ga < m && gcol >= 0 && gcol < n;
                band::stage16(Ins + e * sp + 4 * t, In + (size_t)(ok ? ga : 0) * n + (ok ? gcol : 0), ok ? 16 : 0,
                              In);
            }
        }
    }
    band::stage_wait<false>();
    __syncthreads();
    const int cb = warp * 4;
    const float *xa = Ins + lane * sp + cb;
    for (int tb = 0; tb < nt; tb += 4) {
        const float *fr = Fs + tb * w4 * TC + cb;
        switch (min(4, nt - tb)) {
            case 1: rows_terms<1, H>(xa, sp, fr, w4, Z, m, n, t0 + tb, a0 + lane, c0 + cb); break;
            case 2: rows_terms<2, H>(xa, sp, fr, w4, Z, m, n, t0 + tb, a0 + lane, c0 + cb); break;
            case 3: rows_terms<3, H>(xa, sp, fr, w4, Z, m, n, t0 + tb, a0 + lane, c0 + cb); break;
            default: rows_terms<4, H>(xa, sp, fr, w4, Z, m, n, t0 + tb, a0 + lane, c0 + cb); break;
        }
    }
    __syncthreads();
    band::pdl_trigger();
}

// Four taps (k .. k+3) of one term for the warp's RW rows: z holds the Z
// values of rows rb + k .. rb + k + RW + 3 in the lane's column.
template <int RW, int TA>
__device__ __forceinline__ void cols_taps4(const float (&z)[RW + 4], const float *gk, float (&a)[RW]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int h = 0; h < RW / 4; ++h) {
            const float4 g = lds4(gk + u * TA + 4 * h);
            a[4 * h + 0] = fmaf(g.x, z[u + 4 * h], a[4 * h + 0]);
            a[4 * h + 1] = fmaf(g.y, z[u + 4 * h + 1], a[4 * h + 1]);
            a[4 * h + 2] = fmaf(g.z, z[u + 4 * h + 2], a[4 * h + 2]);
            a[4 * h + 3] = fmaf(g.w, z[u + 4 * h + 3], a[4 * h + 3]);
        }
    }
}

// One term of the column pass for the warp's RW rows (4 or 8): zc is the
// staged Z at (row rb, the lane's column), gr the term's coefficients of rows
// rb .. rb + RW - 1 (row stride TA).  Two steps of 4 taps per trip: the
// second step's window is the first one's shifted by 4 rows plus 4 new
// values, so only the carry into the next trip moves registers.
template <int RW, int TA>
__device__ __forceinline__ void cols_term(const float *zc, const float *gr, int w4, float *acc) {
    float a[RW], w0[RW];
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        a[i] = 0.f;
        w0[i] = zc[i * TC];
    }
    int k = 0;
#pragma unroll 1
    for (; k + 8 <= w4; k += 8) {
        float n8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) n8[i] = zc[(k + RW + i) * TC];
        float za[RW + 4], zb[RW + 4];
#pragma unroll
        for (int i = 0; i < RW + 4; ++i) {
            za[i] = i < RW ? w0[i] : n8[i - RW];
            zb[i] = i + 4 < RW ? w0[i + 4] : n8[i + 4 - RW];
        }
        cols_taps4<RW, TA>(za, gr + k * TA, a);
        cols_taps4<RW, TA>(zb, gr + (k + 4) * TA, a);
#pragma unroll
        for (int i = 0; i < RW; ++i) w0[i] = i + 8 < RW ? w0[i + 8] : n8[i + 8 - RW];
    }
    if (k < w4) {
        float z[RW + 4];
#pragma unroll
        for (int i = 0; i < RW; ++i) z[i] = w0[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) z[RW + i] = zc[(k + RW + i) * TC];
        cols_taps4<RW, TA>(z, gr + k * TA, a);
    }
#pragma unroll
    for (int i = 0; i < RW; ++i) acc[i] += a[i];
}

// sum_i G_i Z_i over all r terms (`chunk` staged per load phase) for the
// RT x 32 tile at (a0, c0), then the epilogue.
template <int EPI, int RT>
__device__ __forceinline__ void cols_item(const float *__restrict__ Z, int m, int n, int r, int chunk,
                                          const float *__restrict__ Gb, int lo, int w, int a0, int c0,
                                          float *__restrict__ Out, const ProxArgs &pa, float *sm) {
    constexpr int TA = RT, RW = RT / 8, GC = RT / 4;   // rows per warp; 4-row chunks per coefficient row
    const int w4 = cols_taps(w), zs = TA + w4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rb = warp * RW;
    const int jz = tid & 7, trz = tid >> 3;           // Z rows: 8 chunks of 4 columns, 32 rows per pass
    const int jg = tid % GC, trg = tid / GC;          // coefficient rows: GC chunks of 4 rows, NT/GC taps per pass
    const bool cok = c0 + 4 * jz < n, rok = a0 + 4 * jg < m;
    float acc[RW];
#pragma unroll
    for (int i = 0; i < RW; ++i) acc[i] = 0.f;
    for (int t0 = 0; t0 < r; t0 += chunk) {
        const int nt = min(chunk, r - t0);
        float *Zs = sm;                    // nt x zs x TC
        float *Gs = sm + nt * zs * TC;     // nt x w4 x TA
        for (int q = 0; q < nt; ++q)
            for (int kp = trg; kp < w4; kp += NT / GC) {
                const bool ok = kp < w && rok;
                band::stage16(Gs + (q * w4 + kp) * TA + 4 * jg,
                              Gb + ((size_t)(t0 + q) * w + (kp < w ? kp : 0)) * m + a0 + 4 * jg, ok ? 16 : 0, Gb);
            }
        band::pdl_wait();
        for (int q = 0; q < nt; ++q) {
            const float *zt = Z + (size_t)(t0 + q) * m * n;
            for (int e = trz; e < zs; e += NT / 8) {
                const int ge = a0 + lo + e;
                const bool ok = cok && ge >= 0 && ge < m;
                band::stage16(Zs + (q * zs + e) * TC + 4 * jz, zt + (size_t)(ok ? ge : 0) * n + c0 + 4 * jz,
                              ok ? 16 : 0, Z);
            }
        }
        band::stage_wait<false>();
        __syncthreads();
        for (int q = 0; q < nt; ++q)
            cols_term<RW, TA>(Zs + (q * zs + rb) * TC + lane, Gs + q * w4 * TA + rb, w4, acc);
        __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < RW / 4; ++h) band::cols_epilogue<float, EPI>(acc + 4 * h, m, n, a0, rb + 4 * h, c0 + lane, Out, pa);
    band::pdl_trigger();
}

// ---------------------------------------------------------------------------
// Columns pass on 128 x 32 tiles (large images): each thread owns two
// adjacent columns and 8 rows, so one broadcast 16-byte coefficient load
// feeds 8 FMAs and one 8-byte Z load (two columns of one row) feeds the
// window of both columns.  Lane l: column pair l % 16, row group l / 16;
// warp w: rows 16 w + 8 (l / 16) .. + 7.  Taps and terms are summed in the
// same order as the 64-row routine, so both give the same result bit for bit.

__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// Four taps for the thread's 8 rows x 2 columns: z holds rows rb + k ..
// rb + k + 11 of its two columns, gk the coefficients of tap k (row stride TA).
template <int TA>
__device__ __forceinline__ void cols_taps4_2(const float2 (&z)[12], const float *gk, float (&a)[8][2]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 g = lds4(gk + u * TA + 4 * h);
            const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[4 * h + i][0] = fmaf(gv[i], z[u + 4 * h + i].x, a[4 * h + i][0]);
                a[4 * h + i][1] = fmaf(gv[i], z[u + 4 * h + i].y, a[4 * h + i][1]);
            }
        }
    }
}

// One term: zc is the staged Z at (row rb, the thread's first column), gr the
// term's coefficients of rows rb .. rb + 7 (row stride TA).
template <int TA>
__device__ __forceinline__ void cols_term2(const float *zc, const float *gr, int w4, float (&acc)[8][2]) {
    float a[8][2];
    float2 w0[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i][0] = a[i][1] = 0.f;
        w0[i] = lds2(zc + i * TC);
    }
    int k = 0;
#pragma unroll 1
    for (; k + 8 <= w4; k += 8) {
        float2 n8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) n8[i] = lds2(zc + (k + 8 + i) * TC);
        float2 za[12], zb[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            za[i] = i < 8 ? w0[i] : n8[i - 8];
            zb[i] = i < 4 ? w0[i + 4] : n8[i - 4];
        }
        cols_taps4_2<TA>(za, gr + k * TA, a);
        cols_taps4_2<TA>(zb, gr + (k + 4) * TA, a);
#pragma unroll
        for (int i = 0; i < 8; ++i) w0[i] = n8[i];
    }
    if (k < w4) {
        float2 z[12];
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = w0[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) z[8 + i] = lds2(zc + (k + 8 + i) * TC);
        cols_taps4_2<TA>(z, gr + k * TA, a);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        acc[i][0] += a[i][0];
        acc[i][1] += a[i][1];
    }
}

// sum_i G_i Z_i over all r terms (`chunk` staged per load phase) for the
// 128 x 32 tile at (a0, c0), then the epilogue on pixel pairs.
template <int EPI>
__device__ __forceinline__ void cols_item128(const float *__restrict__ Z, int m, int n, int r, int chunk,
                                             const float *__restrict__ Gb, int lo, int w, int a0, int c0,
                                             float *__restrict__ Out, const ProxArgs &pa, float *sm) {
    constexpr int TA = 128;
    const int w4 = cols_taps(w), zs = TA + w4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cp = lane & 15, rb = warp * 16 + (lane >> 4) * 8;
    const int jz = tid & 7, trz = tid >> 3;     // Z rows: 8 chunks of 4 columns, 32 rows per pass
    const int jg = tid & 31, trg = tid >> 5;    // coefficient rows: 32 chunks of 4 rows, 8 taps per pass
    const bool cok = c0 + 4 * jz < n, rok = a0 + 4 * jg < m;
    float acc[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = 0.f;
    for (int t0 = 0; t0 < r; t0 += chunk) {
        const int nt = min(chunk, r - t0);
        float *Zs = sm;                    // nt x zs x TC
        float *Gs = sm + nt * zs * TC;     // nt x w4 x TA
        for (int q = 0; q < nt; ++q)
            for (int kp = trg; kp < w4; kp += NT / 32) {
                const bool ok = kp < w && rok;
                band::stage16(Gs + (q * w4 + kp) * TA + 4 * jg,
                              Gb + ((size_t)(t0 + q) * w + (kp < w ? kp : 0)) * m + a0 + 4 * jg, ok ? 16 : 0, Gb);
            }
        band::pdl_wait();
        for (int q = 0; q < nt; ++q) {
            const float *zt = Z + (size_t)(t0 + q) * m * n;
            for (int e = trz; e < zs; e += NT / 8) {
                const int ge = a0 + lo + e;
                const bool ok = cok && ge >= 0 && ge < m;
                band::stage16(Zs + (q * zs + e) * TC + 4 * jz, zt + (size_t)(ok ? ge : 0) * n + c0 + 4 * jz,
                              ok ? 16 : 0, Z);
            }
        }
        band::stage_wait<false>();
        __syncthreads();
        for (int q = 0; q < nt; ++q)
            cols_term2<TA>(Zs + (q * zs + rb) * TC + 2 * cp, Gs + q * w4 * TA + rb, w4, acc);
        __syncthreads();
    }
    const int c = c0 + 2 * cp;
    if (c < n) {   // n is a multiple of 4: the pair is all inside or all outside
        if (EPI == EPI_PROX) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {   // four rows at a time: fewer live registers
                size_t idx[4];
                float g0[4], g1[4];
                bool ok[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ok[i] = a0 + rb + 4 * h + i < m;
                    idx[i] = (size_t)(a0 + rb + 4 * h + i) * n + c;
                    g0[i] = acc[4 * h + i][0];
                    g1[i] = acc[4 * h + i][1];
                }
                prox_momentum2_n<4>(pa, idx, g0, g1, ok);
            }
        } else {
            float2 bv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const size_t idx = (size_t)(a0 + rb + i) * n + c;
                bv[i] = EPI == EPI_RESIDUAL && a0 + rb + i < m ? __ldcg(reinterpret_cast<const float2 *>(pa.Bd + idx))
                                                               : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (a0 + rb + i >= m) break;
                const size_t idx = (size_t)(a0 + rb + i) * n + c;
                *reinterpret_cast<float2 *>(Out + idx) =
                    EPI == EPI_STORE ? make_float2(acc[i][0], acc[i][1])
                                     : make_float2(acc[i][0] - bv[i].x, acc[i][1] - bv[i].y);
            }
        }
    }
    band::pdl_trigger();
}

}  // namespace band4
}  // namespace sfista
