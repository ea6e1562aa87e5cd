// Tile routines of the banded operator, shared by the standalone, grouped and
// persistent kernels.  One block (256 threads, 8 warps) computes a 32 x 32
// output tile.
//
// rows item:  Z_i[a][c] = sum_k In[a][c + lo + k] * F_i[c][c + lo + k]  for the
//             terms i in [t0, t0 + nt).  Lane l owns image row a0 + l, warp w
//             owns columns c0 + 4w .. c0 + 4w + 3: per k it needs the four band
//             entries F_i[c..c+3][k] (one broadcast 16-byte load) and one new
//             input value (a four-register window slides along the row).
// cols item:  acc[a][c] = sum_i sum_k G_i[a][a + lo + k] * Z_i[a + lo + k][c]
//             over all r terms (staged `chunk` terms per load phase).  Lane l
//             owns column c0 + l, warp w rows a0 + 4w .. a0 + 4w + 3: per k one
//             broadcast load of G_i[a..a+3][k] and one new Z value (window
//             slides down the column); then the epilogue (plain store,
//             residual, or shrink + momentum), row-contiguous across lanes.
// Band entries come from compact storage band[(i*w + k)*len + row].  Shared
// tiles use odd row strides (conflict-free); all loads of a phase are
// independent and issued back to back.  CG selects ld.global.cg for data
// written earlier in the same launch (persistent kernel).
#pragma once

#include "epilogue.cuh"

namespace sfista {
namespace band {

constexpr int NT = 256;   // threads per block
constexpr int TC = 32;    // output columns per tile
constexpr int TA = 32;    // output rows per tile

// Padded, odd row length of the rows-pass input tile (one spare column for
// the window's look-ahead read).
__host__ __device__ inline int rows_span(int w) { return (TC + w) | 1; }

// FP32 vector paths: taps padded to a multiple of 4 (the rows pass also
// shifts them by up to 3 so the input tile starts on a 4-aligned column).
__host__ __device__ inline int rows_taps4(int w, int off) { return (w + off + 3) & ~3; }
__host__ __device__ inline int cols_taps4(int w) { return (w + 3) & ~3; }
__host__ __device__ inline int rows_span4(int w4) { return 4 * (((TC + w4) / 4) | 1); }

template <typename T>
__host__ __device__ inline size_t rows_smem(int w, int nt) {
    if (sizeof(T) == 4) {   // the larger of the vector layout (worst offset) and the scalar one
        const int w4 = rows_taps4(w, 3);
        return sizeof(T) * ((size_t)TA * rows_span4(w4) + (size_t)nt * w4 * TC);
    }
    return sizeof(T) * ((size_t)TA * rows_span(w) + (size_t)nt * w * TC);
}
// Per staged term: (TA + w) x TC values of Z (one spare row) and w x TA band
// entries; w padded to cols_taps4(w) for FP32.
template <typename T>
__host__ __device__ inline size_t cols_smem(int w, int chunk) {
    if (sizeof(T) == 4) w = cols_taps4(w);
    return sizeof(T) * (size_t)chunk * ((size_t)(TA + w) * TC + (size_t)w * TA);
}

// Stage one element global -> shared.  Plain kernels use cp.async (no
// register round trip, so every copy of a load phase is in flight at once;
// src-size 0 zero-fills); the persistent kernel reads through L2 (ld.cg)
// because other blocks wrote the data earlier in the same launch.
template <typename T, bool CG>
__device__ __forceinline__ void stage(T *dst, const T *src, bool pred, const T *safe) {
    if (CG) {
        *dst = pred ? __ldcg(src) : T(0);
    } else {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(pred ? src : safe),
                     "n"((int)sizeof(T)), "r"(pred ? (int)sizeof(T) : 0)
                     : "memory");
    }
}
// Programmatic dependent launch: wait for the preceding kernel in the stream
// (its writes become visible), and let the next one start its prologue.
// Both are no-ops when the kernel was not launched with the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 16-byte global -> shared copy of `bytes` (0..16) bytes, zero-filling the
// rest; dst and src must be 16-byte aligned (src unused when bytes == 0).
__device__ __forceinline__ void stage16(float *dst, const float *src, int bytes, const float *safe) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(bytes > 0 ? src : safe), "r"(bytes)
                 : "memory");
}

template <bool CG>
__device__ __forceinline__ void stage_wait() {
    if (!CG) asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void load4(const T *p, T &a, T &b, T &c, T &d) {
    a = p[0];
    b = p[1];
    c = p[2];
    d = p[3];
}
template <>
__device__ __forceinline__ void load4<float>(const float *p, float &a, float &b, float &c, float &d) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x;
    b = v.y;
    c = v.z;
    d = v.w;
}

// K terms at once: the input window is shared by every term, so one new
// input value feeds 4 K FMAs per step; the K accumulator chains are independent.
template <typename T, int K>
__device__ __forceinline__ void rows_terms(const T *xr, const T *fr, int w, T *__restrict__ Z, int m, int n, int t,
                                           int ga, int c) {
    T acc[K][4];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = T(0);
    T x0 = xr[0], x1 = xr[1], x2 = xr[2], x3 = xr[3];
#pragma unroll 2
    for (int k = 0; k < w; ++k) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            T f0, f1, f2, f3;
            load4<T>(fr + (q * w + k) * TC, f0, f1, f2, f3);
            acc[q][0] = fma(x0, f0, acc[q][0]);
            acc[q][1] = fma(x1, f1, acc[q][1]);
            acc[q][2] = fma(x2, f2, acc[q][2]);
            acc[q][3] = fma(x3, f3, acc[q][3]);
        }
        x0 = x1;
        x1 = x2;
        x2 = x3;
        x3 = xr[k + 4];
    }
    if (ga < m) {
        const int rem = n - c;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            T *zr = Z + ((size_t)(t + q) * m + ga) * n + c;
            if (rem > 0) zr[0] = acc[q][0];
            if (rem > 1) zr[1] = acc[q][1];
            if (rem > 2) zr[2] = acc[q][2];
            if (rem > 3) zr[3] = acc[q][3];
        }
    }
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// FP32 rows pass with 16-byte accesses: the input window advances by one
// 16-byte load per 4 taps; each lane stores its 4 outputs as one float4.
template <int K>
__device__ __forceinline__ void rows_terms4(const float *xr, const float *fr, int w4, float *__restrict__ Z, int m,
                                            int n, int t, int ga, int c) {
    float acc[K][4];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    float4 x0 = lds4(xr);
#pragma unroll 1
    for (int k = 0; k < w4; k += 4) {
        const float4 x1 = lds4(xr + k + 4);
        const float xw[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const float4 f = lds4(fr + (q * w4 + k + u) * TC);
                acc[q][0] = fmaf(xw[u], f.x, acc[q][0]);
                acc[q][1] = fmaf(xw[u + 1], f.y, acc[q][1]);
                acc[q][2] = fmaf(xw[u + 2], f.z, acc[q][2]);
                acc[q][3] = fmaf(xw[u + 3], f.w, acc[q][3]);
            }
        }
        x0 = x1;
    }
    if (ga < m && c < n) {
#pragma unroll
        for (int q = 0; q < K; ++q)
            *reinterpret_cast<float4 *>(Z + ((size_t)(t + q) * m + ga) * n + c) =
                make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
    }
}

// Rows item, FP32 with n a multiple of 4 and 16-byte aligned buffers.  The
// input tile is staged from the 4-aligned column c0 + lo - off (off = lo mod
// 4) and the coefficients `off` taps late, padded with zero taps to w4 (zero
// taps add exact zeros in the loop's order, so the sums equal the scalar
// path's).
__device__ __forceinline__ void rows_item4(const float *__restrict__ In, int m, int n, const float *__restrict__ Fb,
                                           int lo, int w, int t0, int nt, int a0, int c0, float *__restrict__ Z,
                                           float *sm) {
    const int off = ((lo % 4) + 4) % 4, w4 = rows_taps4(w, off), sp = rows_span4(w4);
    float *Ins = sm;                 // TA x sp
    float *Fs = sm + TA * sp;        // nt x w4 x TC
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int j = tid & 7, tr = tid >> 3;
        const int fb = c0 + 4 * j < n ? 16 : 0;
        for (int q = 0; q < nt; ++q)
            for (int kp = tr; kp < w4; kp += NT / 8) {
                const int k = kp - off;
                const bool ok = k >= 0 && k < w;
                stage16(Fs + (q * w4 + kp) * TC + 4 * j, Fb + ((size_t)(t0 + q) * w + (ok ? k : 0)) * n + c0 + 4 * j,
                        ok ? fb : 0, Fb);
            }
    }
    pdl_wait();
    {
        const int colbase = c0 + lo - off, nch = (TC + w4) >> 2;
        const int lsh = nch <= 16 ? 4 : 5;   // threads per staged row: 1 << lsh
        const int tr = tid >> lsh, tc = tid & ((1 << lsh) - 1);
        for (int e = tr; e < TA; e += NT >> lsh) {
            const int ga = a0 + e;
            for (int t = tc; t < nch; t += 1 << lsh) {
                const int gcol = colbase + 4 * t;
                const bool ok = ga < m && gcol >= 0 && gcol < n;
                stage16(Ins + e * sp + 4 * t, In + (size_t)(ok ? ga : 0) * n + (ok ? gcol : 0), ok ? 16 : 0, In);
            }
        }
    }
    stage_wait<false>();
    __syncthreads();
    const int cb = warp * 4, ga = a0 + lane;
    const float *xr = Ins + lane * sp + cb;
    for (int tb = 0; tb < nt; tb += 4) {
        const float *fr = Fs + tb * w4 * TC + cb;
        switch (min(4, nt - tb)) {
            case 1: rows_terms4<1>(xr, fr, w4, Z, m, n, t0 + tb, ga, c0 + cb); break;
            case 2: rows_terms4<2>(xr, fr, w4, Z, m, n, t0 + tb, ga, c0 + cb); break;
            case 3: rows_terms4<3>(xr, fr, w4, Z, m, n, t0 + tb, ga, c0 + cb); break;
            default: rows_terms4<4>(xr, fr, w4, Z, m, n, t0 + tb, ga, c0 + cb); break;
        }
    }
    __syncthreads();
    pdl_trigger();
}

template <typename T, bool CG>
__device__ __forceinline__ void rows_item(const T *__restrict__ In, int m, int n, const T *__restrict__ Fb, int lo,
                                          int w, int t0, int nt, int a0, int c0, T *__restrict__ Z, T *sm) {
    if constexpr (sizeof(T) == 4 && !CG) {
        if ((n & 3) == 0 && aligned16(In) && aligned16(Fb) && aligned16(Z)) {
            rows_item4(In, m, n, Fb, lo, w, t0, nt, a0, c0, Z, sm);
            return;
        }
    }
    const int span = TC + w - 1, sp = rows_span(w);
    T *Ins = sm;                 // TA x sp (columns >= span are zero)
    T *Fs = sm + TA * sp;        // nt x w x TC
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool cin = c0 + lane < n;
    for (int tk = warp; tk < nt * w; tk += NT / 32)   // band tables: constant, staged before the wait
        stage<T, false>(Fs + tk * TC + lane, Fb + ((size_t)t0 * w + tk) * n + c0 + lane, cin, Fb);
    if (!CG) pdl_wait();
    {
        const int row = tid >> 3, j0 = tid & 7;          // 32 rows x 8 threads
        const int ga = a0 + row;
        for (int col = j0; col < sp; col += 8) {
            const int gc = c0 + lo + col;
            stage<T, CG>(Ins + row * sp + col, In + (size_t)ga * n + gc, col < span && ga < m && gc >= 0 && gc < n,
                         In);
        }
    }
    stage_wait<false>();
    __syncthreads();
    const int cb = warp * 4;
    const int ga = a0 + lane;
    const T *xr = Ins + lane * sp + cb;
    for (int tb = 0; tb < nt; tb += 4) {
        switch (min(4, nt - tb)) {
            case 1: rows_terms<T, 1>(xr, Fs + tb * w * TC + cb, w, Z, m, n, t0 + tb, ga, c0 + cb); break;
            case 2: rows_terms<T, 2>(xr, Fs + tb * w * TC + cb, w, Z, m, n, t0 + tb, ga, c0 + cb); break;
            case 3: rows_terms<T, 3>(xr, Fs + tb * w * TC + cb, w, Z, m, n, t0 + tb, ga, c0 + cb); break;
            default: rows_terms<T, 4>(xr, Fs + tb * w * TC + cb, w, Z, m, n, t0 + tb, ga, c0 + cb); break;
        }
    }
    __syncthreads();
    if (!CG) pdl_trigger();
}

// K terms at once, each with its own Z window and accumulator chain; the
// chains are summed into acc at the end (term order is kept).
template <typename T, int K>
__device__ __forceinline__ void cols_terms(const T *zc, const T *gr, int w, int zs, T *acc) {
    T a[K][4], z[K][4];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        a[q][0] = a[q][1] = a[q][2] = a[q][3] = T(0);
        const T *zq = zc + q * zs * TC;
        z[q][0] = zq[0];
        z[q][1] = zq[TC];
        z[q][2] = zq[2 * TC];
        z[q][3] = zq[3 * TC];
    }
#pragma unroll 2
    for (int k = 0; k < w; ++k) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            T g0, g1, g2, g3;
            load4<T>(gr + (q * w + k) * TA, g0, g1, g2, g3);
            a[q][0] = fma(g0, z[q][0], a[q][0]);
            a[q][1] = fma(g1, z[q][1], a[q][1]);
            a[q][2] = fma(g2, z[q][2], a[q][2]);
            a[q][3] = fma(g3, z[q][3], a[q][3]);
            z[q][0] = z[q][1];
            z[q][1] = z[q][2];
            z[q][2] = z[q][3];
            z[q][3] = zc[(q * zs + k + 4) * TC];
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

// FP32 column pass over padded taps (w4, a multiple of 4): the Z window
// holds 8 rows, refilled by 4 loads per 4 taps; zero taps at the end add
// exact zeros.
template <int K>
__device__ __forceinline__ void cols_terms4(const float *zc, const float *gr, int w4, int zs, float *acc) {
    float a[K][4], w0[K][4];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        a[q][0] = a[q][1] = a[q][2] = a[q][3] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) w0[q][i] = zc[(q * zs + i) * TC];
    }
#pragma unroll 1
    for (int k = 0; k < w4; k += 4) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            float z[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                z[i] = w0[q][i];
                z[4 + i] = zc[(q * zs + k + 4 + i) * TC];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 g = lds4(gr + (q * w4 + k + u) * TA);
                a[q][0] = fmaf(g.x, z[u], a[q][0]);
                a[q][1] = fmaf(g.y, z[u + 1], a[q][1]);
                a[q][2] = fmaf(g.z, z[u + 2], a[q][2]);
                a[q][3] = fmaf(g.w, z[u + 3], a[q][3]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) w0[q][i] = z[4 + i];
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

// Epilogue of a cols item: lane column c0 + lane, rows a0 + rb .. + 3.
template <typename T, int EPI>
__device__ __forceinline__ void cols_epilogue(const T *acc, int m, int n, int a0, int rb, int gc, T *__restrict__ Out,
                                              const ProxArgs &pa) {
    if (gc >= n) return;
    if (EPI == EPI_PROX) {
        size_t idx[4];
        float g[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ok[j] = a0 + rb + j < m;
            idx[j] = (size_t)(a0 + rb + j) * n + gc;
            g[j] = (float)acc[j];
        }
        prox_momentum_n<4>(pa, idx, g, ok);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ga = a0 + rb + j;
            if (ga >= m) break;
            const size_t idx = (size_t)ga * n + gc;
            if (EPI == EPI_STORE) Out[idx] = acc[j];
            else Out[idx] = acc[j] - (T)pa.Bd[idx];
        }
    }
}

// Cols item, FP32 with m, n multiples of 4 and 16-byte aligned buffers: Z rows
// and band tiles staged with 16-byte copies, taps padded to w4 with zeros.
template <int EPI>
__device__ __forceinline__ void cols_item4(const float *__restrict__ Z, int m, int n, int r, int chunk,
                                           const float *__restrict__ Gb, int lo, int w, int a0, int c0,
                                           float *__restrict__ Out, const ProxArgs &pa, float *sm) {
    const int w4 = cols_taps4(w), zs = TA + w4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = tid & 7, tr = tid >> 3;
    const int rb = warp * 4;
    const bool cok = c0 + 4 * j < n, rok = a0 + 4 * j < m;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t0 = 0; t0 < r; t0 += chunk) {
        const int nt = min(chunk, r - t0);
        float *Zs = sm;                      // nt x zs x TC
        float *Gs = sm + nt * zs * TC;       // nt x w4 x TA
        for (int q = 0; q < nt; ++q)
            for (int kp = tr; kp < w4; kp += NT / 8) {
                const bool ok = kp < w && rok;
                stage16(Gs + (q * w4 + kp) * TA + 4 * j, Gb + ((size_t)(t0 + q) * w + (kp < w ? kp : 0)) * m + a0 + 4 * j,
                        ok ? 16 : 0, Gb);
            }
        pdl_wait();
        for (int q = 0; q < nt; ++q) {
            const float *zt = Z + (size_t)(t0 + q) * m * n;
            for (int e = tr; e < zs; e += NT / 8) {
                const int ge = a0 + lo + e;
                const bool ok = cok && ge >= 0 && ge < m;
                stage16(Zs + (q * zs + e) * TC + 4 * j, zt + (size_t)(ok ? ge : 0) * n + c0 + 4 * j, ok ? 16 : 0, Z);
            }
        }
        stage_wait<false>();
        __syncthreads();
        for (int tb = 0; tb < nt; tb += 4) {
            const float *zc = Zs + (tb * zs + rb) * TC + lane;
            const float *gr = Gs + tb * w4 * TA + rb;
            switch (min(4, nt - tb)) {
                case 1: cols_terms4<1>(zc, gr, w4, zs, acc); break;
                case 2: cols_terms4<2>(zc, gr, w4, zs, acc); break;
                case 3: cols_terms4<3>(zc, gr, w4, zs, acc); break;
                default: cols_terms4<4>(zc, gr, w4, zs, acc); break;
            }
        }
        __syncthreads();
    }
    cols_epilogue<float, EPI>(acc, m, n, a0, rb, c0 + lane, Out, pa);
    pdl_trigger();
}

template <typename T, int EPI, bool CG>
__device__ __forceinline__ void cols_item(const T *__restrict__ Z, int m, int n, int r, int chunk,
                                          const T *__restrict__ Gb, int lo, int w, int a0, int c0, T *__restrict__ Out,
                                          const ProxArgs &pa, T *sm) {
    if constexpr (sizeof(T) == 4 && !CG) {
        if ((n & 3) == 0 && (m & 3) == 0 && aligned16(Z) && aligned16(Gb)) {
            cols_item4<EPI>(Z, m, n, r, chunk, Gb, lo, w, a0, c0, Out, pa, sm);
            return;
        }
    }
    const int span = TA + w - 1, zs = TA + w;   // one spare (zero) row for the window's look-ahead
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gc = c0 + lane;
    const bool cin = gc < n;
    const int rb = warp * 4;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int t0 = 0; t0 < r; t0 += chunk) {
        const int nt = min(chunk, r - t0);
        T *Zs = sm;                        // nt x zs x TC
        T *Gs = sm + nt * zs * TC;         // nt x w x TA
        const bool rin = a0 + lane < m;
        for (int tk = warp; tk < nt * w; tk += NT / 32)   // band tables: constant, staged before the wait
            stage<T, false>(Gs + tk * TA + lane, Gb + ((size_t)t0 * w + tk) * m + a0 + lane, rin, Gb);
        if (!CG) pdl_wait();
        for (int t = 0; t < nt; ++t) {
            const T *zt = Z + (size_t)(t0 + t) * m * n;
            for (int row = warp; row < zs; row += NT / 32) {
                const int ge = a0 + lo + row;
                stage<T, CG>(Zs + (t * zs + row) * TC + lane, zt + (size_t)ge * n + gc,
                             row < span && cin && ge >= 0 && ge < m, Z);
            }
        }
        stage_wait<false>();
        __syncthreads();
        for (int tb = 0; tb < nt; tb += 4) {
            const T *zc = Zs + (tb * zs + rb) * TC + lane;
            const T *gr = Gs + tb * w * TA + rb;
            switch (min(4, nt - tb)) {
                case 1: cols_terms<T, 1>(zc, gr, w, zs, acc); break;
                case 2: cols_terms<T, 2>(zc, gr, w, zs, acc); break;
                case 3: cols_terms<T, 3>(zc, gr, w, zs, acc); break;
                default: cols_terms<T, 4>(zc, gr, w, zs, acc); break;
            }
        }
        __syncthreads();
    }
    cols_epilogue<T, EPI>(acc, m, n, a0, rb, gc, Out, pa);
    if (!CG) pdl_trigger();
}

}  // namespace band
}  // namespace sfista
