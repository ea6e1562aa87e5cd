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

template <typename T>
__host__ __device__ inline size_t rows_smem(int w, int nt) {
    return sizeof(T) * ((size_t)TA * rows_span(w) + (size_t)nt * w * TC);
}
// Per staged term: (TA + w) x TC values of Z (one spare row) and w x TA band entries.
template <typename T>
__host__ __device__ inline size_t cols_smem(int w, int chunk) {
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

template <typename T, bool CG>
__device__ __forceinline__ void rows_item(const T *__restrict__ In, int m, int n, const T *__restrict__ Fb, int lo,
                                          int w, int t0, int nt, int a0, int c0, T *__restrict__ Z, T *sm) {
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

template <typename T, int EPI, bool CG>
__device__ __forceinline__ void cols_item(const T *__restrict__ Z, int m, int n, int r, int chunk,
                                          const T *__restrict__ Gb, int lo, int w, int a0, int c0, T *__restrict__ Out,
                                          const ProxArgs &pa, T *sm) {
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
