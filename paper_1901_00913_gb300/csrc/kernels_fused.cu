// One kernel per operator application of the banded FP32 operator:
//   Out[a][c] = sum_i sum_k G_i[a][a + loG + k] * Z_i[a + loG + k][c],
//   Z_i[e][c] = sum_k In[e][c + loF + k] * F_i[c][c + loF + k],
// i.e. sum_i B_i (In A_i^T) with (F, G) = (A, B), or sum_i B_i^T (In A_i) with
// (F, G) = (A^T, B^T), followed by the epilogue (store, residual, or Step 1
// shrink + Step 3 momentum).  A block computes a 32 x 32 output tile: it
// stages the input tile with its halo in both directions and all band tiles
// (cp.async, one load phase), computes the intermediate rows Z_i for the
// 32 + wG - 1 rows the column pass needs into shared memory, then runs the
// column pass.  Z never goes to global memory and an iteration of Alg. 2 is
// two launches.  The row pass repeats the halo rows' work ((32 + wG - 1) / 32
// times the two-pass count); at small and medium sizes the launch and load
// latency saved outweighs it.
#include <algorithm>

#include "band_items.cuh"
#include "epilogue.cuh"
#include "internal.h"

namespace sfista {
namespace {

using band::NT;
using band::TA;
using band::TC;
constexpr int ZST = TC + 4;   // Z row stride: float4 stores of 32 consecutive rows hit distinct banks

struct FusedGeom {
    int zs;    // staged Z rows per term: TA + wG (last one spare, zero)
    int sp;    // input tile row stride: (TC + wF) | 1
    size_t off_f, off_g, off_z, total;   // float offsets / size
};

__host__ __device__ inline FusedGeom fused_geom(int r, int wF, int wG) {
    FusedGeom g;
    g.zs = TA + wG;
    g.sp = (TC + wF) | 1;
    const size_t in = (size_t)g.zs * g.sp;
    g.off_f = (in + 3) & ~size_t(3);
    g.off_g = g.off_f + (size_t)r * wF * TC;
    g.off_z = g.off_g + (size_t)r * wG * TA;
    g.total = g.off_z + (size_t)r * g.zs * ZST;
    return g;
}

// Row pass into shared memory for K terms: lane l owns Z rows rbase + l, warp
// w columns 4w .. 4w+3; the input window is shared by the K terms.
template <int K>
__device__ __forceinline__ void rows_to_smem(const float *xr, const float *fr, int wF, float *zs_out, int zs_stride) {
    float acc[K][4];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    float x0 = xr[0], x1 = xr[1], x2 = xr[2], x3 = xr[3];
#pragma unroll 2
    for (int k = 0; k < wF; ++k) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float4 f = *reinterpret_cast<const float4 *>(fr + (q * wF + k) * TC);
            acc[q][0] = fmaf(x0, f.x, acc[q][0]);
            acc[q][1] = fmaf(x1, f.y, acc[q][1]);
            acc[q][2] = fmaf(x2, f.z, acc[q][2]);
            acc[q][3] = fmaf(x3, f.w, acc[q][3]);
        }
        x0 = x1;
        x1 = x2;
        x2 = x3;
        x3 = xr[k + 4];
    }
#pragma unroll
    for (int q = 0; q < K; ++q)
        *reinterpret_cast<float4 *>(zs_out + q * zs_stride) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
}

template <int EPI>
__global__ void __launch_bounds__(NT) band_op_fused_kernel(const float *__restrict__ In, int m, int n, int r,
                                                           const float *__restrict__ Fb, int loF, int wF,
                                                           const float *__restrict__ Gb, int loG, int wG,
                                                           float *__restrict__ Out, ProxArgs pa) {
    extern __shared__ __align__(16) float sm[];
    const FusedGeom geo = fused_geom(r, wF, wG);
    float *Ins = sm, *Fs = sm + geo.off_f, *Gs = sm + geo.off_g, *Zs = sm + geo.off_z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int a0 = blockIdx.y * TA, c0 = blockIdx.x * TC;
    const int e0 = a0 + loG;                 // first staged row
    const int spanc = TC + wF - 1, spanr = TA + wG - 1;
    // Constant band tiles first, then (after the previous kernel) the input tile.
    if ((n & 3) == 0 && (m & 3) == 0) {
        // 16-byte copies: thread (row tk, quad j) copies 4 band entries; the
        // tail of a ragged tile is zero-filled by the copy's source size.
        const int j = tid & 7;
        const int fb = min(16, max(0, (n - (c0 + 4 * j)) * 4)), gb = min(16, max(0, (m - (a0 + 4 * j)) * 4));
        for (int tk = tid >> 3; tk < r * wF; tk += NT / 8)
            band::stage16(Fs + tk * TC + 4 * j, Fb + (size_t)tk * n + c0 + 4 * j, fb, Fb);
        for (int tk = tid >> 3; tk < r * wG; tk += NT / 8)
            band::stage16(Gs + tk * TA + 4 * j, Gb + (size_t)tk * m + a0 + 4 * j, gb, Gb);
    } else {
        const bool cin = c0 + lane < n, rin = a0 + lane < m;
        for (int tk = warp; tk < r * wF; tk += NT / 32)
            band::stage<float, false>(Fs + tk * TC + lane, Fb + (size_t)tk * n + c0 + lane, cin, Fb);
        for (int tk = warp; tk < r * wG; tk += NT / 32)
            band::stage<float, false>(Gs + tk * TA + lane, Gb + (size_t)tk * m + a0 + lane, rin, Gb);
    }
    band::pdl_wait();
    for (int row = warp; row < geo.zs; row += NT / 32) {
        const int ge = e0 + row;
        const bool rok = row < spanr && ge >= 0 && ge < m;
        for (int col = lane; col < geo.sp; col += 32) {
            const int gc = c0 + loF + col;
            band::stage<float, false>(Ins + row * geo.sp + col, In + (size_t)ge * n + gc,
                                      rok && col < spanc && gc >= 0 && gc < n, In);
        }
    }
    band::stage_wait<false>();
    __syncthreads();
    // Row pass: Z_i for staged rows [0, zs) (row zs-1 and out-of-image rows come out 0).
    const int cb = warp * 4;
    for (int rbase = 0; rbase < geo.zs; rbase += 32) {
        const int row = rbase + lane;
        if (row < geo.zs) {
            const float *xr = Ins + row * geo.sp + cb;
            for (int tb = 0; tb < r; tb += 4) {
                float *zo = Zs + ((size_t)tb * geo.zs + row) * ZST + cb;
                const float *fr = Fs + tb * wF * TC + cb;
                switch (min(4, r - tb)) {
                    case 1: rows_to_smem<1>(xr, fr, wF, zo, geo.zs * ZST); break;
                    case 2: rows_to_smem<2>(xr, fr, wF, zo, geo.zs * ZST); break;
                    case 3: rows_to_smem<3>(xr, fr, wF, zo, geo.zs * ZST); break;
                    default: rows_to_smem<4>(xr, fr, wF, zo, geo.zs * ZST); break;
                }
            }
        }
    }
    __syncthreads();
    // Column pass: lane l column c0 + l, warp w rows a0 + 4w .. a0 + 4w + 3.
    const int rb = warp * 4, gc = c0 + lane;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int tb = 0; tb < r; tb += 4) {
        const float *zc = Zs + ((size_t)tb * geo.zs + rb) * ZST + lane;
        const float *gr = Gs + tb * wG * TA + rb;
        switch (min(4, r - tb)) {
            case 1: band::cols_terms<float, 1, ZST>(zc, gr, wG, geo.zs, acc); break;
            case 2: band::cols_terms<float, 2, ZST>(zc, gr, wG, geo.zs, acc); break;
            case 3: band::cols_terms<float, 3, ZST>(zc, gr, wG, geo.zs, acc); break;
            default: band::cols_terms<float, 4, ZST>(zc, gr, wG, geo.zs, acc); break;
        }
    }
    if (gc < n) {
        if (EPI == EPI_PROX) {
            size_t idx[4];
            float g[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ok[j] = a0 + rb + j < m;
                idx[j] = (size_t)(a0 + rb + j) * n + gc;
                g[j] = acc[j];
            }
            prox_momentum_n<4>(pa, idx, g, ok);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ga = a0 + rb + j;
                if (ga >= m) break;
                const size_t idx = (size_t)ga * n + gc;
                Out[idx] = EPI == EPI_STORE ? acc[j] : acc[j] - pa.Bd[idx];
            }
        }
    }
    band::pdl_trigger();
}

constexpr size_t kFusedSmemMax = 227 * 1024;

}  // namespace

size_t band_op_fused_smem(int r, int wF, int wG) { return sizeof(float) * fused_geom(r, wF, wG).total; }

// Sets the kernels' shared-memory limit; false if one tile does not fit.
bool band_op_fused_prepare(int r, int wF, int wG) {
    const size_t sm = band_op_fused_smem(r, wF, wG);
    if (sm > kFusedSmemMax) return false;
    for (auto k : {band_op_fused_kernel<EPI_STORE>, band_op_fused_kernel<EPI_RESIDUAL>, band_op_fused_kernel<EPI_PROX>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax) != cudaSuccess)
            return false;
    return true;
}

void launch_band_op_fused(const float *In, int m, int n, int r, const float *Fb, int loF, int wF, const float *Gb,
                          int loG, int wG, EpiKind epi, float *Out, const ProxArgs &pa, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((n + TC - 1) / TC, (m + TA - 1) / TA);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = band_op_fused_smem(r, wF, wG);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (epi == EPI_STORE)
        cudaLaunchKernelEx(&cfg, band_op_fused_kernel<EPI_STORE>, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out, pa);
    else if (epi == EPI_RESIDUAL)
        cudaLaunchKernelEx(&cfg, band_op_fused_kernel<EPI_RESIDUAL>, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out, pa);
    else
        cudaLaunchKernelEx(&cfg, band_op_fused_kernel<EPI_PROX>, In, m, n, r, Fb, loF, wF, Gb, loG, wG, Out, pa);
}

}  // namespace sfista
