// The whole Alg. 2 loop in one persistent, cooperatively launched kernel
// (banded FP32 operator, double-float FISTA state).
//
// For small and medium images one iteration is only a few hundred MFLOP, so
// four dependent launches per iteration spend most of their time in launch
// latency and ramp-up.  Here every block stays resident for the whole solve
// and walks the four phases of each iteration,
//   phase 0  Z_i = Y A_i^T          (rows pass, work item = term x tile)
//   phase 1  R   = sum_i B_i Z_i - B (cols pass + residual)
//   phase 2  Z_i = R A_i            (rows pass with the band of A^T)
//   phase 3  G   = sum_i B_i^T Z_i; shrink, optional projection, momentum
// separated by a grid-wide barrier.  The barrier is a counter plus a
// generation word in global memory; its spin is bounded (about one second),
// after which the block records DEV_TIMEOUT and the kernel returns.  The
// cooperative launch guarantees that all blocks are co-resident.  Data that
// another block wrote earlier in the same launch is read with ld.global.cg
// (L2, not the non-coherent L1).
#include <algorithm>

#include "band_items.cuh"
#include "band_items4.cuh"
#include "epilogue.cuh"
#include "internal.h"

namespace sfista {
namespace {

constexpr int PT = 256;          // threads per block
constexpr int PR_A = band::TA;     // rows-pass tile: 32 x 32
constexpr int PR_C = band::TC;
constexpr int PC_A = band::TA;     // cols-pass tile: 16 rows x 64 columns
constexpr int PC_C = band::TC;
constexpr long long kBarrierCycles = 2000000000LL;

struct PersistArgs {
    int m, n, r;
    const float *fA, *fB, *fAT, *fBT;
    int loA, wA, loB, wB, loAT, wAT, loBT, wBT;
    float *Z, *R;
    ProxArgs pa;             // Bd, Y, Yop, beta, constants, status (Xin/Xout set per iteration)
    float2 *Xb0, *Xb1;
    int k0, iters;
    unsigned *bar_count, *bar_gen;
    int rows_chunk, cols_chunk;   // terms staged per load phase
};

// Grid-wide barrier with a bounded spin.  Returns false if it gave up.
__device__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, unsigned *status, int *abort_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > kBarrierCycles) {
                    atomicOr(status, DEV_TIMEOUT);
                    *abort_sh = 1;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *abort_sh == 0;
}

__device__ __forceinline__ void rows_item(const float *In, int m, int n, const float *Fb, int lo, int w, int t0,
                                          int nt, int a0, int c0, float *Z, float *sm) {
    band::rows_item<float, true>(In, m, n, Fb, lo, w, t0, nt, a0, c0, Z, sm);
}

template <int EPI>
__device__ __forceinline__ void cols_item(const float *Z, int m, int n, int r, int chunk, const float *Gb, int lo,
                                          int w, int a0, int c0, float *Out, const ProxArgs &pa, float *sm) {
    band::cols_item<float, EPI, true>(Z, m, n, r, chunk, Gb, lo, w, a0, c0, Out, pa, sm);
}

__global__ void __launch_bounds__(PT) band_solve_persistent(PersistArgs a) {
    extern __shared__ float sm[];
    __shared__ int abort_sh;
    if (threadIdx.x == 0) abort_sh = 0;
    __syncthreads();
    const int m = a.m, n = a.n, r = a.r;
    const int rt_c = (n + PR_C - 1) / PR_C, rt_a = (m + PR_A - 1) / PR_A;
    const int ct_c = (n + PC_C - 1) / PC_C, ct_a = (m + PC_A - 1) / PC_A;
    const int rch = a.rows_chunk, nrch = (r + rch - 1) / rch;
    const int rows_items = nrch * rt_a * rt_c, cols_items = ct_a * ct_c;
    const unsigned nb = gridDim.x;
    ProxArgs pa = a.pa;
    for (int k = a.k0 + 1; k <= a.k0 + a.iters; ++k) {
        pa.k = k;
        pa.Xin = (k - 1) & 1 ? a.Xb1 : a.Xb0;
        pa.Xout = k & 1 ? a.Xb1 : a.Xb0;
        for (int it = blockIdx.x; it < rows_items; it += nb) {
            const int q = it / (rt_a * rt_c), t = it - q * rt_a * rt_c;
            rows_item(pa.Yop, m, n, a.fA, a.loA, a.wA, q * rch, min(rch, r - q * rch), (t / rt_c) * PR_A,
                      (t % rt_c) * PR_C, a.Z, sm);
        }
        if (!grid_barrier(a.bar_count, a.bar_gen, nb, pa.status, &abort_sh)) return;
        for (int it = blockIdx.x; it < cols_items; it += nb)
            cols_item<EPI_RESIDUAL>(a.Z, m, n, r, a.cols_chunk, a.fB, a.loB, a.wB, (it / ct_c) * PC_A, (it % ct_c) * PC_C, a.R, pa,
                                    sm);
        if (!grid_barrier(a.bar_count, a.bar_gen, nb, pa.status, &abort_sh)) return;
        for (int it = blockIdx.x; it < rows_items; it += nb) {
            const int q = it / (rt_a * rt_c), t = it - q * rt_a * rt_c;
            rows_item(a.R, m, n, a.fAT, a.loAT, a.wAT, q * rch, min(rch, r - q * rch), (t / rt_c) * PR_A,
                      (t % rt_c) * PR_C, a.Z, sm);
        }
        if (!grid_barrier(a.bar_count, a.bar_gen, nb, pa.status, &abort_sh)) return;
        for (int it = blockIdx.x; it < cols_items; it += nb)
            cols_item<EPI_PROX>(a.Z, m, n, r, a.cols_chunk, a.fBT, a.loBT, a.wBT, (it / ct_c) * PC_A, (it % ct_c) * PC_C, nullptr,
                                pa, sm);
        if (!grid_barrier(a.bar_count, a.bar_gen, nb, pa.status, &abort_sh)) return;
    }
}

}  // namespace

constexpr size_t kPersistSmemBudget = 100 * 1024;   // two blocks per SM
constexpr size_t kPersistSmemMax = 227 * 1024;      // the most one block may use

// Terms staged per load phase so that one item fits the shared-memory budget.
void persistent_chunks(int r, int wmax, int *rows_chunk, int *cols_chunk, size_t *smem) {
    const size_t rows_fixed = band::rows_smem<float>(wmax, 0);
    const size_t rows_term = band::rows_smem<float>(wmax, 1) - rows_fixed;
    const size_t cols_term = band::cols_smem<float>(wmax, 1);
    int rc = rows_fixed < kPersistSmemBudget ? (int)((kPersistSmemBudget - rows_fixed) / rows_term) : 1;
    int cc = (int)(kPersistSmemBudget / cols_term);
    rc = std::max(1, std::min(r, rc));
    cc = std::max(1, std::min(r, cc));
    *rows_chunk = rc;
    *cols_chunk = cc;
    *smem = std::max(rows_fixed + rc * rows_term, cc * cols_term);
}

void grouped_chunks(int r, int wmax, bool vec, int rows_req, int cols_req, int *rows_chunk, int *cols_chunk,
                    size_t *smem) {
    auto rows_b = [&](int c) { return vec ? band4::rows_smem(64, wmax, c) : band::rows_smem<float>(wmax, c); };
    auto cols_b = [&](int c) { return vec ? band4::cols_smem(64, wmax, c) : band::cols_smem<float>(wmax, c); };
    // Default: as many terms as fit in the persistent solver's budget.
    int rc = 1, cc = 1;
    while (rc < r && rows_b(rc + 1) <= kPersistSmemBudget) ++rc;
    while (cc < r && cols_b(cc + 1) <= kPersistSmemBudget) ++cc;
    if (rows_req > 0 && rows_b(std::min(rows_req, r)) <= 227 * 1024) rc = std::min(rows_req, r);
    if (cols_req > 0 && cols_b(std::min(cols_req, r)) <= 227 * 1024) cc = std::min(cols_req, r);
    *rows_chunk = rc;
    *cols_chunk = cc;
    *smem = std::max(rows_b(rc), cols_b(cc));
}

namespace {

// Grouped stages: block b runs work item items[b] of problem items[b].prob.
__global__ void __launch_bounds__(PT) band_rows_grouped(const BandProb *probs, const BandItem *items, int phase) {
    extern __shared__ float sm[];
    const BandItem it = items[blockIdx.x];
    const BandProb &P = probs[it.prob];
    const int rt_c = (P.n + PR_C - 1) / PR_C;
    const int t0 = it.q * P.rows_chunk, nt = min(P.rows_chunk, P.r - t0);
    const float *In = phase == 0 ? P.pa.Yop : P.R;
    const float *F = phase == 0 ? P.fA : P.fAT;
    const int lo = phase == 0 ? P.loA : P.loAT, w = phase == 0 ? P.wA : P.wAT;
    // Separate launches per stage: the input was written by an earlier launch,
    // so the cp.async staging of the plain kernels applies.
    if (P.vec)
        band4::rows_item<64>(In, P.m, P.n, F, lo, w, t0, nt, (it.tile / rt_c) * 64, (it.tile % rt_c) * PR_C, P.Z, sm);
    else
        band::rows_item<float, false>(In, P.m, P.n, F, lo, w, t0, nt, (it.tile / rt_c) * PR_A,
                                      (it.tile % rt_c) * PR_C, P.Z, sm);
}

__global__ void __launch_bounds__(PT) band_cols_grouped(const BandProb *probs, const BandItem *items, int phase,
                                                        int k) {
    extern __shared__ float sm[];
    const BandItem it = items[blockIdx.x];
    const BandProb &P = probs[it.prob];
    const int ct_c = (P.n + PC_C - 1) / PC_C;
    const int a0 = (it.tile / ct_c) * (P.vec ? 64 : PC_A), c0 = (it.tile % ct_c) * PC_C;
    ProxArgs pa = P.pa;
    if (phase == 1) {
        if (P.vec)
            band4::cols_item<EPI_RESIDUAL, 64>(P.Z, P.m, P.n, P.r, P.cols_chunk, P.fB, P.loB, P.wB, a0, c0, P.R, pa,
                                               sm);
        else
            band::cols_item<float, EPI_RESIDUAL, false>(P.Z, P.m, P.n, P.r, P.cols_chunk, P.fB, P.loB, P.wB, a0, c0,
                                                        P.R, pa, sm);
    } else {
        float2 *b0 = const_cast<float2 *>(pa.Xin), *b1 = pa.Xout;
        pa.k = k;
        pa.Xin = (k - 1) & 1 ? b1 : b0;
        pa.Xout = k & 1 ? b1 : b0;
        if (P.vec)
            band4::cols_item<EPI_PROX, 64>(P.Z, P.m, P.n, P.r, P.cols_chunk, P.fBT, P.loBT, P.wBT, a0, c0, nullptr,
                                           pa, sm);
        else
            band::cols_item<float, EPI_PROX, false>(P.Z, P.m, P.n, P.r, P.cols_chunk, P.fBT, P.loBT, P.wBT, a0, c0,
                                                    nullptr, pa, sm);
    }
}

}  // namespace

int band_rows_tiles(int m, int n, bool vec) {
    return vec ? band4::tiles(64, m, n) : ((m + PR_A - 1) / PR_A) * ((n + PR_C - 1) / PR_C);
}
int band_cols_tiles(int m, int n, bool vec) {
    return vec ? band4::tiles(64, m, n) : ((m + PC_A - 1) / PC_A) * ((n + PC_C - 1) / PC_C);
}

// The attribute is per kernel, not per batch: allow the largest size, so that
// a later batch with smaller tiles never lowers an earlier batch's limit.
cudaError_t band_grouped_prepare(size_t smem) {
    if (smem > kPersistSmemMax) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(band_rows_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPersistSmemMax);
    if (e) return e;
    return cudaFuncSetAttribute(band_cols_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPersistSmemMax);
}

void launch_band_grouped_stage(int st, const BandProb *probs, const BandItem *items, int nitems, int k, size_t smem,
                               cudaStream_t s) {
    if (st == 0 || st == 2) band_rows_grouped<<<nitems, PT, smem, s>>>(probs, items, st);
    else band_cols_grouped<<<nitems, PT, smem, s>>>(probs, items, st, k);
}


// Grid size for the persistent solver: all co-resident blocks, capped by the work.
sfista_status persistent_config(int m, int n, int r, int wmax, int dev, int *grid, size_t *smem, int *rows_chunk,
                                int *cols_chunk) {
    persistent_chunks(r, wmax, rows_chunk, cols_chunk, smem);
    // The attribute is per kernel: the largest size it may take (the device's
    // opt-in maximum less its static shared memory), never this one's.
    cudaFuncAttributes fa{};
    int optin = 0;
    cudaError_t e = cudaFuncGetAttributes(&fa, band_solve_persistent);
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e) return fail(SFISTA_ECUDA, std::string("persistent attributes: ") + cudaGetErrorString(e));
    const int lim = optin - (int)fa.sharedSizeBytes;
    if (*smem > (size_t)lim) return fail(SFISTA_ENOTSUP, "persistent solver tile exceeds shared memory");
    e = cudaFuncSetAttribute(band_solve_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return fail(SFISTA_ENOTSUP, std::string("persistent smem: ") + cudaGetErrorString(e));
    int per_sm = 0, sms = 0, coop = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, band_solve_persistent, PT, *smem)) ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)))
        return fail(SFISTA_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (!coop || per_sm < 1) return fail(SFISTA_ENOTSUP, "cooperative launch unavailable for the persistent solver");
    const long nrch = (r + *rows_chunk - 1) / *rows_chunk;
    const long work = std::max<long>(nrch * ((m + PR_A - 1) / PR_A) * ((n + PR_C - 1) / PR_C),
                                     (long)((m + PC_A - 1) / PC_A) * ((n + PC_C - 1) / PC_C));
    *grid = (int)std::min<long>((long)std::min(per_sm, 2) * sms, work);
    return SFISTA_OK;
}

cudaError_t launch_persistent(int grid, size_t smem, int rows_chunk, int cols_chunk, int m, int n, int r, const float *fA, const Band &A,
                              const float *fB, const Band &B, const float *fAT, const Band &AT, const float *fBT,
                              const Band &BT, float *Z, float *R, float2 *Xb0, float2 *Xb1, const ProxArgs &pa,
                              int k0, int iters, unsigned *bar, cudaStream_t s) {
    PersistArgs a{};
    a.m = m;
    a.n = n;
    a.r = r;
    a.fA = fA;
    a.fB = fB;
    a.fAT = fAT;
    a.fBT = fBT;
    a.loA = A.lo;
    a.wA = A.w;
    a.loB = B.lo;
    a.wB = B.w;
    a.loAT = AT.lo;
    a.wAT = AT.w;
    a.loBT = BT.lo;
    a.wBT = BT.w;
    a.Z = Z;
    a.R = R;
    a.pa = pa;
    a.Xb0 = Xb0;
    a.Xb1 = Xb1;
    a.k0 = k0;
    a.iters = iters;
    a.bar_count = bar;
    a.bar_gen = bar + 1;
    a.rows_chunk = rows_chunk;
    a.cols_chunk = cols_chunk;
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)band_solve_persistent, dim3(grid), dim3(PT), args, smem, s);
}

}  // namespace sfista
