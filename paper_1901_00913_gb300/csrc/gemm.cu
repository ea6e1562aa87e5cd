// Tensor-core execution of the Kronecker operator: tcgen05.mma with the
// accumulator in TMEM, operands staged by TMA, fused epilogues.
//
// One iteration of Alg. 2 (Step 1) is four products, each written as a GEMM
// C[M][N] = sum_k P[M][k] Q[N][k] with both operands K-major in memory:
//   stage 0  Tt[i][c][a] = sum_b A_i[c][b]  Y[a][b]         (Y A_i^T, stored transposed)
//   stage 1  R[a][c]     = sum_{i,e} B_i[a][e] Tt[i][c][e]  - Bdata[a][c]
//   stage 2  Ut[j][b][a] = sum_c A^T_j[b][c] R[a][c]        (R A_j, stored transposed)
//   stage 3  G[a][b]     = sum_{j,e} B^T_j[a][e] Ut[j][b][e];  then Step 1 shrink and
//                          Step 3 momentum in the epilogue (double-float state).
// Stages 0 and 2 stack the r terms along M (one M tile belongs to one term);
// stages 1 and 3 sum the r terms along K.  The factors are banded, so an M
// tile of rows [m0, m0+128) only meets K columns [m0 + lo, m0 + 127 + hi];
// in band mode the K loop covers just that range (exact: the skipped factor
// entries are zero), in dense mode the whole K extent.
//
// Split precision: operands are stored as hi + lo pairs (BF16 or TF32) and
// each K step issues hi*hi + lo*hi + hi*lo into the same FP32 accumulator.
//
// Kernel roles (320 threads): warp 0 lane 0 issues TMA loads into a ring of
// shared-memory stages; warp 1 owns the TMEM allocation and lane 0 issues the
// MMAs, releasing each stage with tcgen05.commit; warps 2-9 wait for the
// accumulator, read it with tcgen05.ld in chunks of 64 columns (two warps per
// 32-lane quarter, 32 columns each) and run the epilogue.  Tile shapes: N
// tile 64, 128 or 256 (BN), and for the stacked stages optionally a resident
// factor panel (RES); the four stages are chained by programmatic dependent
// launch.  Every mbarrier wait is bounded (about one second); on expiry the
// kernel records DEV_TIMEOUT in the status word, drains what it issued and
// returns, so the host sees SFISTA_ETIMEOUT instead of a hang.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "epilogue.cuh"
#include "gemm.h"

namespace sfista {
namespace {

constexpr int BM = 128;                 // MMA M (rows of P per tile)
constexpr int KB_BYTES = 128;           // bytes of one K block per row (one 128 B swizzle span)
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

enum Fmt : int { FMT_BF16 = 0, FMT_TF32 = 1 };
enum GEpi : int { GE_SPLIT = 0, GE_RESID = 1, GE_PROX = 2, GE_STORE = 3 };

struct GemmArgs {
    int rows;        // P rows per term (extent of M within one term)
    int m_tiles;     // M tiles per term
    int N;           // extent of N
    int K;           // extent of K within one segment
    int band_lo;     // K range of the tile at m0: [m0 + band_lo, m0 + BM - 1 + band_hi]
    int band_hi;
    int dense;       // 1: whole K range
    int segs;        // K segments (terms summed along K); 1 when terms stack along M
    int type_b;      // 1: P and Q both indexed by the K segment; 0: P by the tile's term
    void *out_hi, *out_lo;   // GE_SPLIT / GE_RESID operand copies
    float *out_f32;          // GE_STORE
    const float *Bd;         // GE_RESID
    int split_kind;          // 1 bf16, 2 tf32 (fp32 storage)
    int keep_l2;             // GE_SPLIT, BF16: tensor-store the output with an L2 evict-last policy
    ProxArgs pa;             // GE_PROX
    unsigned *status;
};

template <int FMT, bool SPLIT, int BN>
struct Cfg {
    static constexpr int P_BYTES = BM * KB_BYTES;
    static constexpr int Q_BYTES = BN * KB_BYTES;
    static constexpr int NOP = SPLIT ? 2 : 1;
    static constexpr int STAGE_BYTES = NOP * (P_BYTES + Q_BYTES);
    static constexpr int KSTEPS = KB_BYTES / 32;    // MMA K step = 32 bytes (16 bf16 / 8 tf32)
    static constexpr int KB_ELEMS = FMT == FMT_BF16 ? 64 : 32;
    static constexpr int ALIGN = FMT == FMT_BF16 ? 8 : 4;   // 16-byte TMA x alignment
    // Instruction descriptor: D=F32, A/B = BF16 (kind::f16) or TF32 (kind::tf32),
    // both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
    static constexpr uint32_t IDESC = (1u << 4) | ((FMT == FMT_BF16 ? 1u : 2u) << 7) |
                                      ((FMT == FMT_BF16 ? 1u : 2u) << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false (and DEV_TIMEOUT) on expiry.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned *status) {
    if (mbar_try(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(status, DEV_TIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
// Tensor store of one box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     (uint64_t)map),
                 "r"(src), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
// The same with an L2 eviction-priority policy (from l2_evict_last).
__device__ __forceinline__ void tma_store_3d_hint(const CUtensorMap *map, uint32_t src, int x, int y, int z,
                                                  uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3, %4}], [%1], %5;" ::"l"(
            (uint64_t)map),
        "r"(src), "r"(x), "r"(y), "r"(z), "l"(policy)
        : "memory");
}
// An L2 policy that keeps the lines it covers over normal ones when L2 evicts.
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// The committed stores have finished reading shared memory (the buffer may be rewritten).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// The committed stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Generic-proxy shared-memory writes become visible to the async proxy (TMA).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1 (bit 46), layout SWIZZLE_128B (2 << 61).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
template <int FMT>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (FMT == FMT_BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
}
// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Store four neighbouring values (idx a multiple of 4) as split operand
// copies: one 8-byte (BF16) or 16-byte (TF32) store per copy.
__device__ __forceinline__ void store_split4(void *hi, void *lo, int kind, size_t idx, float4 v) {
    if (kind == 1) {
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
        *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(hi) + idx) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&h01), *reinterpret_cast<const uint32_t *>(&h23));
        if (lo)
            *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(lo) + idx) =
                make_uint2(pack_bf16x2(v.x - __bfloat162float(h01.x), v.y - __bfloat162float(h01.y)),
                           pack_bf16x2(v.z - __bfloat162float(h23.x), v.w - __bfloat162float(h23.y)));
    } else {
        const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(hi) + idx) = h;
        if (lo)
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(lo) + idx) =
                make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y), tf32_round(v.z - h.z),
                            tf32_round(v.w - h.w));
    }
}

struct WorkItem {
    int prob, mt, nt, pad;
};

// Shared-memory plan of a kernel instance.  RES: the P panel of a tile (all
// its K blocks, hi and lo) stays resident in its own region while the tiles
// that share it run, and the ring carries Q blocks only.
template <int FMT, bool SPLIT, int BN, bool RES>
struct PCfg {
    using C = Cfg<FMT, SPLIT, BN>;
    static_assert(BN % 64 == 0 && BN <= 256, "the epilogue drains 64-column chunks; MMA N <= 256");
    static_assert(!RES || FMT == FMT_BF16, "a resident panel holds 3 K blocks of 64 BF16 values");
    static constexpr int CW = 64;                        // accumulator columns per epilogue chunk
    static constexpr int STAGING = BM * (CW + 1) * 4;    // one chunk, row stride CW + 1 floats
    static constexpr int RES_KB = RES ? 3 : 0;           // K blocks a resident panel holds
    static constexpr int P_REGION = RES_KB * C::NOP * C::P_BYTES;
    static constexpr int STAGE_BYTES = RES ? C::NOP * C::Q_BYTES : C::STAGE_BYTES;
    static constexpr int RING_MAX = 225 * 1024 - STAGING - P_REGION;
    static constexpr int STAGES_RAW = RING_MAX / STAGE_BYTES;
    static constexpr int STAGES = STAGES_RAW > 6 ? 6 : (STAGES_RAW < 2 ? 2 : STAGES_RAW);
    static constexpr int SMEM = P_REGION + STAGES * STAGE_BYTES + STAGING + 1024;
    static_assert(SMEM <= 227 * 1024 - 256, "dynamic plus static shared memory of one CTA");
    static constexpr uint32_t TMEM_COLS = 2 * BN;   // two accumulators
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// K range of the M tile starting at m0 (band mode) and the number of K blocks.
template <int FMT, bool SPLIT, int BN>
__device__ __forceinline__ void tile_k_range(const GemmArgs &g, int m0, int *k_lo, int *nkb) {
    using C = Cfg<FMT, SPLIT, BN>;
    int lo = 0, hi = g.K;
    if (!g.dense) {
        lo = max(0, m0 + g.band_lo);
        hi = min(g.K, m0 + BM + g.band_hi);
        lo = (lo / C::ALIGN) * C::ALIGN;
    }
    *k_lo = lo;
    *nkb = hi > lo ? (hi - lo + C::KB_ELEMS - 1) / C::KB_ELEMS : 0;
}

// Persistent GEMM stage.  CTA c walks tiles c, c + gridDim.x, ... (RES: a
// contiguous run of tiles, so that consecutive tiles share their P panel);
// the TMA producer and the MMA issuer run ahead through a ring of
// shared-memory stages while the eight epilogue warps drain the previous tile
// from the other of two TMEM accumulators.  Tiles come from (mt, nt) =
// (t / ntn, t % ntn) of one problem, or from a work list over many problems
// (GROUPED), whose tensor maps and arguments then live in global memory; for
// the grouped prox epilogue, k selects X_{k-1} / X_k among each problem's two
// state buffers (stored in pa.Xin / pa.Xout as buffers 0 / 1).
//
// RES (stacked stages, one term per tile): the P operand of a tile depends
// only on its row tile (term and m0), not on nt.  The producer loads that
// panel (every K block of the tile's band range, hi and lo) once into a
// resident region and streams only Q blocks through the ring; before it
// overwrites the panel for the next row tile it waits until the MMAs that
// read the old one have completed (the MMA warp commits `pempty` when it
// moves to a tile of another panel).
template <int FMT, bool SPLIT, int BN, int EPI, bool GROUPED, bool RES>
__global__ void __launch_bounds__(320, 1)
    umma_gemm_persistent(const __grid_constant__ CUtensorMap tPhi, const __grid_constant__ CUtensorMap tPlo,
                         const __grid_constant__ CUtensorMap tQhi, const __grid_constant__ CUtensorMap tQlo,
                         const __grid_constant__ CUtensorMap tOhi, const __grid_constant__ CUtensorMap tOlo,
                         const __grid_constant__ GemmArgs g1, int ntn, int ntiles, const CUtensorMap *maps,
                         const GemmArgs *args, const WorkItem *work, int kswap) {
    using C = Cfg<FMT, SPLIT, BN>;
    using PC = PCfg<FMT, SPLIT, BN, RES>;
    constexpr int S = PC::STAGES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * S + 7];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int ep_abort;   // epilogue warps leave the tile loop together

    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *ring = smem + PC::P_REGION;   // the resident panel (RES) sits below the ring
    float *tile = reinterpret_cast<float *>(ring + S * PC::STAGE_BYTES);
    constexpr int CW = PC::CW;     // columns per epilogue chunk
    constexpr int TS = CW + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[S]);
    const uint32_t tfull0 = smem_u32(&bars[2 * S]), tempty0 = smem_u32(&bars[2 * S + 2]);
    const uint32_t drainb = smem_u32(&bars[2 * S + 4]);
    const uint32_t pfull = smem_u32(&bars[2 * S + 5]), pempty = smem_u32(&bars[2 * S + 6]);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(full0 + 8 * q, 1);
            mbar_init(empty0 + 8 * q, 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(tfull0 + 8 * q, 1);
            mbar_init(tempty0 + 8 * q, 8);
        }
        mbar_init(drainb, 1);
        mbar_init(pfull, 1);
        mbar_init(pempty, 1);
        ep_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(PC::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    // Programmatic dependent launch: the next stage may launch now (its CTAs
    // start as ours exit and run their prologue), and this one waits here
    // until the previous kernel in the stream has completed and its writes
    // are visible.  Both are no-ops for a plain launch.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // This CTA's tiles: t_first, t_first + t_step, ... < t_end.
    int t_first = blockIdx.x, t_step = gridDim.x, t_end = ntiles;
    if (RES) {
        const int per = ntiles / (int)gridDim.x, rem = ntiles - per * (int)gridDim.x;
        t_first = (int)blockIdx.x * per + min((int)blockIdx.x, rem);
        t_end = t_first + per + ((int)blockIdx.x < rem ? 1 : 0);
        t_step = 1;
    }

    // Tile t -> its tensor maps, arguments, (mt, nt) and the key of its P
    // panel (problem and row tile).
    auto fetch = [&](int t, const CUtensorMap *&m4, const GemmArgs *&ga, int &mt, int &nt, int &key) {
        if (GROUPED) {
            const WorkItem w = work[t];
            m4 = maps + 6 * w.prob;
            ga = args + w.prob;
            mt = w.mt;
            nt = w.nt;
            key = (w.prob << 16) | w.mt;
        } else {
            m4 = nullptr;
            ga = &g1;
            mt = t / ntn;
            nt = t - mt * ntn;
            key = mt;
        }
    };
    // K range of a tile; a band wider than the resident panel (the host does
    // not choose RES then) leaves the tile empty instead of overrunning it.
    auto k_range = [&](const GemmArgs &ga, int m0, int &k_lo, int &nkb) {
        tile_k_range<FMT, SPLIT, BN>(ga, m0, &k_lo, &nkb);
        if (RES && nkb > PC::RES_KB) nkb = 0;
    };

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, panels = 0, key_prev = -1;
            bool abort = false;
            unsigned *st0 = GROUPED ? args[0].status : g1.status;
            for (int t = t_first; t < t_end && !abort; t += t_step) {
                const CUtensorMap *m4;
                const GemmArgs *ga;
                int mt, nt, key;
                fetch(t, m4, ga, mt, nt, key);
                const int term = ga->type_b ? 0 : mt / ga->m_tiles;
                const int m0 = (mt % ga->m_tiles) * BM, n0 = nt * BN;
                int k_lo, nkb;
                k_range(*ga, m0, k_lo, nkb);
                if (RES) {
                    int nkb_full;
                    tile_k_range<FMT, SPLIT, BN>(*ga, m0, &k_lo, &nkb_full);
                    if (nkb_full > PC::RES_KB) atomicOr(ga->status, DEV_BADARG);
                }
                const int total = nkb * ga->segs;
                const CUtensorMap *pPhi = GROUPED ? m4 : &tPhi, *pPlo = GROUPED ? m4 + 1 : &tPlo;
                const CUtensorMap *pQhi = GROUPED ? m4 + 2 : &tQhi, *pQlo = GROUPED ? m4 + 3 : &tQlo;
                if (RES && key != key_prev) {
                    // The previous panel is free once the MMAs that read it are done.
                    if (panels > 0 && !mbar_wait(pempty, (panels - 1) & 1, st0)) break;
                    mbar_expect_tx(pfull, (uint32_t)(nkb * C::NOP * C::P_BYTES));
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint32_t dst = smem_u32(smem + kb * C::NOP * C::P_BYTES);
                        tma_load_3d(dst, pPhi, pfull, k_lo + kb * C::KB_ELEMS, m0, term);
                        if (SPLIT) tma_load_3d(dst + C::P_BYTES, pPlo, pfull, k_lo + kb * C::KB_ELEMS, m0, term);
                    }
                    ++panels;
                    key_prev = key;
                }
                for (int q = 0; q < total; ++q, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (it / S) & 1;
                    if (!mbar_wait(empty0 + 8 * s, ph ^ 1, ga->status)) {
                        abort = true;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * s;
                    mbar_expect_tx(fb, PC::STAGE_BYTES);
                    const int seg = q / nkb, kb = q - seg * nkb;
                    const int kx = k_lo + kb * C::KB_ELEMS;
                    const int pz = ga->type_b ? seg : term, qz = ga->type_b ? seg : 0;
                    const uint32_t base = smem_u32(ring + s * PC::STAGE_BYTES);
                    const uint32_t qb = RES ? base : base + C::NOP * C::P_BYTES;
                    if (!RES) {
                        tma_load_3d(base, pPhi, fb, kx, m0, pz);
                        if (SPLIT) tma_load_3d(base + C::P_BYTES, pPlo, fb, kx, m0, pz);
                    }
                    tma_load_3d(qb, pQhi, fb, kx, n0, qz);
                    if (SPLIT) tma_load_3d(qb + C::Q_BYTES, pQlo, fb, kx, n0, qz);
                }
            }
            // Drain: the last fill of every stage (and of the panel) has landed
            // before the CTA can exit.
            for (int x = max(0, it - S); x < it; ++x) mbar_wait(full0 + 8 * (x % S), (x / S) & 1, st0);
            if (RES && panels > 0) mbar_wait(pfull, (panels - 1) & 1, st0);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, j = 0, panels = 0, key_prev = -1;
            bool abort = false;
            unsigned *st = GROUPED ? args[0].status : g1.status;
            for (int t = t_first; t < t_end && !abort; t += t_step, ++j) {
                const CUtensorMap *m4;
                const GemmArgs *ga;
                int mt, nt, key;
                fetch(t, m4, ga, mt, nt, key);
                const int m0 = (mt % ga->m_tiles) * BM;
                int k_lo, nkb;
                k_range(*ga, m0, k_lo, nkb);
                const int total = nkb * ga->segs;
                const int b = j & 1;
                if (!mbar_wait(tempty0 + 8 * b, ((j >> 1) & 1) ^ 1, st)) break;
                tc_fence_after();
                if (RES && key != key_prev) {
                    if (panels > 0) tc_commit(pempty);   // arrives when every MMA issued so far has completed
                    if (!mbar_wait(pfull, panels & 1, st)) break;
                    tc_fence_after();
                    ++panels;
                    key_prev = key;
                }
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int q = 0; q < total; ++q, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (it / S) & 1;
                    if (!mbar_wait(full0 + 8 * s, ph, st)) {
                        abort = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(ring + s * PC::STAGE_BYTES);
                    const uint32_t p_hi = RES ? smem_u32(smem + q * C::NOP * C::P_BYTES) : base;
                    const uint32_t p_lo = p_hi + C::P_BYTES;
                    const uint32_t q_hi = RES ? base : base + C::NOP * C::P_BYTES, q_lo = q_hi + C::Q_BYTES;
#pragma unroll
                    for (int ks = 0; ks < C::KSTEPS; ++ks) {
                        const uint32_t acc = (q > 0 || ks > 0) ? 1u : 0u;
                        tc_mma<FMT>(d, sw128_desc(p_hi + 32 * ks), sw128_desc(q_hi + 32 * ks), C::IDESC, acc);
                        if (SPLIT) {
                            tc_mma<FMT>(d, sw128_desc(p_lo + 32 * ks), sw128_desc(q_hi + 32 * ks), C::IDESC, 1u);
                            tc_mma<FMT>(d, sw128_desc(p_hi + 32 * ks), sw128_desc(q_lo + 32 * ks), C::IDESC, 1u);
                        }
                    }
                    tc_commit(empty0 + 8 * s);
                }
                tc_commit(tfull0 + 8 * b);   // arrives once this tile's MMAs complete
            }
            // Every MMA issued above has completed before TMEM is released.
            tc_commit(drainb);
            mbar_wait(drainb, 0, st);
        }
        __syncwarp();
    } else {
        // Epilogue, warps 2..9, one chunk of CW = 64 accumulator columns at a
        // time.  Phase 1: warp w reads TMEM lane quarter w % 4 (the only
        // quarter it may access), 32 of the chunk's columns, into the staging
        // tile; after the last chunk the accumulator is released to the MMA
        // warp.  Phase 2: the eight warps walk whole rows of the chunk so
        // global accesses are row-contiguous.
        const int lg = warp & 3, sub = (warp - 2) >> 2, ew = warp - 2;
        int j = 0;
        for (int t = t_first; t < t_end; t += t_step, ++j) {
            const CUtensorMap *m4;
            const GemmArgs *ga;
            int mt, nt, key;
            fetch(t, m4, ga, mt, nt, key);
            const int term = ga->type_b ? 0 : mt / ga->m_tiles;
            const int m0 = (mt % ga->m_tiles) * BM;
            int k_lo, nkb;
            k_range(*ga, m0, k_lo, nkb);
            const int total = nkb * ga->segs;
            const int b = j & 1;
            const bool ok = mbar_wait(tfull0 + 8 * b, (j >> 1) & 1, ga->status);
            tc_fence_after();
            if (!ok) ep_abort = 1;
            ProxArgs pa = ga->pa;
            if (EPI == GE_PROX && GROUPED) {
                float2 *b0 = const_cast<float2 *>(pa.Xin), *b1 = pa.Xout;
                float *f0 = const_cast<float *>(pa.Xin32), *f1 = pa.Xout32;
                pa.k = kswap;
                pa.Xin = (kswap - 1) & 1 ? b1 : b0;
                pa.Xout = kswap & 1 ? b1 : b0;
                pa.Xin32 = (kswap - 1) & 1 ? f1 : f0;
                pa.Xout32 = kswap & 1 ? f1 : f0;
            }
#pragma unroll 1
            for (int h = 0; h < BN / CW; ++h) {
                const bool last = h == BN / CW - 1;
                if constexpr (FMT == FMT_BF16 && (EPI == GE_SPLIT || EPI == GE_RESID)) {
                    // Split outputs: each warp converts its 32 x 32 block to
                    // BF16 hi/lo straight from TMEM into two 128B-swizzled boxes
                    // (the next stage's operand layout), and one thread stores
                    // them with TMA, asynchronously.
                    uint8_t *box_hi = reinterpret_cast<uint8_t *>(tile), *box_lo = box_hi + BM * 128;
                    if (ew == 0 && lane == 0) bulk_wait_read();   // the previous boxes have been read out
                    asm volatile("bar.sync 1, 256;" ::: "memory");
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + h * CW + sub * 32), v);
                    const int R = lg * 32 + lane;   // tile row of this lane
                    if (!ok || total == 0) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = 0.0f;
                    } else if (EPI == GE_RESID) {
                        const int row = m0 + R, col0 = nt * BN + h * CW + sub * 32;
                        if (row < ga->rows) {
                            const float *bp = ga->Bd + (size_t)row * ga->N + col0;
#pragma unroll
                            for (int g8 = 0; g8 < 4; ++g8) {
                                if (col0 + 8 * g8 < ga->N) {   // N is a multiple of 8
                                    const float4 x0 = __ldg(reinterpret_cast<const float4 *>(bp + 8 * g8));
                                    const float4 x1 = __ldg(reinterpret_cast<const float4 *>(bp + 8 * g8 + 4));
                                    v[8 * g8 + 0] -= x0.x;
                                    v[8 * g8 + 1] -= x0.y;
                                    v[8 * g8 + 2] -= x0.z;
                                    v[8 * g8 + 3] -= x0.w;
                                    v[8 * g8 + 4] -= x1.x;
                                    v[8 * g8 + 5] -= x1.y;
                                    v[8 * g8 + 6] -= x1.z;
                                    v[8 * g8 + 7] -= x1.w;
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int c8 = 0; c8 < 4; ++c8) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float a0 = v[8 * c8 + 2 * e], a1 = v[8 * c8 + 2 * e + 1];
                            const __nv_bfloat162 hh = __floats2bfloat162_rn(a0, a1);
                            hw[e] = *reinterpret_cast<const uint32_t *>(&hh);
                            lw[e] = pack_bf16x2(a0 - __bfloat162float(hh.x), a1 - __bfloat162float(hh.y));
                        }
                        const int pos = ((sub * 4 + c8) ^ (R & 7)) * 16;
                        *reinterpret_cast<uint4 *>(box_hi + R * 128 + pos) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if (SPLIT)
                            *reinterpret_cast<uint4 *>(box_lo + R * 128 + pos) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                    if (last) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tempty0 + 8 * b);
                    }
                    fence_async_smem();
                    asm volatile("bar.sync 1, 256;" ::: "memory");
                    if (ew == 0 && lane == 0) {
                        const CUtensorMap *oh = GROUPED ? m4 + 4 : &tOhi, *ol = GROUPED ? m4 + 5 : &tOlo;
                        const int x = nt * BN + h * CW;
                        if (x < ga->N) {   // boxes reaching past N or the last row are clipped by the unit
                            if (EPI == GE_SPLIT && ga->keep_l2) {
                                // T / U are read back by the next stage: stored with the
                                // evict-last priority (a request; without a persisting-L2
                                // set-aside most of them still reach DRAM).
                                const uint64_t pol = l2_evict_last();
                                tma_store_3d_hint(oh, smem_u32(box_hi), x, m0, term, pol);
                                if (SPLIT) tma_store_3d_hint(ol, smem_u32(box_lo), x, m0, term, pol);
                            } else {
                                tma_store_3d(oh, smem_u32(box_hi), x, m0, term);
                                if (SPLIT) tma_store_3d(ol, smem_u32(box_lo), x, m0, term);
                            }
                        }
                        bulk_commit();
                    }
                    continue;
                }
                {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + h * CW + sub * 32), v);
                    const bool zero = !ok || total == 0;
#pragma unroll
                    for (int q = 0; q < 32; ++q) tile[(lg * 32 + lane) * TS + sub * 32 + q] = zero ? 0.0f : v[q];
                }
                if (last) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty0 + 8 * b);
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");
                const int n0 = nt * BN + h * CW;
                if (EPI == GE_PROX && !pa.Y32) {
                    // Double-float state (8 bytes per pixel): one column pair
                    // per lane, so that each 16-byte state access of a warp is
                    // contiguous; warp ew owns rows ew, ew + 8, ..., ew + 120
                    // and handles them eight at a time, every global load of a
                    // batch issued before its first use.
                    const int c2 = 2 * lane, col2 = n0 + c2;
                    if (col2 < ga->N) {
#pragma unroll 1
                        for (int rl = ew; rl < BM; rl += 64) {
                            size_t idx[8];
                            float g0[8], g1v[8];
                            bool okr[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const int rr = rl + 8 * q, row = m0 + rr;
                                okr[q] = row < ga->rows;
                                idx[q] = (size_t)row * ga->N + col2;
                                g0[q] = tile[rr * TS + c2];
                                g1v[q] = tile[rr * TS + c2 + 1];
                            }
                            prox_momentum2_n<8>(pa, idx, g0, g1v, okr);
                        }
                    }
                    asm volatile("bar.sync 1, 256;" ::: "memory");   // staging tile free again
                    continue;
                }
                const int c = 4 * (lane & 15);   // CW == 64: four columns per lane, 16 lanes per row
                const int col = n0 + c;
                // Warp ew owns rows 2 ew + (lane >> 4) + 16 q (q < 8) of the
                // chunk and handles all eight in one batch, every global load
                // issued before its first use (one memory latency per chunk),
                // with 16-byte loads and stores.
                const int r0 = 2 * ew + (lane >> 4);
                if (col < ga->N) {   // N is a multiple of 8 and col of 4: all four columns inside
                    const int rows = ga->rows, N = ga->N;
                    size_t idx[8];
                    float4 gv[8];
                    bool okr[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int rr = r0 + 16 * q, row = m0 + rr;
                        okr[q] = row < rows;
                        idx[q] = (size_t)row * N + col;
                        const float *tp = tile + rr * TS + c;
                        gv[q] = make_float4(tp[0], tp[1], tp[2], tp[3]);
                    }
                    if (EPI == GE_PROX) {
                        prox_momentum4_n32<8>(pa, idx, gv, okr);   // FP32 state (the other case is above)
                    } else {
                        const int sk = ga->split_kind;
                        void *ohi = ga->out_hi, *olo = ga->out_lo;
                        float4 bb[8];
                        if (EPI == GE_RESID) {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                bb[q] = okr[q] ? __ldg(reinterpret_cast<const float4 *>(ga->Bd + idx[q]))
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (!okr[q]) continue;
                            float4 v = gv[q];
                            if (EPI == GE_SPLIT) {
                                store_split4(ohi, olo, sk, (size_t)term * rows * N + idx[q], v);
                            } else if (EPI == GE_RESID) {
                                v = make_float4(v.x - bb[q].x, v.y - bb[q].y, v.z - bb[q].z, v.w - bb[q].w);
                                store_split4(ohi, olo, sk, idx[q], v);
                            } else {
                                *reinterpret_cast<float4 *>(ga->out_f32 + idx[q]) = v;
                            }
                        }
                    }
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");   // staging tile free again
            }
            if (ep_abort) break;                                  // uniform across the epilogue warps
        }
        if (FMT == FMT_BF16 && (EPI == GE_SPLIT || EPI == GE_RESID) && ew == 0 && lane == 0)
            bulk_wait_all();   // the tensor stores are complete before the CTA exits
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PC::TMEM_COLS)
                     : "memory");
    }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at, so the wait runs out after ~1 s and records DEV_TIMEOUT.
__global__ void wait_timeout_selftest(unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(smem_u32(&bar), 0, status);
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

sfista_status get_encoder() {
    if (g_encode) return SFISTA_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(SFISTA_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return SFISTA_OK;
}

// 3-D tensor [d2][d1][d0] (d0 contiguous), box {kb_elems, box_rows, 1}, 128 B swizzle.
sfista_status make_map(CUtensorMap *map, const void *base, int fmt, int d0, int d1, int d2, int box_rows) {
    if (!base) {
        memset(map, 0, sizeof(*map));
        return SFISTA_OK;
    }
    const size_t es = fmt == FMT_BF16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
    cuuint64_t strides[2] = {(cuuint64_t)d0 * es, (cuuint64_t)d0 * d1 * es};
    cuuint32_t box[3] = {(cuuint32_t)(KB_BYTES / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, fmt == FMT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SFISTA_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SFISTA_OK;
}

struct Operand {
    void *hi = nullptr, *lo = nullptr;
    CUtensorMap map_hi, map_lo;         // boxes of 128 rows (P loads, Q loads with BN = 128, tensor stores)
    CUtensorMap map256_hi, map256_lo;   // Q operands: boxes of 256 rows (BN = 256)
    CUtensorMap map64_hi, map64_lo;     // Q operands: boxes of 64 rows (BN = 64)
};

}  // namespace

struct GemmPath {
    int fmt = FMT_BF16;
    bool split = true, dense = false;
    int split_kind = 1;
    int m = 0, n = 0, r = 0;
    Band bandA, bandB, bandAT, bandBT;   // lo/w only (no host copies of the tables)
    Operand PA, PB, PAT, PBT;            // factor panels (P operands)
    Operand QY, QT, QR, QU;              // Y, Tt, R, Ut (Q operands; Tt/Ut are also outputs)
    const float *Bd = nullptr;
    unsigned *status = nullptr;
    double *dband = nullptr;             // scratch for densify
    int sms = 1;                         // SM count: the persistent grids use one CTA per SM
    // Tile shape of each stage: N tile width (128, or 64 / 256 for the summed
    // stages 1 and 3) and, for the stacked stages 0 and 2, the resident P
    // panel (BF16 band mode only, when every row tile's band spans at most
    // three K blocks: res_ok).
    int bn[4] = {128, 128, 128, 128};
    bool res[4] = {false, false, false, false};
    bool res_ok[4] = {false, false, false, false};
};

namespace {

constexpr int BN_TILE = 128;   // N tile of the grouped launches

template <int FMT, bool SPLIT, int BN, int EPI, bool GROUPED, bool RES>
cudaError_t set_attr1() {
    return cudaFuncSetAttribute(umma_gemm_persistent<FMT, SPLIT, BN, EPI, GROUPED, RES>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, PCfg<FMT, SPLIT, BN, RES>::SMEM);
}

// Every kernel instance the launchers below can select: GE_SPLIT with
// BN = 64 or 128 (streamed or, BF16, resident panel; grouped: 128),
// GE_RESID / GE_PROX / GE_STORE with BN = 64, 128 or 256 (single problems),
// GE_RESID / GE_PROX with 128 (grouped).
template <int FMT, bool SPLIT>
cudaError_t set_attrs() {
    cudaError_t e;
    if ((e = set_attr1<FMT, SPLIT, 128, GE_SPLIT, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 64, GE_SPLIT, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 128, GE_SPLIT, true, false>()) ||
        (e = set_attr1<FMT, SPLIT, 128, GE_RESID, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 256, GE_RESID, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 64, GE_RESID, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 128, GE_RESID, true, false>()) ||
        (e = set_attr1<FMT, SPLIT, 128, GE_PROX, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 256, GE_PROX, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 64, GE_PROX, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 128, GE_PROX, true, false>()) ||
        (e = set_attr1<FMT, SPLIT, 128, GE_STORE, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 256, GE_STORE, false, false>()) ||
        (e = set_attr1<FMT, SPLIT, 64, GE_STORE, false, false>()))
        return e;
    if constexpr (FMT == FMT_BF16) {
        if ((e = set_attr1<FMT, SPLIT, 128, GE_SPLIT, false, true>()) ||
            (e = set_attr1<FMT, SPLIT, 64, GE_SPLIT, false, true>()) ||
            (e = set_attr1<FMT, SPLIT, 128, GE_SPLIT, true, true>()))
            return e;
    }
    return cudaSuccess;
}

// Launch with programmatic stream serialisation (the kernel's prologue may
// overlap the previous kernel's tail; it waits with griddepcontrol.wait).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), int grid, int smem, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(320);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// One persistent launch over the tiles of a stage (one CTA per SM): gy row
// tiles (terms stacked) times ceil(a.N / BN) column tiles.  O: the output
// operand (its tensor maps serve the epilogue's tensor stores), or NULL for
// the stages that write plain FP32 or the FISTA state.
template <int FMT, bool SPLIT, int EPI, int BN, bool RES>
void launch_tiles(const Operand &P, const Operand &Q, const Operand *O, const GemmArgs &a, int gy, int sms,
                  cudaStream_t s) {
    const int gx = (a.N + BN - 1) / BN;
    const int ntiles = gx * gy;
    const int grid = ntiles < sms ? ntiles : sms;
    const Operand &Ou = O ? *O : P;
    const CUtensorMap &qh = BN == 256 ? Q.map256_hi : BN == 64 ? Q.map64_hi : Q.map_hi;
    const CUtensorMap &ql = BN == 256 ? Q.map256_lo : BN == 64 ? Q.map64_lo : Q.map_lo;
    launch_pdl(umma_gemm_persistent<FMT, SPLIT, BN, EPI, false, RES>, grid, PCfg<FMT, SPLIT, BN, RES>::SMEM, s,
               P.map_hi, SPLIT ? P.map_lo : P.map_hi, qh, SPLIT ? ql : qh, Ou.map_hi, SPLIT ? Ou.map_lo : Ou.map_hi,
               a, gx, ntiles, (const CUtensorMap *)nullptr, (const GemmArgs *)nullptr, (const WorkItem *)nullptr,
               0);
}

// The instance for a stage's tile shape (bn, res); shapes without an
// instance (the host never selects them) fall back to BN = 128, streamed.
template <int FMT, bool SPLIT, int EPI>
void launch_shape(const Operand &P, const Operand &Q, const Operand *O, const GemmArgs &a, int gy, int bn, bool res,
                  int sms, cudaStream_t s) {
    if constexpr (EPI == GE_SPLIT && FMT == FMT_BF16) {
        if (res && bn == 64) return launch_tiles<FMT, SPLIT, EPI, 64, true>(P, Q, O, a, gy, sms, s);
        if (res) return launch_tiles<FMT, SPLIT, EPI, 128, true>(P, Q, O, a, gy, sms, s);
    }
    if constexpr (EPI == GE_SPLIT) {
        if (bn == 64) return launch_tiles<FMT, SPLIT, EPI, 64, false>(P, Q, O, a, gy, sms, s);
    }
    if constexpr (EPI != GE_SPLIT) {
        if (bn == 256) return launch_tiles<FMT, SPLIT, EPI, 256, false>(P, Q, O, a, gy, sms, s);
        if (bn == 64) return launch_tiles<FMT, SPLIT, EPI, 64, false>(P, Q, O, a, gy, sms, s);
    }
    launch_tiles<FMT, SPLIT, EPI, 128, false>(P, Q, O, a, gy, sms, s);
}

template <int EPI>
sfista_status dispatch(const GemmPath *g, const Operand &P, const Operand &Q, const Operand *O, const GemmArgs &a,
                       int gy, int bn, bool res, cudaStream_t s) {
    if (g->fmt == FMT_BF16) {
        if (g->split) launch_shape<FMT_BF16, true, EPI>(P, Q, O, a, gy, bn, res, g->sms, s);
        else launch_shape<FMT_BF16, false, EPI>(P, Q, O, a, gy, bn, res, g->sms, s);
    } else {
        if (g->split) launch_shape<FMT_TF32, true, EPI>(P, Q, O, a, gy, bn, res, g->sms, s);
        else launch_shape<FMT_TF32, false, EPI>(P, Q, O, a, gy, bn, res, g->sms, s);
    }
    return SFISTA_OK;
}

GemmArgs base_args(const GemmPath *g) {
    GemmArgs a{};
    a.dense = g->dense ? 1 : 0;
    a.split_kind = g->split_kind;
    a.status = g->status;
    return a;
}

// Stage 0 / 2: out[term][row][col] = sum_k P_term[row][k] Q[col][k] (terms along M).
GemmArgs stacked_args(const GemmPath *g, const Band &band, Operand &Out, int *gy) {
    GemmArgs a = base_args(g);
    a.rows = g->n;
    a.m_tiles = (g->n + BM - 1) / BM;
    a.N = g->m;
    a.K = g->n;
    a.band_lo = band.lo;
    a.band_hi = band.lo + band.w - 1;
    a.segs = 1;
    a.type_b = 0;
    a.out_hi = Out.hi;
    a.out_lo = Out.lo;
    // Large intermediates (beyond a quarter of L2) are tensor-stored with the
    // evict-last priority (measured +2 % per iteration at 2048^2, r = 5; small
    // ones stay in L2 anyway).
    const size_t bytes = (size_t)g->r * g->m * g->n * (g->fmt == FMT_BF16 ? 2 : 4) * (g->split ? 2 : 1);
    a.keep_l2 = bytes > ((size_t)32 << 20) ? 1 : 0;
    *gy = a.m_tiles * g->r;
    return a;
}

// Stage 1 / 3: out[row][col] = sum_{t, k} P_t[row][k] Q_t[col][k] (terms along K).
void summed_args(const GemmPath *g, const Band &band, GemmArgs *a, int *gy) {
    a->rows = g->m;
    a->m_tiles = (g->m + BM - 1) / BM;
    a->N = g->n;
    a->K = g->m;
    a->band_lo = band.lo;
    a->band_hi = band.lo + band.w - 1;
    a->segs = g->r;
    a->type_b = 1;
    *gy = a->m_tiles;
}

// The resident panel applies in band mode only (a dense K range is longer).
bool stage_res(const GemmPath *g, int st) { return g->res[st] && g->res_ok[st] && !g->dense; }

sfista_status run_stacked(const GemmPath *g, int st, const Operand &P, const Band &band, const Operand &Q,
                          Operand &Out, cudaStream_t s) {
    int gy;
    GemmArgs a = stacked_args(g, band, Out, &gy);
    return dispatch<GE_SPLIT>(g, P, Q, &Out, a, gy, g->bn[st], stage_res(g, st), s);
}

template <int EPI>
sfista_status run_summed(const GemmPath *g, int st, const Operand &P, const Band &band, const Operand &Q,
                         const Operand *O, GemmArgs a, cudaStream_t s) {
    int gy;
    summed_args(g, band, &a, &gy);
    return dispatch<EPI>(g, P, Q, O, a, gy, g->bn[st], false, s);
}

// Largest number of K blocks (of kb_elems, start aligned down to `align`)
// that the band range of any row tile of a len x len factor spans; the same
// arithmetic as tile_k_range.
int band_kblocks_max(int len, const Band &band, int align, int kb_elems) {
    int mx = 0;
    for (int m0 = 0; m0 < len; m0 += BM) {
        int lo = std::max(0, m0 + band.lo);
        const int hi = std::min(len, m0 + BM + band.lo + band.w - 1);
        lo = (lo / align) * align;
        mx = std::max(mx, hi > lo ? (hi - lo + kb_elems - 1) / kb_elems : 0);
    }
    return mx;
}

cudaError_t alloc_operand(Operand *o, size_t elems, size_t es, bool split) {
    cudaError_t e = cudaMalloc(&o->hi, elems * es);
    if (e) return e;
    if (split) e = cudaMalloc(&o->lo, elems * es);
    return e;
}

void free_operand(Operand *o) {
    if (o->hi) cudaFree(o->hi);
    if (o->lo) cudaFree(o->lo);
    o->hi = o->lo = nullptr;
}

}  // namespace

sfista_status gemm_create(GemmPath **out, const HostSetup &h, int prec, bool dense, unsigned *status,
                          cudaStream_t s) {
    *out = nullptr;
    if (prec == SFISTA_FP32) return fail(SFISTA_ENOTSUP, "the GEMM operator form runs on the tensor cores (TF32/BF16)");
    if (h.m % 8 || h.n % 8)
        return fail(SFISTA_ENOTSUP, "tensor-core operator needs image sizes that are multiples of 8");
    sfista_status st = get_encoder();
    if (st) return st;
    GemmPath *g = new (std::nothrow) GemmPath();
    if (!g) return fail(SFISTA_ENOMEM, "GEMM path allocation failed");
    g->fmt = (prec == SFISTA_BF16 || prec == SFISTA_BF16X3) ? FMT_BF16 : FMT_TF32;
    g->split = (prec == SFISTA_BF16X3 || prec == SFISTA_TF32X3);
    g->split_kind = g->fmt == FMT_BF16 ? 1 : 2;
    g->dense = dense;
    g->status = status;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g->sms < 1)
            g->sms = 1;
    }
    g->m = h.m;
    g->n = h.n;
    g->r = h.r;
    auto meta = [](const Band &b) {
        Band o;
        o.len = b.len;
        o.r = b.r;
        o.lo = b.lo;
        o.w = b.w;
        return o;
    };
    g->bandA = meta(h.A);
    g->bandB = meta(h.B);
    g->bandAT = meta(h.AT);
    g->bandBT = meta(h.BT);
    const size_t es = g->fmt == FMT_BF16 ? 2 : 4;
    const size_t m = h.m, n = h.n, r = h.r;
    cudaError_t e = cudaSuccess;
    auto bail = [&](sfista_status x) {
        gemm_destroy(g);
        return x;
    };
    if ((e = alloc_operand(&g->PA, r * n * n, es, g->split)) || (e = alloc_operand(&g->PAT, r * n * n, es, g->split)) ||
        (e = alloc_operand(&g->PB, r * m * m, es, g->split)) || (e = alloc_operand(&g->PBT, r * m * m, es, g->split)) ||
        (e = alloc_operand(&g->QY, m * n, es, g->split)) || (e = alloc_operand(&g->QT, r * n * m, es, g->split)) ||
        (e = alloc_operand(&g->QR, m * n, es, g->split)) || (e = alloc_operand(&g->QU, r * n * m, es, g->split)))
        return bail(fail(SFISTA_ENOMEM, std::string("GEMM operand buffers: ") + cudaGetErrorString(e)));
    if (g->fmt == FMT_BF16) e = g->split ? set_attrs<FMT_BF16, true>() : set_attrs<FMT_BF16, false>();
    else e = g->split ? set_attrs<FMT_TF32, true>() : set_attrs<FMT_TF32, false>();
    if (e) return bail(fail(SFISTA_ECUDA, std::string("GEMM smem attribute: ") + cudaGetErrorString(e)));
    // Dense factor panels from the band tables, in the operand format.
    const int kind = g->fmt == FMT_BF16 ? 1 : 2;
    auto dens = [&](const Band &b, Operand &o) -> cudaError_t {
        cudaError_t ee = cudaMalloc((void **)&g->dband, b.band.size() * sizeof(double));
        if (ee) return ee;
        ee = cudaMemcpyAsync(g->dband, b.band.data(), b.band.size() * sizeof(double), cudaMemcpyHostToDevice, s);
        if (!ee) launch_densify(g->dband, b.r, b.len, b.lo, b.w, b.len, kind, o.hi, g->split ? o.lo : nullptr, b.len, s);
        if (!ee) ee = cudaGetLastError();
        if (!ee) ee = cudaStreamSynchronize(s);
        cudaFree(g->dband);
        g->dband = nullptr;
        return ee;
    };
    if ((e = dens(h.A, g->PA)) || (e = dens(h.AT, g->PAT)) || (e = dens(h.B, g->PB)) || (e = dens(h.BT, g->PBT)))
        return bail(fail(SFISTA_ECUDA, std::string("factor panels: ") + cudaGetErrorString(e)));
    // Tensor maps: P operands (box rows BM), Q operands (box rows BN).
    struct M {
        Operand *o;
        int d0, d1, d2, rows;
    } maps[] = {
        {&g->PA, (int)n, (int)n, (int)r, BM},  {&g->PAT, (int)n, (int)n, (int)r, BM},
        {&g->PB, (int)m, (int)m, (int)r, BM},  {&g->PBT, (int)m, (int)m, (int)r, BM},
        {&g->QY, (int)n, (int)m, 1, BN_TILE},  {&g->QR, (int)n, (int)m, 1, BN_TILE},
        {&g->QT, (int)m, (int)n, (int)r, BN_TILE}, {&g->QU, (int)m, (int)n, (int)r, BN_TILE},
    };
    for (auto &mm : maps) {
        if ((st = make_map(&mm.o->map_hi, mm.o->hi, g->fmt, mm.d0, mm.d1, mm.d2, mm.rows))) return bail(st);
        if ((st = make_map(&mm.o->map_lo, mm.o->lo, g->fmt, mm.d0, mm.d1, mm.d2, mm.rows))) return bail(st);
    }
    // Q operands with BN = 256 (summed stages) or 64 (all stages): boxes of 256 / 64 rows.
    for (Operand *o : {&g->QT, &g->QU}) {
        if ((st = make_map(&o->map256_hi, o->hi, g->fmt, (int)m, (int)n, (int)r, 256))) return bail(st);
        if ((st = make_map(&o->map256_lo, o->lo, g->fmt, (int)m, (int)n, (int)r, 256))) return bail(st);
    }
    for (Operand *o : {&g->QT, &g->QU, &g->QY, &g->QR}) {
        const int d0 = (o == &g->QY || o == &g->QR) ? (int)n : (int)m, d1 = (o == &g->QY || o == &g->QR) ? (int)m : (int)n;
        const int d2 = (o == &g->QY || o == &g->QR) ? 1 : (int)r;
        if ((st = make_map(&o->map64_hi, o->hi, g->fmt, d0, d1, d2, 64))) return bail(st);
        if ((st = make_map(&o->map64_lo, o->lo, g->fmt, d0, d1, d2, 64))) return bail(st);
    }
    for (Operand *o : {&g->QY, &g->QR}) {
        o->map256_hi = o->map_hi;
        o->map256_lo = o->map_lo;
    }
    // Resident P panels for the stacked stages: allowed in BF16 band mode when
    // every row tile's band lies within three K blocks of 64 (off by default;
    // the context's options or the tuner switch them on).
    if (g->fmt == FMT_BF16) {
        using CB = Cfg<FMT_BF16, true, 128>;
        constexpr int kres = PCfg<FMT_BF16, true, 128, true>::RES_KB;
        g->res_ok[0] = band_kblocks_max((int)n, h.A, CB::ALIGN, CB::KB_ELEMS) <= kres;
        g->res_ok[2] = band_kblocks_max((int)n, h.AT, CB::ALIGN, CB::KB_ELEMS) <= kres;
    }
    *out = g;
    return SFISTA_OK;
}

void launch_wait_timeout_selftest(unsigned *status, cudaStream_t s) {
    wait_timeout_selftest<<<1, 32, 0, s>>>(status);
}

void gemm_set_dense(GemmPath *g, bool dense) { g->dense = dense; }

int gemm_tile_options(const GemmPath *g, int st, int *bn, int *res) {
    int n = 0;
    if (st == 0 || st == 2) {
        for (int w : {128, 64}) {
            bn[n] = w, res[n++] = 0;
            if (g->res_ok[st] && !g->dense) bn[n] = w, res[n++] = 1;
        }
    } else {
        bn[n] = 64, res[n++] = 0;
        bn[n] = 128, res[n++] = 0;
        bn[n] = 256, res[n++] = 0;
    }
    return n;
}

void gemm_set_tile(GemmPath *g, int st, int bn, int res) {
    if (st == 0 || st == 2) {
        g->bn[st] = bn == 64 ? 64 : 128;
        g->res[st] = res && g->res_ok[st];
    } else {
        g->bn[st] = bn == 256 || bn == 64 ? bn : 128;
        g->res[st] = false;
    }
}

int gemm_default_bn(const GemmPath *g, int st) {
    const int mt = (st % 2 == 0) ? ((g->n + BM - 1) / BM) * g->r : (g->m + BM - 1) / BM;
    const int N = (st % 2 == 0) ? g->m : g->n;
    return (long)mt * ((N + 127) / 128) < g->sms ? 64 : 128;
}

void gemm_get_tile(const GemmPath *g, int st, int *bn, int *res) {
    *bn = g->bn[st];
    *res = stage_res(g, st) ? 1 : 0;
}

void gemm_destroy(GemmPath *g) {
    if (!g) return;
    for (Operand *o : {&g->PA, &g->PB, &g->PAT, &g->PBT, &g->QY, &g->QT, &g->QR, &g->QU}) free_operand(o);
    if (g->dband) cudaFree(g->dband);
    delete g;
}

void gemm_state_operands(GemmPath *g, void **yhi, void **ylo, int *split_kind) {
    *yhi = g->QY.hi;
    *ylo = g->split ? g->QY.lo : nullptr;
    *split_kind = g->split_kind;
}

void gemm_prepare_solve(GemmPath *g, const float *Bd, cudaStream_t) { g->Bd = Bd; }

void gemm_stage(GemmPath *g, int st, const ProxArgs &pa_in, cudaStream_t s) {
    switch (st) {
        case 0:
            run_stacked(g, 0, g->PA, g->bandA, g->QY, g->QT, s);
            break;
        case 1: {
            GemmArgs a = base_args(g);
            a.Bd = g->Bd;
            a.out_hi = g->QR.hi;
            a.out_lo = g->QR.lo;
            run_summed<GE_RESID>(g, 1, g->PB, g->bandB, g->QT, &g->QR, a, s);
            break;
        }
        case 2:
            run_stacked(g, 2, g->PAT, g->bandAT, g->QR, g->QU, s);
            break;
        default: {
            GemmArgs a = base_args(g);
            a.pa = pa_in;
            a.pa.Yop = nullptr;   // the tensor-core operands are the split copies
            a.pa.Yhi = g->QY.hi;
            a.pa.Ylo = g->split ? g->QY.lo : nullptr;
            a.pa.split_kind = g->split_kind;
            a.status = pa_in.status;
            run_summed<GE_PROX>(g, 3, g->PBT, g->bandBT, g->QU, nullptr, a, s);
            break;
        }
    }
}

// ------------------------------------------------------------------ grouped (batched) launches
struct GemmBatch {
    int nprob = 0, fmt = FMT_BF16, sms = 1;
    bool split = true;
    std::vector<GemmPath *> paths;
    CUtensorMap *d_maps[4] = {nullptr, nullptr, nullptr, nullptr};   // per stage: nprob x 6 (P, Q, output)
    GemmArgs *d_args[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<GemmArgs> h_args[4];
    WorkItem *d_work[4] = {nullptr, nullptr, nullptr, nullptr};
    int nwork[4] = {0, 0, 0, 0};
    // Stages 0 and 2 with resident P panels: allowed when every problem
    // allows them (BF16 band mode, bands within three K blocks).
    bool res = false, res_ok = false;
};

void gemm_batch_destroy(GemmBatch *b) {
    if (!b) return;
    for (int st = 0; st < 4; ++st) {
        if (b->d_maps[st]) cudaFree(b->d_maps[st]);
        if (b->d_args[st]) cudaFree(b->d_args[st]);
        if (b->d_work[st]) cudaFree(b->d_work[st]);
    }
    delete b;
}

sfista_status gemm_batch_create(GemmBatch **out, GemmPath *const *paths, int nprob, cudaStream_t s) {
    *out = nullptr;
    if (nprob < 1) return fail(SFISTA_EINVAL, "empty batch");
    GemmBatch *b = new (std::nothrow) GemmBatch();
    if (!b) return fail(SFISTA_ENOMEM, "batch allocation failed");
    b->nprob = nprob;
    b->sms = paths[0]->sms;
    b->fmt = paths[0]->fmt;
    b->split = paths[0]->split;
    b->paths.assign(paths, paths + nprob);
    for (int p = 0; p < nprob; ++p)
        if (paths[p]->fmt != b->fmt || paths[p]->split != b->split) {
            gemm_batch_destroy(b);
            return fail(SFISTA_EINVAL, "all problems of a batch need the same precision");
        }
    // Problems in decreasing order of work so the largest tiles start first.
    std::vector<int> order(nprob);
    for (int p = 0; p < nprob; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const GemmPath *a = paths[x], *c = paths[y];
        return (double)a->m * a->n * a->r > (double)c->m * c->n * c->r;
    });
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < 4 && !e; ++st) {
        std::vector<CUtensorMap> maps(6 * (size_t)nprob);
        std::vector<WorkItem> work;
        b->h_args[st].resize(nprob);
        for (int p = 0; p < nprob; ++p) {
            GemmPath *g = paths[p];
            const Operand *P = nullptr, *Q = nullptr;
            int gy = 0;
            GemmArgs a{};
            if (st == 0) {
                a = stacked_args(g, g->bandA, g->QT, &gy);
                P = &g->PA;
                Q = &g->QY;
            } else if (st == 1) {
                a = base_args(g);
                a.out_hi = g->QR.hi;
                a.out_lo = g->QR.lo;
                summed_args(g, g->bandB, &a, &gy);
                P = &g->PB;
                Q = &g->QT;
            } else if (st == 2) {
                a = stacked_args(g, g->bandAT, g->QU, &gy);
                P = &g->PAT;
                Q = &g->QR;
            } else {
                a = base_args(g);
                summed_args(g, g->bandBT, &a, &gy);
                P = &g->PBT;
                Q = &g->QU;
            }
            b->h_args[st][p] = a;
            const Operand *O = st == 0 ? &g->QT : st == 1 ? &g->QR : st == 2 ? &g->QU : P;
            maps[6 * p + 0] = P->map_hi;
            maps[6 * p + 1] = b->split ? P->map_lo : P->map_hi;
            maps[6 * p + 2] = Q->map_hi;
            maps[6 * p + 3] = b->split ? Q->map_lo : Q->map_hi;
            maps[6 * p + 4] = O->map_hi;
            maps[6 * p + 5] = b->split ? O->map_lo : O->map_hi;
        }
        for (int p : order) {
            GemmPath *g = paths[p];
            int gx = 0, gy = 0;
            if (st == 0 || st == 2) {
                gx = (g->m + BN_TILE - 1) / BN_TILE;
                gy = ((g->n + BM - 1) / BM) * g->r;
            } else {
                gx = (g->n + BN_TILE - 1) / BN_TILE;
                gy = (g->m + BM - 1) / BM;
            }
            for (int mt = 0; mt < gy; ++mt)
                for (int nt = 0; nt < gx; ++nt) work.push_back(WorkItem{p, mt, nt, 0});
        }
        b->nwork[st] = (int)work.size();
        if ((e = cudaMalloc((void **)&b->d_maps[st], maps.size() * sizeof(CUtensorMap)))) break;
        if ((e = cudaMalloc((void **)&b->d_args[st], nprob * sizeof(GemmArgs)))) break;
        if ((e = cudaMalloc((void **)&b->d_work[st], work.size() * sizeof(WorkItem)))) break;
        if ((e = cudaMemcpyAsync(b->d_maps[st], maps.data(), maps.size() * sizeof(CUtensorMap),
                                 cudaMemcpyHostToDevice, s)))
            break;
        if ((e = cudaMemcpyAsync(b->d_work[st], work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                 s)))
            break;
        e = cudaStreamSynchronize(s);
    }
    if (e) {
        gemm_batch_destroy(b);
        return fail(SFISTA_ENOMEM, std::string("batch tables: ") + cudaGetErrorString(e));
    }
    // Resident panels when every problem allows them, and by default when
    // every problem's own stages use them.
    b->res_ok = b->fmt == FMT_BF16;
    b->res = true;
    for (const GemmPath *g : b->paths) {
        b->res_ok = b->res_ok && g->res_ok[0] && g->res_ok[2] && !g->dense;
        b->res = b->res && g->res[0] && g->res[2];
    }
    b->res = b->res && b->res_ok;
    *out = b;
    return SFISTA_OK;
}

bool gemm_batch_res_ok(const GemmBatch *b) { return b->res_ok; }
void gemm_batch_set_res(GemmBatch *b, bool res) { b->res = res && b->res_ok; }

// Per solve: observation pointers and the prox arguments of every problem
// (pa.Xin / pa.Xout hold the problem's state buffers 0 / 1).
sfista_status gemm_batch_bind(GemmBatch *b, const float *const *Bds, const ProxArgs *pas, cudaStream_t s) {
    for (int p = 0; p < b->nprob; ++p) {
        GemmPath *g = b->paths[p];
        b->h_args[1][p].Bd = Bds[p];
        GemmArgs &a = b->h_args[3][p];
        a.pa = pas[p];
        a.pa.Yop = nullptr;
        a.pa.Yhi = g->QY.hi;
        a.pa.Ylo = g->split ? g->QY.lo : nullptr;
        a.pa.split_kind = g->split_kind;
        a.status = pas[p].status;
        for (int st = 0; st < 4; ++st) b->h_args[st][p].status = pas[p].status;
    }
    for (int st = 0; st < 4; ++st) {
        cudaError_t e = cudaMemcpyAsync(b->d_args[st], b->h_args[st].data(), b->nprob * sizeof(GemmArgs),
                                        cudaMemcpyHostToDevice, s);
        if (e) return fail(SFISTA_ECUDA, std::string("batch args: ") + cudaGetErrorString(e));
    }
    return SFISTA_OK;
}

namespace {
template <int FMT, bool SPLIT, int EPI, bool RES>
void launch_grouped(const GemmBatch *b, int st, int k, cudaStream_t s) {
    const int grid = b->nwork[st] < b->sms ? b->nwork[st] : b->sms;
    // The parameter-space maps are unused in grouped mode: pass the first problem's.
    const Operand &P0 = b->paths[0]->PA;
    launch_pdl(umma_gemm_persistent<FMT, SPLIT, BN_TILE, EPI, true, RES>, grid,
               PCfg<FMT, SPLIT, BN_TILE, RES>::SMEM, s, P0.map_hi, P0.map_hi, P0.map_hi, P0.map_hi, P0.map_hi,
               P0.map_hi, b->h_args[st][0], 1, b->nwork[st], (const CUtensorMap *)b->d_maps[st],
               (const GemmArgs *)b->d_args[st], (const WorkItem *)b->d_work[st], k);
}
template <int FMT, bool SPLIT>
void grouped_stage(const GemmBatch *b, int st, int k, cudaStream_t s) {
    if (st == 0 || st == 2) {
        if constexpr (FMT == FMT_BF16) {
            if (b->res) return launch_grouped<FMT, SPLIT, GE_SPLIT, true>(b, st, k, s);
        }
        launch_grouped<FMT, SPLIT, GE_SPLIT, false>(b, st, k, s);
    } else if (st == 1) {
        launch_grouped<FMT, SPLIT, GE_RESID, false>(b, st, k, s);
    } else {
        launch_grouped<FMT, SPLIT, GE_PROX, false>(b, st, k, s);
    }
}
}  // namespace

void gemm_batch_stage(GemmBatch *b, int st, int k, cudaStream_t s) {
    if (b->fmt == FMT_BF16) b->split ? grouped_stage<FMT_BF16, true>(b, st, k, s) : grouped_stage<FMT_BF16, false>(b, st, k, s);
    else b->split ? grouped_stage<FMT_TF32, true>(b, st, k, s) : grouped_stage<FMT_TF32, false>(b, st, k, s);
}

int gemm_batch_launches_per_iteration(const GemmBatch *) { return 4; }

void gemm_residual_operand(GemmPath *g, const float *R, cudaStream_t s) {
    launch_split(R, g->QR.hi, g->split ? g->QR.lo : nullptr, (size_t)g->m * g->n, g->split_kind, s);
}

sfista_status gemm_apply(GemmPath *g, const float *x, float *y, int transpose, cudaStream_t s) {
    const size_t N = (size_t)g->m * g->n;
    Operand &in = transpose ? g->QR : g->QY;
    launch_split(x, in.hi, g->split ? in.lo : nullptr, N, g->split_kind, s);
    GemmArgs a = base_args(g);
    a.out_f32 = y;
    sfista_status st;
    if (!transpose) {
        if ((st = run_stacked(g, 0, g->PA, g->bandA, g->QY, g->QT, s))) return st;
        st = run_summed<GE_STORE>(g, 1, g->PB, g->bandB, g->QT, nullptr, a, s);
    } else {
        if ((st = run_stacked(g, 2, g->PAT, g->bandAT, g->QR, g->QU, s))) return st;
        st = run_summed<GE_STORE>(g, 3, g->PBT, g->bandBT, g->QU, nullptr, a, s);
    }
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e) return fail(SFISTA_ECUDA, std::string("GEMM launch: ") + cudaGetErrorString(e));
    return SFISTA_OK;
}

}  // namespace sfista
