// Banded Kronecker operator on the CUDA cores, plus the fused FISTA epilogue.
//
// The factors of Sec. 2 are banded (Toeplitz, plus Hankel corners for the
// reflective boundary), so each product of Alg. 2, Step 1 is a 1-D banded
// matrix applied along one image axis:
//   rows pass:  Z_i[a][c] = sum_k In[a][c + lo + k] * F_i[c][c + lo + k]
//               (In A_i^T with F = A, or In A_i with F = A^T)
//   cols pass:  Out[a][c] = sum_i sum_k G_i[a][a + lo + k] * Z_i[a + lo + k][c]
//               (B_i Z_i with G = B, or B_i^T Z_i with G = B^T)
// Band entries come from compact storage band[(i*w + k)*len + row], so the
// zero and reflective boundaries (and any PSF centre) run the same code.
// The cols pass ends in the fused epilogue: the residual B_s(Y) - B of the
// forward product, or Step 1's shrink + optional projection + Step 3's
// momentum for the adjoint, with the FISTA state as double-float pairs.
#include <cuda_bf16.h>

#include <type_traits>

#include "band_items.cuh"
#include "band_items4.cuh"
#include "epilogue.cuh"
#include "internal.h"

namespace sfista {

namespace {

template <typename T>
__global__ void __launch_bounds__(band::NT) band_rows_kernel(const T *__restrict__ In, int m, int n,
                                                            const T *__restrict__ Fb, int lo, int w, int r, int chunk,
                                                            T *__restrict__ Z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int t0 = blockIdx.z * chunk;
    band::rows_item<T, false>(In, m, n, Fb, lo, w, t0, min(chunk, r - t0), blockIdx.y * band::TA,
                              blockIdx.x * band::TC, Z, sm);
}

template <typename T, int EPI>
__global__ void __launch_bounds__(band::NT) band_cols_kernel(const T *__restrict__ Z, int m, int n,
                                                            const T *__restrict__ Gb, int lo, int w, int r, int chunk,
                                                            T *__restrict__ Out, ProxArgs pa) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    band::cols_item<T, EPI, false>(Z, m, n, r, chunk, Gb, lo, w, blockIdx.y * band::TA, blockIdx.x * band::TC, Out,
                                   pa, sm);
}

// FP32 kernels with 16-byte accesses, one RT x 32 tile per block.
template <int RT>
__global__ void __launch_bounds__(band::NT) band_rows_kernel4(const float *__restrict__ In, int m, int n,
                                                             const float *__restrict__ Fb, int lo, int w, int r,
                                                             int chunk, float *__restrict__ Z) {
    extern __shared__ __align__(16) float sm4[];
    const int t0 = blockIdx.z * chunk;
    band4::rows_item<RT>(In, m, n, Fb, lo, w, t0, min(chunk, r - t0), blockIdx.y * RT, blockIdx.x * band::TC, Z,
                         sm4);
}

template <int EPI, int RT>
__global__ void __launch_bounds__(band::NT) band_cols_kernel4(const float *__restrict__ Z, int m, int n,
                                                             const float *__restrict__ Gb, int lo, int w, int r,
                                                             int chunk, float *__restrict__ Out, ProxArgs pa) {
    extern __shared__ __align__(16) float sm4[];
    band4::cols_item<EPI, RT>(Z, m, n, r, chunk, Gb, lo, w, blockIdx.y * RT, blockIdx.x * band::TC, Out, pa, sm4);
}

// Columns pass on 128 x 32 tiles, two columns per thread.  The prox
// instantiation is held to three blocks per SM (80 registers, a few spilled
// around the epilogue): measured faster than two blocks without spills.
template <int EPI>
__global__ void __launch_bounds__(band::NT, EPI == EPI_PROX ? 3 : 0) band_cols_kernel128(const float *__restrict__ Z, int m, int n,
                                                               const float *__restrict__ Gb, int lo, int w, int r,
                                                               int chunk, float *__restrict__ Out, ProxArgs pa) {
    extern __shared__ __align__(16) float sm4[];
    band4::cols_item128<EPI>(Z, m, n, r, chunk, Gb, lo, w, blockIdx.y * 128, blockIdx.x * band::TC, Out, pa, sm4);
}

// Out + i * m * n = G_i In for each term i = blockIdx.z (terms not summed).
template <int RT>
__global__ void __launch_bounds__(band::NT) band_cols_each_kernel4(const float *__restrict__ In, int m, int n,
                                                                  const float *__restrict__ Gb, int lo, int w,
                                                                  float *__restrict__ Out) {
    extern __shared__ __align__(16) float sm4[];
    const size_t t = blockIdx.z;
    ProxArgs pa{};
    band4::cols_item<EPI_STORE, RT>(In, m, n, 1, 1, Gb + t * w * m, lo, w, blockIdx.y * RT, blockIdx.x * band::TC,
                                    Out + t * m * n, pa, sm4);
}
__global__ void __launch_bounds__(band::NT) band_cols_each_kernel(const float *__restrict__ In, int m, int n,
                                                                 const float *__restrict__ Gb, int lo, int w,
                                                                 float *__restrict__ Out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t t = blockIdx.z;
    ProxArgs pa{};
    band::cols_item<float, EPI_STORE, false>(In, m, n, 1, 1, Gb + t * w * m, lo, w, blockIdx.y * band::TA,
                                             blockIdx.x * band::TC, Out + t * m * n, pa,
                                             reinterpret_cast<float *>(smem_raw));
}

constexpr size_t kBandSmemBudget = 96 * 1024;
constexpr size_t kBandSmemMax = 227 * 1024;

// Shared memory of a rows (cols) block with `chunk` terms: the 16-byte FP32
// layout with rt-row tiles (rt = 32 or 64), or the scalar one (rt = 0).
template <typename T>
size_t rows_bytes(int rt, int w, int chunk) {
    return rt ? band4::rows_smem(rt, w, chunk) : band::rows_smem<T>(w, chunk);
}
template <typename T>
size_t cols_bytes(int rt, int w, int chunk) {
    return rt ? band4::cols_smem(rt, w, chunk) : band::cols_smem<T>(w, chunk);
}

// Terms staged per load phase so that a block stays within the budget.
template <typename T>
int rows_chunk(int rt, int r, int w) {
    const size_t fixed = rows_bytes<T>(rt, w, 0), per = rows_bytes<T>(rt, w, 1) - fixed;
    int c = fixed < kBandSmemBudget ? (int)((kBandSmemBudget - fixed) / per) : 1;
    return c < 1 ? 1 : (c > r ? r : c);
}
template <typename T>
int cols_chunk(int rt, int r, int w) {
    int c = (int)(kBandSmemBudget / cols_bytes<T>(rt, w, 1));
    return c < 1 ? 1 : (c > r ? r : c);
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    }
    return sms;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

// Launch with programmatic stream serialisation: the kernel may start (and
// stage its constant band tables) while the previous kernel in the stream
// finishes; it waits (griddepcontrol.wait) before reading that kernel's output.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(band::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// The 16-byte FP32 path runs when m and n are multiples of 4 and every buffer
// is 16-byte aligned; its tiles are 64 rows high when that still gives at
// least two tiles per SM, else 32.  Returns 0 for the scalar path.
template <typename T>
int vec_rows(int m, int n, const void *a, const void *b, const void *c) {
    if (!(std::is_same<T, float>::value && m % 4 == 0 && n % 4 == 0 && aligned16(a) && aligned16(b) && aligned16(c)))
        return 0;
    return band4::tiles(64, m, n) >= 2 * sm_count() ? 64 : 32;
}

template <typename T>
void launch_band_rows(const T *In, int m, int n, const T *Fb, int lo, int w, int r, T *Z, cudaStream_t s, int req) {
    const int rt = vec_rows<T>(m, n, In, Fb, Z);
    int chunk = req > 0 ? std::min(req, r) : rows_chunk<T>(rt, r, w);
    if (rows_bytes<T>(rt, w, chunk) > kBandSmemMax) chunk = rows_chunk<T>(rt, r, w);
    const int ta = rt ? rt : band::TA;
    dim3 grid((n + band::TC - 1) / band::TC, (m + ta - 1) / ta, (r + chunk - 1) / chunk);
    const size_t sm = rows_bytes<T>(rt, w, chunk);
    if constexpr (std::is_same<T, float>::value) {
        if (rt == 64) return launch_pdl(band_rows_kernel4<64>, grid, sm, s, In, m, n, Fb, lo, w, r, chunk, Z);
        if (rt == 32) return launch_pdl(band_rows_kernel4<32>, grid, sm, s, In, m, n, Fb, lo, w, r, chunk, Z);
    }
    launch_pdl(band_rows_kernel<T>, grid, sm, s, In, m, n, Fb, lo, w, r, chunk, Z);
}

template <int RT>
void launch_cols4(dim3 grid, size_t sm, cudaStream_t s, const float *Z, int m, int n, const float *Gb, int lo, int w,
                  int r, int chunk, EpiKind epi, float *Out, const ProxArgs &pa) {
    if (epi == EPI_STORE)
        launch_pdl(band_cols_kernel4<EPI_STORE, RT>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
    else if (epi == EPI_RESIDUAL)
        launch_pdl(band_cols_kernel4<EPI_RESIDUAL, RT>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
    else
        launch_pdl(band_cols_kernel4<EPI_PROX, RT>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
}

// Row height of the columns pass: 128 when the 16-byte path has 64-row tiles
// and 128-row tiles still give two per SM, else that of the rows pass.
template <typename T>
int cols_rows(int m, int n, const void *a, const void *b, const void *c) {
    const int rt = vec_rows<T>(m, n, a, b, c);
    return rt == 64 && band4::tiles(128, m, n) >= 2 * sm_count() ? 128 : rt;
}

template <typename T>
void launch_band_cols(const T *Z, int m, int n, const T *Gb, int lo, int w, int r, EpiKind epi, T *Out,
                      const ProxArgs &pa, cudaStream_t s, int req) {
    const int rt = cols_rows<T>(m, n, Z, Gb, Out ? (const void *)Out : (const void *)Z);
    int chunk = req > 0 ? std::min(req, r) : cols_chunk<T>(rt, r, w);
    if (cols_bytes<T>(rt, w, chunk) > kBandSmemMax) chunk = cols_chunk<T>(rt, r, w);
    const int ta = rt ? rt : band::TA;
    dim3 grid((n + band::TC - 1) / band::TC, (m + ta - 1) / ta);
    const size_t sm = cols_bytes<T>(rt, w, chunk);
    if constexpr (std::is_same<T, float>::value) {
        if (rt == 128) {
            if (epi == EPI_STORE)
                return launch_pdl(band_cols_kernel128<EPI_STORE>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
            if (epi == EPI_RESIDUAL)
                return launch_pdl(band_cols_kernel128<EPI_RESIDUAL>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out,
                                  pa);
            return launch_pdl(band_cols_kernel128<EPI_PROX>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
        }
        if (rt == 64) return launch_cols4<64>(grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, epi, Out, pa);
        if (rt == 32) return launch_cols4<32>(grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, epi, Out, pa);
    }
    if (epi == EPI_STORE)
        launch_pdl(band_cols_kernel<T, EPI_STORE>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
    else if (epi == EPI_RESIDUAL)
        launch_pdl(band_cols_kernel<T, EPI_RESIDUAL>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
    else
        launch_pdl(band_cols_kernel<T, EPI_PROX>, grid, sm, s, Z, m, n, Gb, lo, w, r, chunk, Out, pa);
}

void launch_band_cols_each(const float *In, int m, int n, const float *Gb, int lo, int w, int r, float *Out,
                           cudaStream_t s) {
    const int rt = vec_rows<float>(m, n, In, Gb, Out);
    const int ta = rt ? rt : band::TA;
    dim3 grid((n + band::TC - 1) / band::TC, (m + ta - 1) / ta, r);
    const size_t sm = cols_bytes<float>(rt, w, 1);
    if (rt == 64) return launch_pdl(band_cols_each_kernel4<64>, grid, sm, s, In, m, n, Gb, lo, w, Out);
    if (rt == 32) return launch_pdl(band_cols_each_kernel4<32>, grid, sm, s, In, m, n, Gb, lo, w, Out);
    launch_pdl(band_cols_each_kernel, grid, sm, s, In, m, n, Gb, lo, w, Out);
}

size_t band_smem_f32(bool rows, int w, int chunk) {   // the largest of the layouts
    size_t b = 0;
    for (int rt : {0, 32, 64, 128})
        if (rt < 128 || !rows) b = std::max(b, rows ? rows_bytes<float>(rt, w, chunk) : cols_bytes<float>(rt, w, chunk));
    return b;
}

int band_rows_chunk_limit(int r, int w) {
    int c = r;
    while (c > 1 && band_smem_f32(true, w, c) > kBandSmemMax) --c;
    return c;
}
int band_cols_chunk_limit(int r, int w) {
    int c = r;
    while (c > 1 && band_smem_f32(false, w, c) > kBandSmemMax) --c;
    return c;
}

size_t band_rows_smem(int w, size_t elem) {
    return elem == 8 ? band::rows_smem<double>(w, 1) : band::rows_smem<float>(w, 1);
}
size_t band_cols_smem(int w, size_t elem) {
    return elem == 8 ? band::cols_smem<double>(w, 1) : band::cols_smem<float>(w, 1);
}

// Allows the banded kernels the largest dynamic shared memory a block may
// use; fails if even one term of width w does not fit.
cudaError_t band_set_smem_limits(int w) {
    if (band_rows_smem(w, 8) > kBandSmemMax || band_cols_smem(w, 8) > kBandSmemMax) return cudaErrorInvalidValue;
    const int lim = (int)kBandSmemMax;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(band_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    for (auto k : {band_cols_each_kernel4<32>, band_cols_each_kernel4<64>, band_cols_each_kernel})
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    for (auto k : {band_rows_kernel4<32>, band_rows_kernel4<64>})
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    for (auto k : {band_cols_kernel4<EPI_STORE, 32>, band_cols_kernel4<EPI_RESIDUAL, 32>, band_cols_kernel4<EPI_PROX, 32>,
                   band_cols_kernel4<EPI_STORE, 64>, band_cols_kernel4<EPI_RESIDUAL, 64>, band_cols_kernel4<EPI_PROX, 64>,
                   band_cols_kernel128<EPI_STORE>, band_cols_kernel128<EPI_RESIDUAL>, band_cols_kernel128<EPI_PROX>})
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(band_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(band_cols_kernel<float, EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(band_cols_kernel<float, EPI_RESIDUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(band_cols_kernel<float, EPI_PROX>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(band_cols_kernel<double, EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    return cudaSuccess;
}

template void launch_band_rows<float>(const float *, int, int, const float *, int, int, int, float *, cudaStream_t, int);
template void launch_band_rows<double>(const double *, int, int, const double *, int, int, int, double *, cudaStream_t,
                                       int);
template void launch_band_cols<float>(const float *, int, int, const float *, int, int, int, EpiKind, float *,
                                      const ProxArgs &, cudaStream_t, int);
template void launch_band_cols<double>(const double *, int, int, const double *, int, int, int, EpiKind, double *,
                                       const ProxArgs &, cudaStream_t, int);

// ------------------------------------------------------------------ helpers
namespace {

__global__ void fill_f64_kernel(double *p, size_t count, double v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void f64_to_f32_kernel(const double *in, float *out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
__global__ void df_to_f32_kernel(const float2 *in, float *out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = dfp::to_float(in[i]);
}
__global__ void f32_to_df_kernel(const float *in, float2 *out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2(in[i], 0.0f);
}
__global__ void df_to_f64_kernel(const float2 *in, double *out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = dfp::to_double(in[i]);
}
__global__ void f64_to_df_kernel(const double *in, float2 *out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = dfp::from_double(in[i]);
}
__global__ void f32_to_f64_kernel(const float *in, double *out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}
__global__ void check_finite_kernel(const float *in, size_t count, unsigned *status) {
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite(in[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, DEV_NONFINITE);
}
// Deterministic positive start vector for the power iteration: a 64-bit
// integer hash of the pixel index mapped to [0.5, 1.5).
__global__ void seed_image_kernel(double *v, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = 0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
}
// partial[b*2 + {0,1}] = block sums of u.v and v.v; fixed grid => deterministic.
__global__ void dots_kernel(const double *u, const double *v, size_t count, double *partial) {
    __shared__ double s0[256], s1[256];
    double a = 0, b = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        a += u[i] * v[i];
        b += v[i] * v[i];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s0[0];
        partial[2 * blockIdx.x + 1] = s1[0];
    }
}
// sum_i (a_i - b_i)^2 (b may be NULL: sum_i a_i^2) in FP64, per block, then
// summed in block order by sumsq_final_kernel (deterministic).
__global__ void sumsq_kernel(const float *a, const float *b, size_t count, double *partial) {
    __shared__ double s0[256];
    double acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (b ? (double)b[i] : 0.0);
        acc += d * d;
    }
    s0[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s0[threadIdx.x] += s0[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s0[0];
}
__global__ void __launch_bounds__(256) sumsq_final_kernel(const double *partial, int nblk, double *out) {
    __shared__ double s0[256];
    double a = 0;
    for (int i = threadIdx.x; i < nblk; i += 256) a += partial[i];
    s0[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s0[threadIdx.x] += s0[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s0[0];
}
// Final sums of the per-block partials: 256 threads, each adding its strided
// share in order, then a shared-memory tree (a fixed order: deterministic).
__global__ void __launch_bounds__(256) dots_final_kernel(const double *partial, int nblk, double *dot) {
    __shared__ double s0[256], s1[256];
    double a = 0, b = 0;
    for (int i = threadIdx.x; i < nblk; i += 256) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dot[0] = s0[0];
        dot[1] = s1[0];
    }
}
// v *= 1 / sqrt(dot[1])
__global__ void scale_kernel(double *v, size_t count, const double *dot) {
    double s = 1.0 / sqrt(dot[1]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        v[i] *= s;
}
__device__ __forceinline__ int ext_index_dev(int t, int len, int bc) {
    if (t >= 0 && t < len) return t;
    if (bc == 0) return -1;
    t = (t < 0) ? -1 - t : 2 * len - 1 - t;
    return (t >= 0 && t < len) ? t : -1;
}
// Exact blur of Eq. (1.1), one output pixel per thread, FP64 accumulation.
__global__ void blur_exact_kernel(const float *X, int m, int n, const float *P, int p, int q,
                                  int cr, int cc, int bc, float *Y) {
    int b = blockIdx.x * blockDim.x + threadIdx.x, a = blockIdx.y;
    if (b >= n || a >= m) return;
    double s = 0.0;
    for (int i = 0; i < p; ++i) {
        int ra = ext_index_dev(a - i + cr, m, bc);
        if (ra < 0) continue;
        const float *xr = X + (size_t)ra * n;
        for (int j = 0; j < q; ++j) {
            int cb = ext_index_dev(b - j + cc, n, bc);
            if (cb >= 0) s += (double)P[i * q + j] * (double)xr[cb];
        }
    }
    Y[(size_t)a * n + b] = (float)s;
}
// Dense factor panel F[i][row][col] (row < len, col < cols, leading dim ld)
// from band storage, in the operand format `kind`.
__global__ void densify_kernel(const double *band, int r, int len, int lo, int w, int cols, int kind,
                               void *hi, void *lo_out, size_t ld) {
    size_t total = (size_t)r * len * ld;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        size_t col = t % ld, rest = t / ld;
        int row = (int)(rest % len), i = (int)(rest / len);
        long k = (long)col - row - lo;
        double v = 0.0;
        if ((int)col < cols && k >= 0 && k < w) v = band[((size_t)i * w + k) * len + row];
        if (kind == 0) {
            reinterpret_cast<float *>(hi)[t] = (float)v;
        } else if (kind == 1) {
            __nv_bfloat16 h = __double2bfloat16(v);
            reinterpret_cast<__nv_bfloat16 *>(hi)[t] = h;
            if (lo_out) reinterpret_cast<__nv_bfloat16 *>(lo_out)[t] = __double2bfloat16(v - (double)__bfloat162float(h));
        } else if (kind == 2) {
            float h = tf32_round((float)v);
            reinterpret_cast<float *>(hi)[t] = h;
            if (lo_out) reinterpret_cast<float *>(lo_out)[t] = tf32_round((float)(v - (double)h));
        } else {
            reinterpret_cast<double *>(hi)[t] = v;
        }
    }
}
__global__ void split_kernel(const float *in, void *hi, void *lo, size_t count, int kind) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        float v = in[i];
        if (kind == 1) {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16 *>(hi)[i] = h;
            if (lo) reinterpret_cast<__nv_bfloat16 *>(lo)[i] = __float2bfloat16_rn(v - __bfloat162float(h));
        } else {
            float h = tf32_round(v);
            reinterpret_cast<float *>(hi)[i] = h;
            if (lo) reinterpret_cast<float *>(lo)[i] = tf32_round(v - h);
        }
    }
}

int grid_for(size_t count) {
    size_t g = (count + 255) / 256;
    return (int)(g < 4096 ? (g ? g : 1) : 4096);
}

}  // namespace

void launch_fill_f64(double *p, size_t count, double v, cudaStream_t s) {
    fill_f64_kernel<<<grid_for(count), 256, 0, s>>>(p, count, v);
}
void launch_f64_to_f32(const double *in, float *out, size_t count, cudaStream_t s) {
    f64_to_f32_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
}
void launch_df_to_f32(const float2 *in, float *out, size_t count, cudaStream_t s) {
    df_to_f32_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
}
void launch_f32_to_df(const float *in, float2 *out, size_t count, cudaStream_t s) {
    f32_to_df_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
}
void launch_df_to_f64(const float2 *in, double *out, size_t count, cudaStream_t s) {
    df_to_f64_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
}
void launch_f64_to_df(const double *in, float2 *out, size_t count, cudaStream_t s) {
    f64_to_df_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
}
void launch_f32_to_f64(const float *in, double *out, size_t count, cudaStream_t s) {
    f32_to_f64_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count);
}
void launch_check_finite(const float *in, size_t count, unsigned *status, cudaStream_t s) {
    check_finite_kernel<<<grid_for(count), 256, 0, s>>>(in, count, status);
}
void launch_seed_image(double *v, size_t count, cudaStream_t s) {
    seed_image_kernel<<<grid_for(count), 256, 0, s>>>(v, count);
}
void launch_dots(const double *u, const double *v, size_t count, double *partial, int nblk, double *dot,
                 cudaStream_t s) {
    dots_kernel<<<nblk, 256, 0, s>>>(u, v, count, partial);
    dots_final_kernel<<<1, 256, 0, s>>>(partial, nblk, dot);
}
void launch_sumsq(const float *a, const float *b, size_t count, double *partial, int nblk, double *out,
                  cudaStream_t s) {
    sumsq_kernel<<<nblk, 256, 0, s>>>(a, b, count, partial);
    sumsq_final_kernel<<<1, 256, 0, s>>>(partial, nblk, out);
}
void launch_scale(double *v, size_t count, const double *dot, cudaStream_t s) {
    scale_kernel<<<grid_for(count), 256, 0, s>>>(v, count, dot);
}
void launch_blur_exact(const float *X, int m, int n, const float *P, int p, int q, int cr, int cc, int bc,
                       float *Y, cudaStream_t s) {
    dim3 grid((n + 127) / 128, m);
    blur_exact_kernel<<<grid, 128, 0, s>>>(X, m, n, P, p, q, cr, cc, bc, Y);
}
void launch_densify(const double *band, int r, int len, int lo, int w, int cols, int kind, void *hi,
                    void *lo_out, size_t ld, cudaStream_t s) {
    densify_kernel<<<grid_for((size_t)r * len * ld), 256, 0, s>>>(band, r, len, lo, w, cols, kind, hi, lo_out, ld);
}
void launch_split(const float *in, void *hi, void *lo, size_t count, int kind, cudaStream_t s) {
    split_kernel<<<grid_for(count), 256, 0, s>>>(in, hi, lo, count, kind);
}

}  // namespace sfista
