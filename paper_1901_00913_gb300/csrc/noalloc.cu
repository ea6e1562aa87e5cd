// sfista_apply_static: the banded Kronecker operator without any device
// allocation.  The paper has no counterpart; this exists for callers that
// cannot allocate device memory themselves, e.g. a plugin running inside a
// host framework that owns every byte of GPU memory through its own arena and
// forbids direct cudaMalloc, or a latency-critical loop that cannot accept
// the implicit synchronisation and possible failure of an allocation.
//
// The intermediate products Z_i = X A_i^T (r images of m x n floats) live in
// one file-scope device array of fixed size instead of a context buffer.
// Every GPU that loads this library holds that array until the process
// exits.  All calls share it: two calls whose work overlaps on the GPU (on
// different streams, or on different host threads without ordering) race on
// it.  Nothing in it needs to start at zero: the rows pass writes every
// element the cols pass reads, so a call never sees the previous call's data.
#include <mutex>

#include "internal.h"

namespace sfista {
namespace {

// 8 Mi floats = 32 MiB: r * m * n <= 8,388,608 (e.g. 1024^2 with r <= 8,
// 2048^2 with r <= 2).
constexpr size_t kStaticScratchFloats = size_t(8) << 20;

static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (in host code the array's name is only a host-side stand-in).  The
// address is kept for the life of the process: after a cudaDeviceReset the
// module is loaded again and the kept address is stale, so the entry point
// must not be used across a device reset.
sfista_status scratch_for_current_device(float **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SFISTA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(SFISTA_ENOTSUP, "device ordinal beyond the static table");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(SFISTA_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SFISTA_OK;
}

}  // namespace
}  // namespace sfista

using namespace sfista;

extern "C" sfista_status sfista_apply_static(const float *d_x, float *d_y, int img_rows, int img_cols, int r,
                                             const float *d_band_right, int lo_right, int w_right,
                                             const float *d_band_left, int lo_left, int w_left, void *stream) {
    if (!d_x || !d_y || !d_band_right || !d_band_left) return fail(SFISTA_EINVAL, "NULL pointer");
    if (d_x == d_y) return fail(SFISTA_EINVAL, "x and y must be distinct buffers");
    if (img_rows < 1 || img_cols < 1 || r < 1) return fail(SFISTA_EINVAL, "sizes and r must be positive");
    if (w_right < 1 || w_left < 1 || w_right > 2 * img_cols || w_left > 2 * img_rows)
        return fail(SFISTA_EINVAL, "band widths must be in [1, 2 * image size]");
    // A band whose offset lies further out than this touches no column of
    // the image, and the kernels form row + lo (+ tap) in int: bounding lo
    // keeps that arithmetic far from overflow.
    if (lo_right < -2 * img_cols || lo_right > img_cols || lo_left < -2 * img_rows || lo_left > img_rows)
        return fail(SFISTA_EINVAL, "band offsets must be in [-2 * image size, image size]");
    if (img_rows > (1 << 28) || img_cols > (1 << 28))
        return fail(SFISTA_EINVAL, "image side above 2^28");
    size_t need = (size_t)r * img_rows * img_cols;
    if (need > kStaticScratchFloats)
        return fail(SFISTA_EINVAL, "r * img_rows * img_cols = " + std::to_string(need) +
                                       " exceeds the static scratch of " + std::to_string(kStaticScratchFloats) +
                                       " floats (32 MiB)");
    float *Z = nullptr;
    sfista_status st = scratch_for_current_device(&Z);
    if (st) return st;
    cudaError_t e = band_set_smem_limits(w_right > w_left ? w_right : w_left);
    if (e != cudaSuccess) return fail(SFISTA_ENOTSUP, std::string("band too wide: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    ProxArgs pa{};
    launch_band_rows<float>(d_x, img_rows, img_cols, d_band_right, lo_right, w_right, r, Z, s);
    launch_band_cols<float>(Z, img_rows, img_cols, d_band_left, lo_left, w_left, r, EPI_STORE, d_y, pa, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SFISTA_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SFISTA_OK;
}
