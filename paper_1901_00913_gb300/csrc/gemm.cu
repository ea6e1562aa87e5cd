#include "gemm.h"

namespace sfista {
struct GemmPath {};
sfista_status gemm_create(GemmPath **out, const HostSetup &, int, bool, float *, float *, cudaStream_t) {
    *out = nullptr;
    return fail(SFISTA_ENOTSUP, "tensor-core operator not built yet");
}
void gemm_destroy(GemmPath *g) { delete g; }
void gemm_state_operands(GemmPath *, void **a, void **b, int *k) { *a = *b = nullptr; *k = 0; }
void gemm_prepare_solve(GemmPath *, const float *, cudaStream_t) {}
void gemm_stage(GemmPath *, int, const ProxArgs &, cudaStream_t) {}
sfista_status gemm_apply(GemmPath *, const float *, float *, int, cudaStream_t) { return SFISTA_ENOTSUP; }
}  // namespace sfista
