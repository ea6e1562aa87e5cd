// Tensor-core (tcgen05 / TMEM / TMA) execution of the Kronecker operator as
// four GEMMs per iteration with fused epilogues.  Library-internal.
#pragma once

#include "internal.h"

namespace sfista {

struct GemmPath;

// Builds operand panels and intermediates for precision `prec` from the
// host setup.  dense = true uses the full K range, otherwise K tiles outside
// the factor band are skipped.  status is the context's device status word
// (timeouts of the bounded mbarrier waits are reported there).
sfista_status gemm_create(GemmPath **out, const HostSetup &h, int prec, bool dense, unsigned *status,
                          cudaStream_t s);
void gemm_destroy(GemmPath *g);
// Switches between band-limited and full K ranges (the panels are the same).
void gemm_set_dense(GemmPath *g, bool dense);
// Tile shapes of stage st (0..3) that can be selected: the count returned,
// entries of (N tile width, resident P panel) written to bn / res (at most
// 4); the stacked stages 0 and 2 offer the widths 128 and 64, each also with
// the resident panel in BF16 band mode when the band fits it, the summed
// stages 1 and 3 the widths 64, 128, 256.
int gemm_tile_options(const GemmPath *g, int st, int *bn, int *res);
void gemm_set_tile(GemmPath *g, int st, int bn, int res);
// The default N tile of stage st: 64 when the stage has fewer tiles of 128
// columns than the GPU has SMs (most SMs would idle), else 128.
int gemm_default_bn(const GemmPath *g, int st);
// The shape stage st runs with (res as it applies in the current K mode).
void gemm_get_tile(const GemmPath *g, int st, int *bn, int *res);
// Split-operand copies of Y that the prox epilogue must write.
void gemm_state_operands(GemmPath *g, void **yhi, void **ylo, int *split_kind);
// Called once per solve after B has been copied in (binds its pointer).
void gemm_prepare_solve(GemmPath *g, const float *Bd, cudaStream_t s);
// Stage st (0..3) of one iteration of Alg. 2: the four GEMMs with the
// residual (stage 1) and prox / momentum (stage 3) epilogues.
void gemm_stage(GemmPath *g, int st, const ProxArgs &pa, cudaStream_t s);
// Converts an FP32 residual R (m x n) into the operand of stages 2 and 3
// (what stage 1 writes), for residuals computed outside the GEMMs.
void gemm_residual_operand(GemmPath *g, const float *R, cudaStream_t s);
// The operator alone (transpose = 0: A_s, 1: A_s^T) on FP32 device buffers.
sfista_status gemm_apply(GemmPath *g, const float *x, float *y, int transpose, cudaStream_t s);

// Launches a kernel whose bounded mbarrier wait expires (nothing arrives);
// it records DEV_TIMEOUT in *status and returns after about one second.
void launch_wait_timeout_selftest(unsigned *status, cudaStream_t s);

// Grouped execution of many problems (same precision, any sizes, ranks and
// bands): one launch per stage covers every problem's tiles.
struct GemmBatch;
sfista_status gemm_batch_create(GemmBatch **out, GemmPath *const *paths, int nprob, cudaStream_t s);
// Per solve: B pointers and prox arguments (pa.Xin / pa.Xout = state buffers 0 / 1).
sfista_status gemm_batch_bind(GemmBatch *b, const float *const *Bds, const ProxArgs *pas, cudaStream_t s);
void gemm_batch_stage(GemmBatch *b, int st, int k, cudaStream_t s);
// Resident P panels in the grouped stages 0 and 2 (allowed when every
// problem allows them; on by default then).
bool gemm_batch_res_ok(const GemmBatch *b);
void gemm_batch_set_res(GemmBatch *b, bool res);
void gemm_batch_destroy(GemmBatch *b);

}  // namespace sfista
