/*
 * sfista.h -- C ABI of the GB300 structured-FISTA library (libsfista.so).
 *
 * Structured FISTA (sFISTA) for Tikhonov-regularised image deblurring,
 * Chen, Nagy, Xi, Yu, "Structured FISTA for Image Restoration",
 * arXiv 1901.00913.  The blur matrix A of b = A x + e (Eq. 1.1) is replaced
 * by the Kronecker sum A_s = sum_{i=1..r} A_i kron B_i (Eq. Kronecker
 * structure, Theorem 1), and Alg. 2 minimises
 *     0.5 || sum_i B_i X A_i^T - B ||_F^2 + 0.5 lambda^2 ||X||_F^2
 * (Eq. matrix minimization model) with the fixed-step FISTA iteration.
 *
 * Paper notation: the paper's left factor H_i is B_i here (m x m, acts on
 * the row index of the image) and its right factor K_i is A_i (n x n, acts on
 * the column index); the paper's number of terms s is r here.
 *
 * Conventions for every call
 *   - Images are row-major, img_rows x img_cols (m x n): X[a][b] at
 *     X[a * n + b], a the row (vertical) index.  The paper's vec() stacks
 *     columns; the library never relies on that order in memory.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the context's device.  The caller owns every buffer
 *     it passes; the library copies what it keeps.  A context owns its own
 *     device memory until sfista_destroy().
 *   - Every call returns an sfista_status; nothing throws across the ABI.
 *     A failed call writes no output and leaves *out NULL where it has one.
 *     sfista_last_error() gives a one-line description of the most recent
 *     failure on the calling thread.
 *   - A context is used by one host thread at a time; calls on one context
 *     are ordered on the stream they are given (device calls) or on the
 *     context's own stream (host calls).
 */
#ifndef SFISTA_H
#define SFISTA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfista_ctx sfista_ctx;

typedef enum {
    SFISTA_OK = 0,
    SFISTA_EINVAL = 1,    /* bad argument (size, centre, rank, NaN/Inf input, tied singular values) */
    SFISTA_ENOMEM = 2,    /* host or device allocation failed */
    SFISTA_ECUDA = 3,     /* a CUDA runtime/driver call failed */
    SFISTA_ENOTSUP = 4,   /* valid request this library does not implement (e.g. periodic boundary) */
    SFISTA_ENUMERIC = 5,  /* the iteration produced a non-finite value */
    SFISTA_ETIMEOUT = 6   /* a device-side wait exceeded its bound; the kernel returned early */
} sfista_status;

/* Boundary condition (Sec. 2).  Periodic is recognised but not supported:
 * the paper leaves it out because it rings at the image border. */
typedef enum {
    SFISTA_BC_ZERO = 0,       /* A is BTTB; factors are banded Toeplitz             */
    SFISTA_BC_REFLEXIVE = 1,  /* A is BTHTHB; factors are Toeplitz + Hankel          */
    SFISTA_BC_PERIODIC = 2    /* -> SFISTA_ENOTSUP                                   */
} sfista_bc;

/* Arithmetic of the Kronecker operator (the four products of Step 1).
 * The FISTA state (X_k, X_{k-1}, Y_k) is always carried as double-float pairs
 * (hi + lo, two FP32 words, about 48 significant bits). */
typedef enum {
    SFISTA_FP32 = 0,     /* FP32 FMA on the CUDA cores                                  */
    SFISTA_TF32 = 1,     /* one TF32 tensor-core product, FP32 accumulate                */
    SFISTA_TF32X3 = 2,   /* split TF32: hi*hi + lo*hi + hi*lo, FP32 accumulate           */
    SFISTA_BF16 = 3,     /* one BF16 tensor-core product, FP32 accumulate                */
    SFISTA_BF16X3 = 4    /* split BF16: hi*hi + lo*hi + hi*lo, FP32 accumulate           */
} sfista_prec;

/* How the operator is executed. */
typedef enum {
    SFISTA_OP_AUTO = 0,        /* library's choice for (size, r, band, precision)           */
    SFISTA_OP_BANDED = 1,      /* factors applied from compact band storage (FP32/FP64 FMA)  */
    SFISTA_OP_GEMM_BAND = 2,   /* dense-factor GEMMs that skip K tiles outside the band       */
    SFISTA_OP_GEMM_DENSE = 3,  /* dense-factor GEMMs over the full K range (Sec. 3.3 O(s(nm^2+mn^2))) */
    SFISTA_OP_BANDED_PERSISTENT = 4, /* banded FP32 operator, the whole iteration loop in one
                                        persistent cooperative launch (grid barrier between phases):
                                        the fused operator form with band tiles and state resident
                                        when every th x 32 output tile has its own resident block
                                        (th, a multiple of 4 from 16 to 64, picked per problem; m, n
                                        multiples of 4), else the two-pass form */
    SFISTA_OP_BANDED_FUSED = 5, /* banded FP32 operator, one kernel per operator application: the
                                  row pass is kept in shared memory for the column pass (the
                                  automatic FP32 choice up to 1024^2 pixels and band width 48;
                                  SFISTA_OP_BANDED_PERSISTENT with the fused form when every
                                  tile also has its own resident block) */
    SFISTA_OP_FFT = 6,         /* FP32 FFT form of the structured product (Sec. 2, fast
                                  Toeplitz-plus-Hankel products by FFT): the extension of the
                                  image that toep + hank encode is separable, so
                                  sum_i B_i X A_i^T is one 2-D convolution of the extended
                                  image with the rank-r kernel sum_i c_i d_i^T, done by
                                  mixed-radix (2 - 16, 3, 9, 5) FFTs in shared memory; cost
                                  O(mn log mn) per application, independent of r and of the
                                  PSF width.  Requires m + psf_rows - 1 and
                                  n + psf_cols - 1 <= 8192. */
    SFISTA_OP_EXACT_FFT = 7    /* reported by sfista_info for contexts made by
                                  sfista_setup_exact (the exact blur A by the same FFT
                                  engine); not accepted by sfista_setup */
} sfista_operator;

typedef struct {
    int prec;               /* sfista_prec, default SFISTA_FP32                          */
    int op;                 /* sfista_operator, default SFISTA_OP_AUTO                   */
    int project_nonneg;     /* 1: X_k <- max(X_k, 0) after the shrink (x >= 0 constraint) */
    int use_graph;          /* 1 (default): replay the iteration loop as a CUDA graph     */
    double lipschitz;       /* > 0: use this L; <= 0: estimate lambda_max(A_s^T A_s)      */
    double lipschitz_tol;   /* relative change that stops the power iteration (1e-10)     */
    int lipschitz_maxit;    /* power-iteration cap (1000)                                 */
    int device;             /* CUDA device ordinal (default: current device)              */
    double l1;              /* mu >= 0 (default 0): adds mu ||X||_1 to the regulariser, so
                               Step 1 becomes S_mu(L Y_k - grad f(Y_k)) / (L + lambda^2)
                               with S_mu the soft threshold (the minimiser of Q_L of
                               Sec. 3.1 for that g; Sec. 1 and Sec. 5 name the l1 term
                               as future work).  Applied before the projection.         */
    int refine_every;       /* k_ref >= 0 (default 0: off).  Tensor-core forms: in every
                               iteration k that is a multiple of k_ref, all of Step 1 of
                               Alg. 2 -- the residual R_k = sum_i B_i Y_k A_i^T - B and
                               the adjoint product sum_j B_j^T R_k A_j -- is computed by
                               the FP32 band kernels from the FP32 factors instead of by
                               the low-precision GEMMs, with the shrink and momentum on
                               the form's own state; Y_{k+1} is written in the GEMMs'
                               operand format.  Such iterations add no product error, so
                               the error against exact arithmetic falls with k_ref (1:
                               the FP32 operator's).  The FP32 band forms compute every
                               iteration this way already, so it has no effect there.
                               Batches reject contexts that set it on a tensor-core form
                               (SFISTA_ENOTSUP).                                         */
    int tile_override;      /* 0 (default): the one-launch solver
                               (SFISTA_OP_BANDED_PERSISTENT, fused form) picks its tile
                               height th by a work model at setup, and sfista_tune by
                               measurement; 16..64 (a multiple of 4): use th x 32 tiles
                               (blocks of 256 threads up to 32 rows, 512 above;
                               SFISTA_EINVAL otherwise; ignored where the one-launch fused
                               solver is not used, and the two-pass persistent form is
                               used instead if those tiles do not all fit).             */
    int gemm_bn;            /* tensor-core forms: N tile width of the GEMM stages: 0
                               (default): per stage, 64 where the stage has fewer tiles
                               of 128 columns than the GPU has SMs, else 128; 64 or 128
                               for all four stages; 256 for the summed stages 1 and 3
                               (the left-factor products; stages 0 and 2 keep 128);
                               SFISTA_EINVAL otherwise.  Wider tiles read each factor
                               block once for more columns, narrower ones spread the
                               tiles more evenly over the SMs; sfista_tune measures
                               every width per stage.                                   */
    int gemm_resident_panels; /* tensor-core forms, stacked stages 0 and 2 (the right-
                               factor products): 0 (default) streams each tile's factor
                               panel with the tile's other operand; 1 keeps the panel of
                               a row tile (all K blocks of its band, hi and lo) resident
                               in shared memory while the tiles that share it run, where
                               that is possible (BF16 and BF16x3 band mode, every band
                               within three K blocks of 64).  sfista_tune measures both. */
} sfista_opts;

/* Fill *opts with the defaults listed above. */
void sfista_default_opts(sfista_opts *opts);

/*
 * sfista_setup -- form the Kronecker approximation of the blur (Sec. 2).
 *
 * psf      host, row-major psf_rows x psf_cols PSF P (FP64, finite; used as
 *          given, not normalised).
 * center_row, center_col
 *          0-based pixel of P that images a point source (the paper's
 *          centre (l, q)); -1 selects the middle pixel.
 * img_rows, img_cols
 *          image size m x n; requires psf_rows <= m and psf_cols <= n.
 * bc       sfista_bc.
 * r        number of Kronecker terms, 1 <= r <= min(psf_rows, psf_cols).
 * opts     NULL for defaults.
 * out      receives the new context.
 *
 * In FP64 on the host: the Gram weights of Theorem 1, their Cholesky factors
 * R (R^T R = G), the SVD of the weighted PSF P_bar = R_r P R_c^T, and the
 * factor profiles c_k = sqrt(s_k) R_r^{-1} u_k (left) and
 * d_k = sqrt(s_k) R_c^{-1} v_k (right).  Then, on the device, the banded
 * factors B_k = toep(c_k) [+ hank(c_k)], A_k = toep(d_k) [+ hank(d_k)] in
 * the operand formats the precision needs, and (unless opts->lipschitz > 0)
 * L = lambda_max(A_s^T A_s) by FP64 power iteration.
 * Errors: EINVAL for bad sizes/centre/rank, non-finite PSF, or
 * s_r == s_{r+1} > 0 (the truncation is not unique); ENOTSUP for periodic
 * boundary or a precision/operator pair this library lacks; ENOMEM; ECUDA.
 */
sfista_status sfista_setup(const double *psf, int psf_rows, int psf_cols,
                           int center_row, int center_col,
                           int img_rows, int img_cols, sfista_bc bc, int r,
                           const sfista_opts *opts, sfista_ctx **out);

/*
 * sfista_setup_exact -- a context whose operator is the exact blur A of
 * Eq. (1.1) (no Kronecker approximation), for vector FISTA on the
 * unapproximated problem, Alg. 1: the comparison system of Sec. 4.  Every
 * solve call (sfista_solve, sfista_solve_device, sfista_solve_state),
 * sfista_apply (A x and A^T x) and sfista_objective then use A.  Alg. 1's
 * Step 1 on vec(X) is the same element-wise update as Alg. 2's (Theorem 3
 * with A in place of A_s), so the iteration, its double-float state and its
 * epilogue are shared.  A is applied as a 2-D convolution of the zero or
 * reflected extension of X with the PSF, by the FFT engine of SFISTA_OP_FFT,
 * in FP32.  L = lambda_max(A^T A) by power iteration with that operator
 * (FP64 sums) unless opts->lipschitz > 0; opts->prec must be SFISTA_FP32 and
 * opts->op SFISTA_OP_AUTO (or SFISTA_OP_EXACT_FFT).  Arguments as sfista_setup
 * without r.  sfista_info reports op = SFISTA_OP_EXACT_FFT, no singular
 * values (approx_err 0) and band widths 0; sfista_get_profiles,
 * sfista_get_factors, sfista_tune, the reverse-mode calls and batches return
 * SFISTA_ENOTSUP for such contexts.
 * Errors: as sfista_setup; ENOTSUP when m + psf_rows - 1 or n + psf_cols - 1
 * exceeds 8192.
 */
sfista_status sfista_setup_exact(const double *psf, int psf_rows, int psf_cols,
                                 int center_row, int center_col,
                                 int img_rows, int img_cols, sfista_bc bc,
                                 const sfista_opts *opts, sfista_ctx **out);

/*
 * sfista_factorize -- the host half of sfista_setup alone (no device work):
 * the FP64 Kronecker factorisation of Sec. 2 / Theorem 1 for an m x n image.
 * sigma      host, min(psf_rows, psf_cols) singular values of P_bar (may be NULL)
 * C          host, r x psf_rows column profiles c_k (left factors B_k)
 * D          host, r x psf_cols row profiles d_k (right factors A_k)
 * approx_err host, sqrt(sum_{k>r} s_k^2) = ||A - A_s||_F (may be NULL)
 * Same argument checks and errors as sfista_setup.
 */
sfista_status sfista_factorize(const double *psf, int psf_rows, int psf_cols,
                               int center_row, int center_col,
                               int img_rows, int img_cols, sfista_bc bc, int r,
                               double *sigma, double *C, double *D,
                               double *approx_err);

/*
 * sfista_factor_bands -- the band storage the banded kernels use for one
 * factor family (host only, no device work), from the same factorisation:
 *   which 0: A_k (right factors, img_cols x img_cols)   1: A_k^T
 *         2: B_k (left factors, img_rows x img_rows)    3: B_k^T
 *   F_k[c][c + lo + t] = band[(k * w + t) * len + c], t in [0, w),
 *   len = img_cols (which 0, 1) or img_rows (2, 3); entries whose column
 *   falls outside [0, len) are 0.  In the interior of the axis a factor
 *   T + H of Sec. 2 is Toeplitz: interior[0..1] = [i0, i1), the widest run
 *   of rows around len / 2 whose FP32 values equal row len / 2 bit for bit
 *   (the rows whose kernels take one shared coefficient row).
 * lo, w      out, the band's first offset and width.
 * band       host, r * w * len doubles, or NULL to query lo and w first.
 * interior   host, 2 ints (may be NULL).
 * Same argument checks and errors as sfista_setup; which outside 0..3 is
 * SFISTA_EINVAL.
 */
sfista_status sfista_factor_bands(const double *psf, int psf_rows, int psf_cols,
                                  int center_row, int center_col,
                                  int img_rows, int img_cols, sfista_bc bc, int r,
                                  int which, int *lo, int *w, double *band,
                                  int *interior);

/* Release every resource of ctx (NULL is ignored). */
void sfista_destroy(sfista_ctx *ctx);

/*
 * sfista_solve -- Alg. 2 from X_0 = 0 for `iters` iterations (host buffers).
 *
 * b      host, m x n observed image B (FP32).
 * lambda Tikhonov parameter (>= 0; the penalty is 0.5 lambda^2 ||X||^2).
 * iters  >= 0; 0 returns X_0 = 0.
 * x      host, m x n output X_iters (FP32).
 * Copies b in, runs the loop on the context's stream, copies x out and
 * synchronises.  ENUMERIC if a non-finite value appeared, ETIMEOUT if a
 * device wait gave up, EINVAL for non-finite b or bad arguments.
 */
sfista_status sfista_solve(sfista_ctx *ctx, const float *b, double lambda,
                           int iters, float *x);

/*
 * sfista_solve_device -- as sfista_solve with device buffers d_b, d_x (FP32,
 * m x n) on the CUDA stream `stream` (cudaStream_t, NULL = legacy default).
 * Asynchronous: returns after enqueueing; status words are checked on the
 * next call that synchronises (sfista_sync).
 */
sfista_status sfista_solve_device(sfista_ctx *ctx, const float *d_b,
                                  double lambda, int iters, float *d_x,
                                  void *stream);

/*
 * sfista_solve_state -- resumable form of Alg. 2 on FP64 device state
 * (converted to the internal double-float state on entry and back to FP64
 * on exit).
 *
 * d_X, d_Xprev  device, m x n FP64: on entry X_{k0} and X_{k0-1}; on exit
 *               X_{k0+iters} and X_{k0+iters-1}.  With k0 = 0, d_X is the
 *               starting point X_0 = Y_1 and d_Xprev is ignored on entry.
 * k0            number of iterations already done (t_k depends on k only,
 *               so (X_k, X_{k-1}, k) is the whole state of Alg. 2).
 */
sfista_status sfista_solve_state(sfista_ctx *ctx, const float *d_b,
                                 double lambda, int k0, int iters,
                                 double *d_X, double *d_Xprev, void *stream);

/*
 * Batched solves: many independent problems (any image sizes, PSFs, ranks,
 * one precision and operator family) advance together, one launch per stage
 * of Alg. 2 covering the tiles of every problem, the iteration loop replayed
 * as one CUDA graph.  A banded FP32 batch whose images all have m, n
 * multiples of 4 and whose 32 x 32 tiles all fit as co-resident blocks (one
 * block per tile of every problem) runs instead as one cooperative launch of
 * the fused solver for all iterations; sfista_batch_tune compares the two.
 *
 * sfista_batch_create -- group nprob contexts made by sfista_setup (same
 *   device, same precision; all tensor-core forms or all banded forms).  The
 *   batch uses each context's state buffers: do not solve with a grouped
 *   context on its own while a batch solve of it is in flight.
 * sfista_batch_solve -- Alg. 2 from X_0 = 0 for every problem.
 *   d_b, d_x  host arrays of nprob device pointers (FP32, problem p is
 *             m_p x n_p); lambdas host array of nprob values.
 *   Asynchronous on `stream`: each d_b[p] is read, and d_x[p] written, in
 *   stream order (an output may alias an input).  The one-launch form reads
 *   d_b[p] in place and writes X_iters straight into d_x[p].
 *   sfista_batch_sync reports device status of every problem (the first
 *   error found).
 * sfista_solve_batched -- create, solve, sync and destroy in one call.
 */
typedef struct sfista_batch sfista_batch;
sfista_status sfista_batch_create(sfista_ctx *const *ctxs, int nprob,
                                  sfista_batch **out);
sfista_status sfista_batch_solve(sfista_batch *batch, const float *const *d_b,
                                 const double *lambdas, int iters,
                                 float *const *d_x, void *stream);
sfista_status sfista_batch_sync(sfista_batch *batch, void *stream);
void sfista_batch_destroy(sfista_batch *batch);
sfista_status sfista_solve_batched(sfista_ctx *const *ctxs,
                                   const float *const *d_b,
                                   const double *lambdas, int nprob, int iters,
                                   float *const *d_x, void *stream);

/*
 * Differentiating the unrolled solve (Alg. 2 for a fixed number of
 * iterations, no projection, L held fixed).  Both calls need a context with
 * a banded operator form (SFISTA_FP32 with SFISTA_OP_BANDED,
 * SFISTA_OP_BANDED_PERSISTENT or SFISTA_OP_BANDED_FUSED); otherwise ENOTSUP.
 *
 * sfista_unrolled_fwd -- X_iters from X_0 = 0 into d_x (device FP32, m x n),
 *   saving (X_k, X_{k-1}) at k = 0, ckpt_every, 2 ckpt_every, ... into d_ckpt
 *   (device FP64, caller-owned, 2 * ceil(iters / ckpt_every) * m * n values).
 *
 * sfista_unrolled_bwd -- given d_gX = dl/dX_iters (device FP32, m x n) and the
 *   checkpoints of the forward with the same b, lambda, iters, ckpt_every:
 *     d_gb      device FP32 m x n: dl/db
 *     g_lambda  host FP64 scalar:  dl/dlambda
 *     d_gA      device FP32 r x n x n (or NULL): dl/dA_i, the dense right factors
 *     d_gB      device FP32 r x m x m (or NULL): dl/dB_i, the dense left factors
 *   The adjoint of each step is the step's own symmetric operator
 *   M = (L I - A_s^T A_s) / (L + lambda^2); segments between checkpoints are
 *   recomputed from their checkpoint.  Synchronous.
 */
sfista_status sfista_unrolled_fwd(sfista_ctx *ctx, const float *d_b, double lambda,
                                  int iters, int ckpt_every, double *d_ckpt,
                                  float *d_x, void *stream);
sfista_status sfista_unrolled_bwd(sfista_ctx *ctx, const float *d_b, double lambda,
                                  int iters, int ckpt_every, const double *d_ckpt,
                                  const float *d_gX, float *d_gb, double *g_lambda,
                                  float *d_gA, float *d_gB, void *stream);

/* Wait for the context's work on `stream`, then report device-side status
 * (ENUMERIC / ETIMEOUT) raised since the last sync. */
sfista_status sfista_sync(sfista_ctx *ctx, void *stream);

/*
 * sfista_apply -- the Kronecker operator alone, on device FP32 buffers:
 *   transpose = 0:  d_y = sum_i B_i d_x A_i^T     (A_s, Eq. matrix equation)
 *   transpose = 1:  d_y = sum_i B_i^T d_x A_i     (A_s^T, Alg. 2 Step 1)
 * in the context's precision and operator form.  Asynchronous on `stream`.
 */
sfista_status sfista_apply(sfista_ctx *ctx, const float *d_x, float *d_y,
                           int transpose, void *stream);

/*
 * sfista_info -- scalars of the setup.
 * lipschitz   L used by Step 1 (estimated or given).
 * sigma       if non-NULL, min(psf_rows, psf_cols) singular values of P_bar.
 * approx_err  if non-NULL, sqrt(sum_{k>r} s_k^2) = ||A - A_s||_F (Theorem 1).
 * config      if non-NULL, int[8]: effective precision, operator form, band
 *             widths w of A_i and B_i, then the band offsets lo of A_i, B_i,
 *             A_i^T, B_i^T (row `row` of a factor holds its nonzeros in
 *             columns row + lo .. row + lo + w - 1).
 */
sfista_status sfista_info(const sfista_ctx *ctx, double *lipschitz,
                          double *sigma, double *approx_err, int *config);

/*
 * sfista_set_factors -- replace the context's Kronecker factors with given
 * dense ones (the matrix model of Sec. 1 with any banded A_i, B_i in place of
 * the factorisation's), e.g. so that the unrolled solve and its gradients
 * follow factors that an optimiser has changed.
 * A  host, r x n x n FP64 right factors A_i, or NULL to keep the current ones.
 * B  host, r x m x m FP64 left factors B_i, or NULL to keep the current ones.
 * Every entry outside the band of the context's factors (rows a: columns
 * a + lo .. a + lo + w - 1, as sfista_info reports) must be zero.  L is kept
 * (held fixed, as in the reverse mode).  Later solves, sfista_apply,
 * sfista_objective and the reverse-mode calls use the new factors;
 * sfista_get_factors returns them; sfista_get_profiles then returns ENOTSUP.
 * Errors: ENOTSUP unless the context has a banded FP32 operator form;
 * EINVAL for a nonzero entry outside the band.  Synchronous.
 */
sfista_status sfista_set_factors(sfista_ctx *ctx, const double *A, const double *B);

/* Factor profiles: C (r x psf_rows) column profiles c_k of the left factors,
 * D (r x psf_cols) row profiles d_k of the right factors (host, FP64). *
sfista_status sfista_get_profiles(const sfista_ctx *ctx, double *C, double *D);

/* Dense factors on the host, FP64: B (r x m x m), A (r x n x n). */
sfista_status sfista_get_factors(const sfista_ctx *ctx, double *A, double *B);

/*
 * sfista_blur -- the exact blur of Eq. (1.1) (not the approximation):
 *   d_y[a][b] = sum_{i,j} P[i][j] * Xext[a - i + cr][b - j + cc]
 * with Xext the zero or half-sample-reflected extension of d_x.  Used to
 * synthesise observations.  psf is host FP64; d_x, d_y device FP32 (m x n,
 * distinct buffers).  Synchronous.
 */
sfista_status sfista_blur(const double *psf, int psf_rows, int psf_cols,
                          int center_row, int center_col, sfista_bc bc,
                          const float *d_x, int img_rows, int img_cols,
                          float *d_y, void *stream);

/*
 * sfista_objective -- Phi_s(X) = 1/2 ||A_s X - B||_F^2 + 1/2 lambda^2 ||X||_F^2,
 * the function Alg. 2 minimises (the matrix model with the Kronecker
 * approximation A_s of Sec. 2), for monitoring convergence or divergence.
 * d_b, d_x  device, m x n FP32 (B and X).  phi: host out (FP64 sums of the
 * FP32 operator result).  Synchronous.  Errors: SFISTA_EINVAL for NULL
 * pointers or lambda < 0.
 */
sfista_status sfista_objective(sfista_ctx *ctx, const float *d_b, const float *d_x, double lambda,
                               double *phi, void *stream);

/*
 * sfista_time_stages -- per-kernel timing of one iteration of Alg. 2 on the
 * context's own stream, for roofline reporting.  Runs `reps` iterations
 * (k = 1..reps, launched one by one, no graph) on the device observation
 * d_b, with CUDA events recorded between the four stages of each iteration:
 *   0: forward right-factor product   (Y A_i^T)
 *   1: forward left-factor product + residual epilogue
 *   2: adjoint right-factor product   (R A_i)
 *   3: adjoint left-factor product + shrink / momentum epilogue
 * ms (host, float[4]) receives the mean duration of each stage in ms.
 * Synchronous.  Leaves the solver state undefined (the next solve resets it).
 */
sfista_status sfista_time_stages(sfista_ctx *ctx, const float *d_b, double lambda,
                                 int reps, float *ms);

/* One configuration measured by sfista_tune. */
typedef struct {
    int op;            /* sfista_operator of the configuration                        */
    int stage;         /* 0..3: one stage timed alone (see sfista_time_stages);
                          -1: whole iterations                                         */
    int chunk;         /* terms staged per block in that stage (two-pass banded form);
                          for SFISTA_OP_BANDED_PERSISTENT entries the one-launch
                          solver's tile height th; for tensor-core stage entries the
                          N tile width (64, 128 or 256), plus 1 for a resident factor
                          panel (stages 0 and 2: 65 / 129); batch entries (stage -1):
                          1 / 0 for resident / streamed panels; 0 where none applies */
    float ms;          /* mean time per stage (or per iteration), ms                  */
} sfista_tune_entry;

/*
 * sfista_tune -- autotuner for this context's problem shape.  The paper has no
 * counterpart (its operator runs in serial MATLAB).  Times `iters` repetitions
 * of each candidate on the context's own stream, on an all-zero observation
 * (timing does not depend on the data), and keeps the fastest.  Candidates for
 * a single stage are launched directly; whole-iteration candidates run the
 * iteration loop exactly as a solve does (a CUDA graph of the iterations when
 * use_graph is set, or the one-launch solver), so forms with several launches
 * per iteration carry the launch cost a solve has:
 *   - two-pass banded FP32 form: for each of the four stages, the number of
 *     terms staged per block (1 .. r, those that fit in shared memory); this
 *     sets shared memory per block and so the blocks resident per SM;
 *   - if the operator form was left to SFISTA_OP_AUTO: FP32 contexts also
 *     compare the tuned two-pass form with the fused form, the FFT form
 *     (SFISTA_OP_FFT, when its transforms fit) and, when every th x 32 tile
 *     (th from 64 down to 16) can have its own resident block, the one-launch
 *     solver (SFISTA_OP_BANDED_PERSISTENT, timed per iteration over
 *     max(iters, 40) iterations of one launch, for every tile height th);
 *     tensor-core contexts compare the band-limited and full (dense) K
 *     ranges;
 *   - tensor-core forms: for each stage, timed alone in the chosen K range,
 *     its tile shapes: N tile 64, 128 or 256 for stages 1 and 3 (the choice
 *     gemm_bn fixes); N tile 64 or 128 for stages 0 and 2, each with a
 *     streamed or (where the panel fits) resident factor panel.
 * An explicitly chosen form is kept (only its stages are tuned).  The chosen
 * configuration applies to later solves, sfista_apply and batches created
 * afterwards (sfista_info reports the form).
 * entries      host, caller-owned array of max_entries (may be NULL): every
 *              measurement, in order.
 * n_entries    host out (may be NULL): number of measurements made.
 * Synchronous.  Leaves the solver state undefined (the next solve resets it).
 * Errors: SFISTA_EINVAL for iters < 1 or max_entries < 0.
 */
sfista_status sfista_tune(sfista_ctx *ctx, int iters, sfista_tune_entry *entries, int max_entries,
                          int *n_entries);

/*
 * sfista_batch_tune -- autotuner of a banded batch.  The grouped launches of a
 * batch share one shared-memory size (that of the largest tile of any
 * problem), which sets the blocks resident per SM for every problem, so the
 * batch is tuned as a whole: for each shared-memory budget in a fixed list
 * (and for the problems' own chunks, budget 0) every problem takes the largest
 * term chunks that fit, the batch solves `iters` iterations of an all-zero
 * observation twice (the second timed), and the fastest plan is kept.  When
 * every 32 x 32 tile of every problem can have its own resident block (and
 * m, n are multiples of 4), the whole batch solve as one cooperative launch
 * of the fused solver is a further plan (the default for such batches).
 * entries: one per distinct plan, stage = -1, ms = time per iteration;
 * op = SFISTA_OP_BANDED with chunk = the budget in KB (0: each problem's own
 * chunks), or op = SFISTA_OP_BANDED_PERSISTENT (chunk 0) for the one-launch
 * plan.
 * Tensor-core batches: when every problem allows resident factor panels in
 * the grouped stages 0 and 2 (BF16 band mode, bands within three K blocks),
 * the batch solve is timed with resident and with streamed panels (entries:
 * op = the problems' form, stage -1, chunk 1 / 0) and the faster is kept;
 * otherwise there is nothing to choose (no entries, SFISTA_OK).
 * Synchronous.  Leaves every grouped context's state undefined.
 */
sfista_status sfista_batch_tune(sfista_batch *batch, int iters, sfista_tune_entry *entries, int max_entries,
                                int *n_entries);

/*
 * sfista_apply_static -- the banded operator of sfista_apply without any
 * device allocation.  The paper has no counterpart: this call exists for
 * callers that cannot allocate device memory themselves, such as a plugin
 * inside a host framework that owns all GPU memory through its own arena and
 * forbids direct cudaMalloc, or a latency-critical loop that cannot take the
 * implicit synchronisation and possible failure of an allocation.  It needs
 * no context, so the caller supplies the factors in band storage.
 *
 *   d_y = sum_i B_i d_x A_i^T,  with
 *   A_i[c][c + lo_right + k] = d_band_right[(i * w_right + k) * img_cols + c]
 *   B_i[a][a + lo_left + k]  = d_band_left[(i * w_left + k) * img_rows + a]
 * for k in [0, w); entries whose column falls outside the image must be 0.
 * Pass the bands of A_i^T and B_i^T instead to apply A_s^T.
 *
 * d_x, d_y            device, img_rows x img_cols FP32, distinct buffers.
 * d_band_right/left   device FP32 band tables as above (caller-owned).
 * stream              cudaStream_t (NULL = legacy default); asynchronous.
 *
 * Scratch: the r intermediate images live in one file-scope device array of
 * 8 Mi floats (32 MiB) that every GPU loading this library keeps until the
 * process exits; r * img_rows * img_cols above 8,388,608 returns EINVAL.
 * All calls share the array and each call overwrites what it reads, so no
 * state carries over, but calls whose work overlaps on the GPU (different
 * streams, or unordered host threads) race on it.  The first call on each
 * device looks up the array's device address with cudaGetSymbolAddress;
 * make that first call before any stream capture on that device.  The
 * address is kept for the life of the process, so do not use this call on a
 * device after cudaDeviceReset.
 * Calls no cudaMalloc or cudaFree.
 * Errors: EINVAL for NULL or aliased buffers, sizes or r below 1, band widths
 * outside [1, 2 * image size], band offsets lo outside
 * [-2 * image size, image size], or the scratch limit above.
 */
sfista_status sfista_apply_static(const float *d_x, float *d_y, int img_rows,
                                  int img_cols, int r,
                                  const float *d_band_right, int lo_right,
                                  int w_right, const float *d_band_left,
                                  int lo_left, int w_left, void *stream);

/*
 * sfista_selftest_wait_timeout -- exercises the failure path of the bounded
 * device-side waits: launches a kernel that waits on an mbarrier nothing
 * arrives at.  The wait gives up after about one second, the kernel records
 * the timeout and returns, and this call reports SFISTA_ETIMEOUT (any other
 * status means the guard did not work).  The context stays usable.
 */
sfista_status sfista_selftest_wait_timeout(sfista_ctx *ctx);

const char *sfista_strerror(sfista_status s);
const char *sfista_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFISTA_H */
