/*
 * FP64 CPU oracle for structured FISTA (sFISTA), Chen, Nagy, Xi, Yu,
 * "Structured FISTA for Image Restoration" (arXiv 1901.00913).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the
 * CUDA path is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it.  It
 * shares no code, header or table with the library under
 * paper_1901_00913_gb300/.
 *
 * Conventions (row-major, 0-based):
 *   image X[a][b], a = row (vertical) index in [0,m), b = column in [0,n).
 *   PSF P[i][j] is p x q with centre (cr, cc): the pixel that images a
 *   point source (Sec. 2, "the PSF ... stored as an array", centre p_lq).
 *   bc = 0: zero boundary (BTTB A); bc = 1: reflective boundary (BTHTHB A),
 *   half-sample reflection  -1 -> 0, -2 -> 1, m -> m-1  (the reflection that
 *   the banded Hankel matrix of Sec. 2 encodes).
 *
 * Kronecker factors (Sec. 2, Eqs. for toep/hank): term i has a column
 * profile c_i (length p, centre cr) giving the left factor B_i (m x m,
 * acts on the row index a) and a row profile d_i (length q, centre cc)
 * giving the right factor A_i (n x n).  The operator of Eq. (matrix
 * equation) is  A_s(X) = sum_i B_i X A_i^T.  The oracle never forms B_i or
 * A_i: it applies each as a 1-D convolution along one image axis, as a
 * gather (forward) or the matching scatter (transpose).
 *
 * Loops are deliberately plain; OpenMP only splits independent image
 * lines, so every output is summed in the same order at any thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Extended-image index map for one axis of length len.  Returns the source
 * index in [0,len) or -1 when the extended pixel is zero (zero boundary or
 * beyond one reflection). */
static int ext_index(int t, int len, int bc)
{
    if (t >= 0 && t < len) return t;
    if (bc == 0) return -1;
    if (t < 0) t = -1 - t;            /* -1 -> 0, -2 -> 1, ... */
    else t = 2 * len - 1 - t;         /* len -> len-1, ... */
    return (t >= 0 && t < len) ? t : -1;
}

/* Exact blur, Eq. (1.1) with A built from the PSF (Sec. 2):
 *   Y[a][b] = sum_{i,j} P[i][j] * Xext[a - i + cr][b - j + cc]
 * i.e. a 2-D convolution of the boundary-extended image with the PSF. */
void orc_blur(const double *X, int m, int n, const double *P, int p, int q,
              int cr, int cc, int bc, double *Y)
{
#pragma omp parallel for schedule(static)
    for (int a = 0; a < m; ++a) {
        for (int b = 0; b < n; ++b) {
            double s = 0.0;
            for (int i = 0; i < p; ++i) {
                int ra = ext_index(a - i + cr, m, bc);
                if (ra < 0) continue;
                for (int j = 0; j < q; ++j) {
                    int cb = ext_index(b - j + cc, n, bc);
                    if (cb < 0) continue;
                    s += P[i * q + j] * X[(size_t)ra * n + cb];
                }
            }
            Y[(size_t)a * n + b] = s;
        }
    }
}

/* Transpose of orc_blur: the scatter of each input pixel through the same
 * index map (column t of A^T's action).  Y = A^T X. */
void orc_blur_T(const double *X, int m, int n, const double *P, int p, int q,
                int cr, int cc, int bc, double *Y)
{
    memset(Y, 0, sizeof(double) * (size_t)m * n);
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < n; ++b) {
            double x = X[(size_t)a * n + b];
            for (int i = 0; i < p; ++i) {
                int ra = ext_index(a - i + cr, m, bc);
                if (ra < 0) continue;
                for (int j = 0; j < q; ++j) {
                    int cb = ext_index(b - j + cc, n, bc);
                    if (cb < 0) continue;
                    Y[(size_t)ra * n + cb] += P[i * q + j] * x;
                }
            }
        }
}

/* Right factor applied along rows, Z = X A^T with A = toep(d,cc) [+ hank]:
 *   Z[a][c] = sum_k d[k] * Xext[a][c - k + cc]                (gather)   */
static void rows_fwd(const double *X, int m, int n, const double *d, int q,
                     int cc, int bc, double *Z)
{
#pragma omp parallel for schedule(static)
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < n; ++c) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) {
                int b = ext_index(c - k + cc, n, bc);
                if (b >= 0) s += d[k] * X[(size_t)a * n + b];
            }
            Z[(size_t)a * n + c] = s;
        }
}

/* Z = X A (transpose of rows_fwd): scatter each X[a][c] to the pixels that
 * the gather above read it from. */
static void rows_adj(const double *X, int m, int n, const double *d, int q,
                     int cc, int bc, double *Z)
{
#pragma omp parallel for schedule(static)
    for (int a = 0; a < m; ++a) {
        double *z = Z + (size_t)a * n;
        for (int b = 0; b < n; ++b) z[b] = 0.0;
        for (int c = 0; c < n; ++c) {
            double x = X[(size_t)a * n + c];
            for (int k = 0; k < q; ++k) {
                int b = ext_index(c - k + cc, n, bc);
                if (b >= 0) z[b] += d[k] * x;
            }
        }
    }
}

/* Left factor applied along columns, W = B Z with B = toep(c,cr) [+ hank]:
 *   W[a][b] = sum_k c[k] * Zext[a - k + cr][b]                 (gather)   */
static void cols_fwd(const double *Z, int m, int n, const double *c, int p,
                     int cr, int bc, double *W)
{
#pragma omp parallel for schedule(static)
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < m; ++a) {
            double s = 0.0;
            for (int k = 0; k < p; ++k) {
                int e = ext_index(a - k + cr, m, bc);
                if (e >= 0) s += c[k] * Z[(size_t)e * n + b];
            }
            W[(size_t)a * n + b] = s;
        }
}

/* W = B^T Z: the scatter matching cols_fwd. */
static void cols_adj(const double *Z, int m, int n, const double *c, int p,
                     int cr, int bc, double *W)
{
#pragma omp parallel for schedule(static)
    for (int b = 0; b < n; ++b) {
        for (int a = 0; a < m; ++a) W[(size_t)a * n + b] = 0.0;
        for (int a = 0; a < m; ++a) {
            double z = Z[(size_t)a * n + b];
            for (int k = 0; k < p; ++k) {
                int e = ext_index(a - k + cr, m, bc);
                if (e >= 0) W[(size_t)e * n + b] += c[k] * z;
            }
        }
    }
}

/* Kronecker-sum operator, Eq. (matrix equation):  Out = sum_i B_i Y A_i^T.
 * C is r x p (column profiles c_i), D is r x q (row profiles d_i). */
void orc_kron_apply(const double *Y, int m, int n, int r, const double *C,
                    int p, int cr, const double *D, int q, int cc, int bc,
                    double *Out)
{
    size_t N = (size_t)m * n;
    double *Z = (double *)malloc(sizeof(double) * N);
    double *W = (double *)malloc(sizeof(double) * N);
    memset(Out, 0, sizeof(double) * N);
    for (int i = 0; i < r; ++i) {
        rows_fwd(Y, m, n, D + (size_t)i * q, q, cc, bc, Z);
        cols_fwd(Z, m, n, C + (size_t)i * p, p, cr, bc, W);
        for (size_t t = 0; t < N; ++t) Out[t] += W[t];
    }
    free(Z);
    free(W);
}

/* Its adjoint (Alg. 2, Step 1 outer sum):  Out = sum_j B_j^T R A_j. */
void orc_kron_apply_T(const double *R, int m, int n, int r, const double *C,
                      int p, int cr, const double *D, int q, int cc, int bc,
                      double *Out)
{
    size_t N = (size_t)m * n;
    double *Z = (double *)malloc(sizeof(double) * N);
    double *W = (double *)malloc(sizeof(double) * N);
    memset(Out, 0, sizeof(double) * N);
    for (int j = 0; j < r; ++j) {
        rows_adj(R, m, n, D + (size_t)j * q, q, cc, bc, Z);
        cols_adj(Z, m, n, C + (size_t)j * p, p, cr, bc, W);
        for (size_t t = 0; t < N; ++t) Out[t] += W[t];
    }
    free(Z);
    free(W);
}

/* Largest eigenvalue of A_s^T A_s by power iteration from the image X0
 * (overwritten with the final normalised iterate).  Stops when the
 * Rayleigh quotient changes by less than tol (relative) or after maxit
 * steps.  Returns the estimate; *iters_out receives the step count. */
double orc_power_lipschitz(double *X0, int m, int n, int r, const double *C,
                           int p, int cr, const double *D, int q, int cc,
                           int bc, double tol, int maxit, int *iters_out)
{
    size_t N = (size_t)m * n;
    double *T = (double *)malloc(sizeof(double) * N);
    double *U = (double *)malloc(sizeof(double) * N);
    double nrm = 0.0, mu = 0.0, prev = 0.0;
    int it = 0;
    for (size_t t = 0; t < N; ++t) nrm += X0[t] * X0[t];
    nrm = sqrt(nrm);
    for (size_t t = 0; t < N; ++t) X0[t] /= nrm;
    for (it = 1; it <= maxit; ++it) {
        orc_kron_apply(X0, m, n, r, C, p, cr, D, q, cc, bc, T);
        orc_kron_apply_T(T, m, n, r, C, p, cr, D, q, cc, bc, U);
        mu = 0.0;
        nrm = 0.0;
        for (size_t t = 0; t < N; ++t) {
            mu += X0[t] * U[t];      /* Rayleigh quotient, ||X0|| = 1 */
            nrm += U[t] * U[t];
        }
        nrm = sqrt(nrm);
        if (nrm == 0.0) break;
        for (size_t t = 0; t < N; ++t) X0[t] = U[t] / nrm;
        if (it > 1 && fabs(mu - prev) <= tol * fabs(mu)) break;
        prev = mu;
    }
    if (iters_out) *iters_out = it;
    free(T);
    free(U);
    return mu;
}

/* Objective of the matrix model (Eq. matrix minimization model):
 *   Phi_s(X) = 0.5 ||A_s(X) - B||_F^2 + 0.5 lambda^2 ||X||_F^2 */
double orc_objective(const double *X, const double *Bd, int m, int n, int r,
                     const double *C, int p, int cr, const double *D, int q,
                     int cc, int bc, double lambda)
{
    size_t N = (size_t)m * n;
    double *T = (double *)malloc(sizeof(double) * N);
    double f = 0.0, g = 0.0;
    orc_kron_apply(X, m, n, r, C, p, cr, D, q, cc, bc, T);
    for (size_t t = 0; t < N; ++t) {
        double e = T[t] - Bd[t];
        f += e * e;
        g += X[t] * X[t];
    }
    free(T);
    return 0.5 * f + 0.5 * lambda * lambda * g;
}

/* Soft threshold S_mu(v) = sign(v) max(|v| - mu, 0): the prox of mu |x|. */
static double soft_threshold(double v, double mu)
{
    if (v > mu) return v - mu;
    if (v < -mu) return v + mu;
    return 0.0;
}

/* sFISTA, Alg. 2, with X_0 = 0 (so Y_1 = 0) and a fixed iteration count.
 *   Step 1: X_k = (L Y_k - sum_j B_j^T (sum_i B_i Y_k A_i^T - B) A_j) / (L + lambda^2)
 *           (optionally followed by max(X_k, 0): the prox of the
 *            non-negativity constraint the introduction motivates)
 *           With mu > 0 the regulariser is g(x) = lambda^2/2 |x|^2 + mu |x|_1
 *           (the l1 term Sec. 1 and Sec. 5 name for future work), and the
 *           minimiser of Q_L(x, Y_k) of Sec. 3.1 is, element by element,
 *           S_mu(L Y_k - grad f(Y_k)) / (L + lambda^2).
 *   Step 2: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  t_1 = 1
 *   Step 3: Y_{k+1} = X_k + (t_k - 1)/t_{k+1} (X_k - X_{k-1})
 * If X_start/Xprev_start are non-NULL the loop resumes from (X_{k0},
 * X_{k0-1}) at iteration k0 + 1 (t_k depends on k only).  Writes X_iters
 * to X_out and, if Xprev_out is non-NULL, X_{iters-1} to Xprev_out. */
void orc_sfista(const double *Bd, int m, int n, int r, const double *C, int p,
                int cr, const double *D, int q, int cc, int bc, double L,
                double lambda, int iters, int project, double mu, int k0,
                const double *X_start, const double *Xprev_start,
                double *X_out, double *Xprev_out)
{
    size_t N = (size_t)m * n;
    double *X = (double *)calloc(N, sizeof(double));
    double *Xp = (double *)calloc(N, sizeof(double));
    double *Y = (double *)calloc(N, sizeof(double));
    double *R = (double *)malloc(sizeof(double) * N);
    double *G = (double *)malloc(sizeof(double) * N);
    double t = 1.0;
    double lam2 = lambda * lambda;
    if (X_start) memcpy(X, X_start, sizeof(double) * N);
    if (Xprev_start) memcpy(Xp, Xprev_start, sizeof(double) * N);
    for (int k = 1; k <= k0; ++k) t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    if (k0 > 0) {
        /* Y_{k0+1} from X_{k0}, X_{k0-1} with t_{k0} -> t_{k0+1} */
        double tprev = 1.0;
        for (int k = 1; k < k0; ++k) tprev = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tprev * tprev));
        double beta = (tprev - 1.0) / t;
        for (size_t s = 0; s < N; ++s) Y[s] = X[s] + beta * (X[s] - Xp[s]);
    } else {
        memcpy(Y, X, sizeof(double) * N);
    }
    for (int k = k0 + 1; k <= k0 + iters; ++k) {
        orc_kron_apply(Y, m, n, r, C, p, cr, D, q, cc, bc, R);
        for (size_t s = 0; s < N; ++s) R[s] -= Bd[s];
        orc_kron_apply_T(R, m, n, r, C, p, cr, D, q, cc, bc, G);
        memcpy(Xp, X, sizeof(double) * N);
        for (size_t s = 0; s < N; ++s) {
            double v = L * Y[s] - G[s];
            if (mu > 0.0) v = soft_threshold(v, mu);
            double x = v / (L + lam2);
            if (project && x < 0.0) x = 0.0;
            X[s] = x;
        }
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double beta = (t - 1.0) / tn;
        for (size_t s = 0; s < N; ++s) Y[s] = X[s] + beta * (X[s] - Xp[s]);
        t = tn;
    }
    memcpy(X_out, X, sizeof(double) * N);
    if (Xprev_out) memcpy(Xprev_out, Xp, sizeof(double) * N);
    free(X);
    free(Xp);
    free(Y);
    free(R);
    free(G);
}

/* Vector FISTA on an explicit N x N matrix A (Alg. 1), x_0 = 0:
 *   x_k = S_mu(L y_k - A^T (A y_k - b)) / (L + lambda^2) (mu = 0: no
 *   threshold), then Steps 2-3. */
void orc_fista_dense(const double *A, const double *b, int N, double L,
                     double lambda, double mu, int iters, double *x_out)
{
    double *x = (double *)calloc((size_t)N, sizeof(double));
    double *xp = (double *)calloc((size_t)N, sizeof(double));
    double *y = (double *)calloc((size_t)N, sizeof(double));
    double *r = (double *)malloc(sizeof(double) * (size_t)N);
    double t = 1.0, lam2 = lambda * lambda;
    for (int k = 1; k <= iters; ++k) {
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int j = 0; j < N; ++j) s += A[(size_t)i * N + j] * y[j];
            r[i] = s - b[i];
        }
        memcpy(xp, x, sizeof(double) * (size_t)N);
        for (int j = 0; j < N; ++j) {
            double g = 0.0;
            for (int i = 0; i < N; ++i) g += A[(size_t)i * N + j] * r[i];
            double v = L * y[j] - g;
            if (mu > 0.0) v = soft_threshold(v, mu);
            x[j] = v / (L + lam2);
        }
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        for (int j = 0; j < N; ++j) y[j] = x[j] + (t - 1.0) / tn * (x[j] - xp[j]);
        t = tn;
    }
    memcpy(x_out, x, sizeof(double) * (size_t)N);
    free(x);
    free(xp);
    free(y);
    free(r);
}

/* Vector FISTA (Alg. 1) on the exact blur A of Eq. (1.1), no Kronecker
 * approximation, x_0 = 0 and a fixed iteration count.  The vector x is the
 * image X (any fixed ordering of its pixels gives the same element-wise
 * steps); A x is orc_blur and A^T r is orc_blur_T:
 *   Step 1: x_k = (L y_k - A^T (A y_k - b)) / (L + lambda^2)
 *   Step 2: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  t_1 = 1
 *   Step 3: y_{k+1} = x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1})          */
void orc_fista_exact(const double *Bd, int m, int n, const double *P, int p,
                     int q, int cr, int cc, int bc, double L, double lambda,
                     int iters, double *X_out)
{
    size_t N = (size_t)m * n;
    double *x = (double *)calloc(N, sizeof(double));
    double *xp = (double *)calloc(N, sizeof(double));
    double *y = (double *)calloc(N, sizeof(double));
    double *r = (double *)malloc(sizeof(double) * N);
    double *g = (double *)malloc(sizeof(double) * N);
    double t = 1.0, lam2 = lambda * lambda;
    for (int k = 1; k <= iters; ++k) {
        orc_blur(y, m, n, P, p, q, cr, cc, bc, r);
        for (size_t s = 0; s < N; ++s) r[s] -= Bd[s];
        orc_blur_T(r, m, n, P, p, q, cr, cc, bc, g);
        memcpy(xp, x, sizeof(double) * N);
        for (size_t s = 0; s < N; ++s) x[s] = (L * y[s] - g[s]) / (L + lam2);
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        for (size_t s = 0; s < N; ++s) y[s] = x[s] + (t - 1.0) / tn * (x[s] - xp[s]);
        t = tn;
    }
    memcpy(X_out, x, sizeof(double) * N);
    free(x);
    free(xp);
    free(y);
    free(r);
    free(g);
}

/* Largest eigenvalue of A^T A for the exact blur by power iteration from
 * X0 (overwritten), stopping rule as orc_power_lipschitz. */
double orc_power_lipschitz_exact(double *X0, int m, int n, const double *P,
                                 int p, int q, int cr, int cc, int bc,
                                 double tol, int maxit, int *iters_out)
{
    size_t N = (size_t)m * n;
    double *T = (double *)malloc(sizeof(double) * N);
    double *U = (double *)malloc(sizeof(double) * N);
    double nrm = 0.0, mu = 0.0, prev = 0.0;
    int it = 0;
    for (size_t t = 0; t < N; ++t) nrm += X0[t] * X0[t];
    nrm = sqrt(nrm);
    for (size_t t = 0; t < N; ++t) X0[t] /= nrm;
    for (it = 1; it <= maxit; ++it) {
        orc_blur(X0, m, n, P, p, q, cr, cc, bc, T);
        orc_blur_T(T, m, n, P, p, q, cr, cc, bc, U);
        mu = 0.0;
        nrm = 0.0;
        for (size_t t = 0; t < N; ++t) {
            mu += X0[t] * U[t];
            nrm += U[t] * U[t];
        }
        nrm = sqrt(nrm);
        if (nrm == 0.0) break;
        for (size_t t = 0; t < N; ++t) X0[t] = U[t] / nrm;
        if (it > 1 && fabs(mu - prev) <= tol * fabs(mu)) break;
        prev = mu;
    }
    if (iters_out) *iters_out = it;
    free(T);
    free(U);
    return mu;
}

/* Number of OpenMP threads for the following calls (n <= 0: leave unchanged);
 * returns the number in effect (1 without OpenMP).  For timing only. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
