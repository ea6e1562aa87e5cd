// Host-side setup of the Kronecker approximation in FP64 (Sec. 2, Theorem 1).
//
// The blur A(P) of Eq. (1.1) is linear in the PSF entries; with M_i the 1-D
// operator that a unit column profile at offset i induces on the row index
// (under the boundary condition) and G_r[i][i'] = <M_i, M_i'>_F its Gram
// matrix, ||A(Q)||_F = ||R_r Q R_c^T||_F with R^T R = G.  The best rank-r
// Kronecker sum therefore comes from the truncated SVD of the weighted PSF
// P_bar = R_r P R_c^T (Theorem 1), with factor profiles
//     c_k = sqrt(s_k) R_r^{-1} u_k   (left factor B_k, acts on rows index),
//     d_k = sqrt(s_k) R_c^{-1} v_k   (right factor A_k, acts on column index).
// For the zero boundary G is diag(n - |i - l|) (W_a^2 of Theorem 1); for the
// reflective one it is the Toeplitz matrix with first row [n, 1, 0, 1, ...].
// The Gram entries are counted from their definition here.
//
// Orientation: the left factor is built from u_k (the PSF's row direction)
// and the right one from v_k.  Sec. 2 states the opposite assignment, which
// reproduces A only for P = P^T under the paper's own column-stacking vec.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "internal.h"

namespace sfista {

namespace {

// Source index of extended pixel t on an axis of len pixels, -1 if zero.
// Reflective boundary: half-sample reflection, one reflection deep.
int ext_index(int t, int len, int bc) {
    if (t >= 0 && t < len) return t;
    if (bc == SFISTA_BC_ZERO) return -1;
    t = (t < 0) ? -1 - t : 2 * len - 1 - t;
    return (t >= 0 && t < len) ? t : -1;
}

// G[i][j] = #{a : ext(a - i + c) == ext(a - j + c) valid}, p x p row-major.
void gram(int p, int centre, int len, int bc, std::vector<double> *G) {
    G->assign((size_t)p * p, 0.0);
    std::vector<int> idx(p);
    for (int a = 0; a < len; ++a) {
        for (int i = 0; i < p; ++i) idx[i] = ext_index(a - i + centre, len, bc);
        for (int i = 0; i < p; ++i) {
            if (idx[i] < 0) continue;
            for (int j = 0; j < p; ++j)
                if (idx[j] == idx[i]) (*G)[(size_t)i * p + j] += 1.0;
        }
    }
}

// Upper Cholesky factor R (R^T R = G), p x p row-major.  false if not SPD.
bool cholesky_upper(const std::vector<double> &G, int p, std::vector<double> *R) {
    R->assign((size_t)p * p, 0.0);
    std::vector<double> &U = *R;
    for (int j = 0; j < p; ++j) {
        double s = G[(size_t)j * p + j];
        for (int k = 0; k < j; ++k) s -= U[(size_t)k * p + j] * U[(size_t)k * p + j];
        if (!(s > 0.0)) return false;
        double d = sqrt(s);
        U[(size_t)j * p + j] = d;
        for (int i = j + 1; i < p; ++i) {
            double t = G[(size_t)j * p + i];
            for (int k = 0; k < j; ++k) t -= U[(size_t)k * p + j] * U[(size_t)k * p + i];
            U[(size_t)j * p + i] = t / d;
        }
    }
    return true;
}

// Solve R x = y for upper-triangular R (back substitution), in place on y.
void solve_upper(const std::vector<double> &R, int p, double *y) {
    for (int i = p - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < p; ++k) s -= R[(size_t)i * p + k] * y[k];
        y[i] = s / R[(size_t)i * p + i];
    }
}

// One-sided (Hestenes) Jacobi SVD of a rows x cols matrix with rows >= cols,
// column-major working copy W (rows x cols).  On return the columns of W are
// U * diag(s) and V (cols x cols, column-major) holds the right vectors.
void jacobi_svd_tall(int rows, int cols, std::vector<double> *W, std::vector<double> *V) {
    V->assign((size_t)cols * cols, 0.0);
    for (int j = 0; j < cols; ++j) (*V)[(size_t)j * cols + j] = 1.0;
    double *w = W->data(), *v = V->data();
    for (int sweep = 0; sweep < 80; ++sweep) {
        int rotated = 0;
        for (int j = 0; j < cols - 1; ++j) {
            for (int k = j + 1; k < cols; ++k) {
                double *wj = w + (size_t)j * rows, *wk = w + (size_t)k * rows;
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < rows; ++i) {
                    al += wj[i] * wj[i];
                    be += wk[i] * wk[i];
                    ga += wj[i] * wk[i];
                }
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                ++rotated;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < rows; ++i) {
                    double a = wj[i], b = wk[i];
                    wj[i] = c * a - s * b;
                    wk[i] = s * a + c * b;
                }
                double *vj = v + (size_t)j * cols, *vk = v + (size_t)k * cols;
                for (int i = 0; i < cols; ++i) {
                    double a = vj[i], b = vk[i];
                    vj[i] = c * a - s * b;
                    vk[i] = s * a + c * b;
                }
            }
        }
        if (!rotated) break;
    }
}

// Full SVD of a p x q row-major matrix: s (min(p,q), descending), U (p x k)
// and V (q x k) column-major with k = min(p, q).
void svd(const std::vector<double> &M, int p, int q, std::vector<double> *s,
         std::vector<double> *U, std::vector<double> *V) {
    bool tall = p >= q;
    int rows = tall ? p : q, cols = tall ? q : p;
    std::vector<double> W((size_t)rows * cols), R;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < q; ++j) {
            if (tall) W[(size_t)j * rows + i] = M[(size_t)i * q + j];   // column j of M
            else W[(size_t)i * rows + j] = M[(size_t)i * q + j];         // column i of M^T
        }
    jacobi_svd_tall(rows, cols, &W, &R);
    int k = cols;
    std::vector<double> sv(k);
    for (int j = 0; j < k; ++j) {
        double t = 0;
        for (int i = 0; i < rows; ++i) t += W[(size_t)j * rows + i] * W[(size_t)j * rows + i];
        sv[j] = sqrt(t);
    }
    std::vector<int> ord(k);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
    // Left vectors of the tall problem: W_j / s_j; right: R_j.
    std::vector<double> Lv((size_t)rows * k, 0.0), Rv((size_t)cols * k, 0.0);
    s->assign(k, 0.0);
    for (int jj = 0; jj < k; ++jj) {
        int j = ord[jj];
        (*s)[jj] = sv[j];
        for (int i = 0; i < cols; ++i) Rv[(size_t)jj * cols + i] = R[(size_t)j * cols + i];
        if (sv[j] > 0)
            for (int i = 0; i < rows; ++i) Lv[(size_t)jj * rows + i] = W[(size_t)j * rows + i] / sv[j];
    }
    if (tall) {
        *U = Lv;   // p x k
        *V = Rv;   // q x k
    } else {
        *U = Rv;   // p x k (right vectors of M^T)
        *V = Lv;   // q x k
    }
}

// Band storage of the r 1-D factors built from profiles prof (r x p, centre c)
// on an axis of len pixels; transpose = true stores F^T.
void make_band(const std::vector<double> &prof, int r, int p, int centre, int len,
               int bc, bool transpose, Band *out) {
    int lo = 1 << 30, hi = -(1 << 30);
    for (int a = 0; a < len; ++a)
        for (int k = 0; k < p; ++k) {
            int e = ext_index(a - k + centre, len, bc);
            if (e < 0) continue;
            int off = transpose ? a - e : e - a;
            lo = std::min(lo, off);
            hi = std::max(hi, off);
        }
    if (lo > hi) lo = hi = 0;
    out->len = len;
    out->r = r;
    out->lo = lo;
    out->w = hi - lo + 1;
    out->band.assign((size_t)r * out->w * len, 0.0);
    for (int i = 0; i < r; ++i)
        for (int a = 0; a < len; ++a)
            for (int k = 0; k < p; ++k) {
                int e = ext_index(a - k + centre, len, bc);
                if (e < 0) continue;
                int row = transpose ? e : a;
                int off = transpose ? a - e : e - a;
                out->band[((size_t)i * out->w + (off - lo)) * len + row] += prof[(size_t)i * p + k];
            }
}

}  // namespace

sfista_status host_setup(const double *psf, int p, int q, int cr, int cc, int m, int n,
                         int bc, int r, HostSetup *out) {
    if (!psf) return fail(SFISTA_EINVAL, "psf is NULL");
    if (p < 1 || q < 1) return fail(SFISTA_EINVAL, "PSF size must be positive");
    if (m < 1 || n < 1) return fail(SFISTA_EINVAL, "image size must be positive");
    if (bc == SFISTA_BC_PERIODIC)
        return fail(SFISTA_ENOTSUP, "periodic boundary is not supported (Sec. 2 excludes it)");
    if (bc != SFISTA_BC_ZERO && bc != SFISTA_BC_REFLEXIVE)
        return fail(SFISTA_EINVAL, "unknown boundary condition");
    if (p > m || q > n) return fail(SFISTA_EINVAL, "PSF larger than the image");
    if (cr < 0 || cr >= p || cc < 0 || cc >= q) return fail(SFISTA_EINVAL, "PSF centre outside the PSF");
    int kmax = std::min(p, q);
    if (r < 1 || r > kmax) return fail(SFISTA_EINVAL, "rank r must be in [1, min(psf_rows, psf_cols)]");
    for (size_t t = 0; t < (size_t)p * q; ++t)
        if (!isfinite(psf[t])) return fail(SFISTA_EINVAL, "PSF has a non-finite entry");

    std::vector<double> Gr, Gc, Rr, Rc;
    gram(p, cr, m, bc, &Gr);
    gram(q, cc, n, bc, &Gc);
    if (!cholesky_upper(Gr, p, &Rr) || !cholesky_upper(Gc, q, &Rc))
        return fail(SFISTA_EINVAL, "Gram matrix of the boundary condition is not positive definite");
    // P_bar = Rr P Rc^T
    std::vector<double> T((size_t)p * q, 0.0), Pb((size_t)p * q, 0.0);
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < q; ++j) {
            double s = 0;
            for (int k = i; k < p; ++k) s += Rr[(size_t)i * p + k] * psf[(size_t)k * q + j];
            T[(size_t)i * q + j] = s;
        }
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < q; ++j) {
            double s = 0;
            for (int k = j; k < q; ++k) s += T[(size_t)i * q + k] * Rc[(size_t)j * q + k];
            Pb[(size_t)i * q + j] = s;
        }
    std::vector<double> sv, U, V;
    svd(Pb, p, q, &sv, &U, &V);
    if (r < kmax && sv[r] > 1e-14 * sv[0] && sv[r - 1] - sv[r] <= 1e-12 * sv[0])
        return fail(SFISTA_EINVAL, "singular values s_r and s_{r+1} of the weighted PSF tie; "
                                   "the rank-r truncation is not unique");

    out->m = m; out->n = n; out->p = p; out->q = q; out->cr = cr; out->cc = cc;
    out->bc = bc; out->r = r;
    out->sigma = sv;
    double tail = 0;
    for (int k = r; k < kmax; ++k) tail += sv[k] * sv[k];
    out->approx_err = sqrt(tail);
    out->C.assign((size_t)r * p, 0.0);
    out->D.assign((size_t)r * q, 0.0);
    for (int k = 0; k < r; ++k) {
        double *u = &U[(size_t)k * p], *v = &V[(size_t)k * q];
        int imax = 0;
        for (int i = 1; i < p; ++i) if (fabs(u[i]) > fabs(u[imax])) imax = i;
        double sg = u[imax] < 0 ? -1.0 : 1.0;
        double rs = sqrt(sv[k]);
        std::vector<double> cu(p), dv(q);
        for (int i = 0; i < p; ++i) cu[i] = sg * rs * u[i];
        for (int j = 0; j < q; ++j) dv[j] = sg * rs * v[j];
        solve_upper(Rr, p, cu.data());
        solve_upper(Rc, q, dv.data());
        std::copy(cu.begin(), cu.end(), out->C.begin() + (size_t)k * p);
        std::copy(dv.begin(), dv.end(), out->D.begin() + (size_t)k * q);
    }
    make_band(out->D, r, q, cc, n, bc, false, &out->A);
    make_band(out->D, r, q, cc, n, bc, true, &out->AT);
    make_band(out->C, r, p, cr, m, bc, false, &out->B);
    make_band(out->C, r, p, cr, m, bc, true, &out->BT);
    return SFISTA_OK;
}

void band_interior(const float *tbl, int len, int cnt, int *i0, int *i1) {
    const int ref = len / 2;
    auto same = [&](int row) {
        for (int t = 0; t < cnt; ++t)
            if (memcmp(&tbl[(size_t)t * len + row], &tbl[(size_t)t * len + ref], sizeof(float))) return false;
        return true;
    };
    int a = ref, b = ref + 1;
    while (a > 0 && same(a - 1)) --a;
    while (b < len && same(b)) ++b;
    *i0 = a;
    *i1 = b;
}

void momentum_table(int k_end, std::vector<double> *beta) {
    beta->assign(std::max(k_end, 1), 0.0);
    double t = 1.0;
    for (int k = 1; k <= k_end; ++k) {
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        (*beta)[k - 1] = (t - 1.0) / tn;
        t = tn;
    }
}

}  // namespace sfista
