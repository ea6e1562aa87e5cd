"""Kronecker-product approximation of the blur matrix (Sec. 2, Theorem 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The blur A of Eq. (1.1) is linear in the PSF: A(P) = sum_{i,j} P[i][j] *
(N_j kron M_i), where M_i (m x m) is the 1-D operator that a unit column
profile at offset i induces on the row index and N_j (n x n) the one a unit
row profile induces on the column index, each under the boundary condition.
Hence ||A(Q)||_F^2 = trace(Q^T G_r Q G_c) with the Gram matrices
G_r[i][i'] = <M_i, M_i'>_F and G_c likewise, and with G = R^T R (R upper
triangular, MATLAB's chol) the best rank-s approximation is the truncated SVD
of the weighted PSF  P_bar = R_r P R_c^T  (Theorem 1):

    c_k = sqrt(sigma_k) R_r^{-1} u_k    (column profile -> left factor B_k)
    d_k = sqrt(sigma_k) R_c^{-1} v_k    (row profile    -> right factor A_k)

and ||A - sum_k A_k kron B_k||_F = sqrt(sum_{k>s} sigma_k^2).

Reading of the paper: Sec. 2 builds the right factor K_i from u_i and the
left factor H_i from v_i; under its own column-stacking vec (Eq. matrix
equation) that is the transpose of what reproduces A for a non-symmetric
PSF, so here the left factor comes from u_k and the right one from v_k.  The
two agree whenever P = P^T.

The Gram matrices are computed from their definition by counting coincident
entries of M_i and M_i' (each row of M_i holds a single 1 at the extended
index a - i + centre); tests compare them with the paper's closed forms
(W_a^2 for the zero boundary, the Toeplitz matrix with first row
[n, 1, 0, 1, 0, ...] for the reflective one).
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg


def ext_index(t, length, bc):
    """Source index of extended pixel t on an axis of ``length`` pixels, or -1.

    bc 0: zero outside; bc 1: half-sample reflection (-1 -> 0, length -> length-1).
    """
    if 0 <= t < length:
        return t
    if bc == 0:
        return -1
    t = -1 - t if t < 0 else 2 * length - 1 - t
    return t if 0 <= t < length else -1


def operator_matrix_1d(profile, centre, length, bc):
    """Dense 1-D factor: M[a][e] = sum_k profile[k] [ext(a - k + centre) == e].

    For bc 0 this is toep(profile, centre) of Sec. 2, for bc 1 toep + hank.
    """
    M = np.zeros((length, length))
    for a in range(length):
        for k, v in enumerate(profile):
            e = ext_index(a - k + centre, length, bc)
            if e >= 0:
                M[a, e] += v
    return M


def gram_matrix(p, centre, length, bc):
    """G[i][i'] = <M_i, M_i'>_F for unit profiles at offsets i, i' in [0, p)."""
    G = np.zeros((p, p))
    for a in range(length):
        idx = [ext_index(a - i + centre, length, bc) for i in range(p)]
        for i in range(p):
            if idx[i] < 0:
                continue
            for j in range(p):
                if idx[j] == idx[i]:
                    G[i, j] += 1.0
    return G


@dataclass
class KronApprox:
    C: np.ndarray       # r x p column profiles c_k (left factors B_k)
    D: np.ndarray       # r x q row profiles d_k (right factors A_k)
    cr: int
    cc: int
    bc: int
    m: int
    n: int
    sigma: np.ndarray   # all singular values of P_bar
    approx_err: float   # sqrt(sum_{k>r} sigma_k^2) = ||A - A_s||_F (Theorem 1)

    @property
    def r(self):
        return self.C.shape[0]


def kron_approx(P, cr, cc, m, n, bc, r, swap_orientation=False):
    """Rank-r Kronecker approximation of the blur for image size m x n.

    ``swap_orientation`` reproduces the paper's literal factor assignment
    (left factor from v, right from u); it exists only so a test can show
    that Theorem 1 fails with it for a non-symmetric PSF.
    """
    P = np.asarray(P, dtype=np.float64)
    p, q = P.shape
    Gr = gram_matrix(p, cr, m, bc)
    Gc = gram_matrix(q, cc, n, bc)
    Rr = np.linalg.cholesky(Gr).T          # upper, Rr^T Rr = Gr
    Rc = np.linalg.cholesky(Gc).T
    Pbar = Rr @ P @ Rc.T
    U, S, Vt = np.linalg.svd(Pbar)
    V = Vt.T
    for k in range(len(S)):
        if U[np.argmax(np.abs(U[:, k])), k] < 0:
            U[:, k] = -U[:, k]
            V[:, k] = -V[:, k]
    C = np.zeros((r, p))
    D = np.zeros((r, q))
    for k in range(r):
        s = np.sqrt(S[k])
        C[k] = s * scipy.linalg.solve_triangular(Rr, U[:, k], lower=False)
        D[k] = s * scipy.linalg.solve_triangular(Rc, V[:, k], lower=False)
    if swap_orientation:
        if p != q:
            raise ValueError("orientation swap needs a square PSF")
        C, D = D.copy(), C.copy()
    err = float(np.sqrt(np.sum(S[r:] ** 2)))
    return KronApprox(C=C, D=D, cr=cr, cc=cc, bc=bc, m=m, n=n, sigma=S,
                      approx_err=err)


def dense_factors(ka):
    """Dense factors: B (r x m x m) left, A (r x n x n) right."""
    B = np.stack([operator_matrix_1d(ka.C[k], ka.cr, ka.m, ka.bc) for k in range(ka.r)])
    A = np.stack([operator_matrix_1d(ka.D[k], ka.cc, ka.n, ka.bc) for k in range(ka.r)])
    return B, A


def explicit_kron_matrix(ka):
    """A_s = sum_k A_k kron B_k acting on column-stacked vec(X) (Eq. Kronecker structure)."""
    B, A = dense_factors(ka)
    N = ka.m * ka.n
    As = np.zeros((N, N))
    for k in range(ka.r):
        As += np.kron(A[k], B[k])
    return As


def explicit_blur_matrix(P, cr, cc, m, n, bc):
    """Exact N x N blur, built column by column as the PSF image of a point source.

    Column t = a0 + b0*m (column-stacked vec) is the blurred image of a single
    bright pixel at (a0, b0) (Sec. 2): the PSF is placed with its centre on the
    point and, for the reflective boundary, also on the point's mirror images
    across each edge, then cropped to the m x n domain.
    """
    P = np.asarray(P, dtype=np.float64)
    p, q = P.shape
    N = m * n
    A = np.zeros((N, N))
    for b0 in range(n):
        for a0 in range(m):
            rows = [a0] if bc == 0 else [a0, -1 - a0, 2 * m - 1 - a0]
            cols = [b0] if bc == 0 else [b0, -1 - b0, 2 * n - 1 - b0]
            img = np.zeros((m, n))
            for ai in rows:
                for bi in cols:
                    for a in range(m):
                        i = a - ai + cr
                        if not 0 <= i < p:
                            continue
                        for b in range(n):
                            j = b - bi + cc
                            if 0 <= j < q:
                                img[a, b] += P[i, j]
            A[:, a0 + b0 * m] = img.flatten(order="F")
    return A
