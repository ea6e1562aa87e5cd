"""Reverse mode of the unrolled sFISTA solve in FP64 (test infrastructure only).

Alg. 2 without projection, from X_0 = 0, K iterations, with the Lipschitz
constant L held fixed (it is an input of the algorithm, not differentiated):

    X_k     = F(Y_k) = (L Y_k - G(Y_k)) / (L + lambda^2)
    G(Y)    = sum_j B_j^T (sum_i B_i Y A_i^T - B) A_j
    Y_{k+1} = X_k + beta_k (X_k - X_{k-1}),   Y_1 = X_0 = 0

The factors are dense matrices here (np.matmul as the primitive), so their
gradients are the dense gradients of the matrix model (Eq. matrix minimization
model) with respect to every entry of A_i (n x n) and B_i (m x m).

Reverse recurrence for a loss l(X_K), written out from the chain rule: with
x_bar_k = dl/dX_k, y_bar_k = dl/dY_k and M = dF/dY (symmetric),

    y_bar_k      = M x_bar_k
    x_bar_{k-1} += (1 + beta_{k-1}) y_bar_k,   x_bar_{k-2} -= beta_{k-1} y_bar_k   (k >= 2)

and the parameter gradients collected at each step (den = L + lambda^2,
R_k = A_s Y_k - B, W = A_s x_bar_k):

    dl/dB       += A_s x_bar_k / den
    dl/dlambda  += <x_bar_k, -2 lambda X_k / den>
    dl/dA_i     -= (R_k^T B_i x_bar_k + W^T B_i Y_k) / den
    dl/dB_i     -= (R_k A_i x_bar_k^T + W A_i Y_k^T) / den
"""
import numpy as np

from .solve import t_schedule


def _As(Y, A, B):
    return sum(B[i] @ Y @ A[i].T for i in range(len(A)))


def _AsT(R, A, B):
    return sum(B[j].T @ R @ A[j] for j in range(len(A)))


def unrolled_forward(Bd, A, B, L, lam, K):
    """Returns X_K and the lists X_0..X_K, Y_1..Y_K and beta_1..beta_K."""
    Bd = np.asarray(Bd, dtype=np.float64)
    den = L + lam * lam
    t = t_schedule(K + 1)
    X = np.zeros_like(Bd)
    Xs, Ys, betas = [X], [], []
    Y = X
    for k in range(1, K + 1):
        Ys.append(Y)
        Xn = (L * Y - _AsT(_As(Y, A, B) - Bd, A, B)) / den
        beta = (t[k - 1] - 1.0) / t[k]
        betas.append(beta)
        Y = Xn + beta * (Xn - X)
        X = Xn
        Xs.append(X)
    return X, Xs, Ys, betas


def unrolled_grad(Bd, A, B, L, lam, K, gX):
    """Gradients (dB, dlambda, dA, dB_factors) of a loss with dl/dX_K = gX."""
    Bd = np.asarray(Bd, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    r = len(A)
    den = L + lam * lam
    XK, Xs, Ys, betas = unrolled_forward(Bd, A, B, L, lam, K)
    xbar = {K: np.array(gX, dtype=np.float64)}
    gB = np.zeros_like(Bd)
    glam = 0.0
    gA = np.zeros_like(A)
    gBf = np.zeros_like(B)
    for k in range(K, 0, -1):
        V = xbar.pop(k, np.zeros_like(Bd))
        Y = Ys[k - 1]
        W = _As(V, A, B)
        ybar = (L * V - _AsT(W, A, B)) / den
        gB += W / den
        glam += float(np.vdot(V, -2.0 * lam * Xs[k] / den))
        R = _As(Y, A, B) - Bd
        for i in range(r):
            gA[i] -= (R.T @ B[i] @ V + W.T @ B[i] @ Y) / den
            gBf[i] -= (R @ A[i] @ V.T + W @ A[i] @ Y.T) / den
        if k >= 2:
            beta = betas[k - 2]            # beta_{k-1}
            xbar[k - 1] = xbar.get(k - 1, 0.0) + (1.0 + beta) * ybar
            xbar[k - 2] = xbar.get(k - 2, 0.0) - beta * ybar
    return gB, glam, gA, gBf


def loss_true(Bd, A, B, L, lam, K, Xtrue):
    """l = ||X_K - X_true||_F^2 and its gradient with respect to X_K."""
    XK = unrolled_forward(Bd, A, B, L, lam, K)[0]
    D = XK - Xtrue
    return float(np.vdot(D, D)), 2.0 * D
