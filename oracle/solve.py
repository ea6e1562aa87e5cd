"""sFISTA driver, exact blur and metrics in FP64 (test infrastructure only).

Thin numpy wrappers over ``sfista_oracle.c`` plus the scalar pieces of
Alg. 2 that are easiest to read in Python.
"""
import ctypes

import numpy as np

from . import _native


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _prof(ka):
    return _f64(ka.C), ka.C.shape[1], _f64(ka.D), ka.D.shape[1]


def blur(X, P, cr, cc, bc):
    """Exact blur A x of Eq. (1.1) with the given boundary condition."""
    X, P = _f64(X), _f64(P)
    m, n = X.shape
    Y = np.empty_like(X)
    _native.lib().orc_blur(X, m, n, P, P.shape[0], P.shape[1], cr, cc, bc, Y)
    return Y


def blur_T(X, P, cr, cc, bc):
    """A^T x for the exact blur (scatter through the same index map)."""
    X, P = _f64(X), _f64(P)
    m, n = X.shape
    Y = np.empty_like(X)
    _native.lib().orc_blur_T(X, m, n, P, P.shape[0], P.shape[1], cr, cc, bc, Y)
    return Y


def kron_apply(Y, ka):
    """sum_k B_k Y A_k^T (Eq. matrix equation), factors applied as 1-D convolutions."""
    Y = _f64(Y)
    m, n = Y.shape
    C, p, D, q = _prof(ka)
    out = np.empty_like(Y)
    _native.lib().orc_kron_apply(Y, m, n, ka.r, C, p, ka.cr, D, q, ka.cc, ka.bc, out)
    return out


def kron_apply_T(R, ka):
    """sum_k B_k^T R A_k, the adjoint used in Step 1 of Alg. 2."""
    R = _f64(R)
    m, n = R.shape
    C, p, D, q = _prof(ka)
    out = np.empty_like(R)
    _native.lib().orc_kron_apply_T(R, m, n, ka.r, C, p, ka.cr, D, q, ka.cc, ka.bc, out)
    return out


def lipschitz(ka, X0, tol=1e-13, maxit=2000):
    """lambda_max(A_s^T A_s) by power iteration from the start image X0.

    Reading of the paper: Step 1 of Alg. 2 needs L >= lambda_max(A_s^T A_s)
    for the problem it actually solves, so L is taken for A_s, not A.
    Returns (L, iterations).
    """
    X = _f64(X0).copy()
    m, n = X.shape
    C, p, D, q = _prof(ka)
    it = ctypes.c_int(0)
    L = _native.lib().orc_power_lipschitz(X, m, n, ka.r, C, p, ka.cr, D, q, ka.cc,
                                           ka.bc, tol, maxit, ctypes.byref(it))
    return float(L), int(it.value)


def objective(X, Bd, ka, lam):
    """Phi_s(X) = 0.5 ||A_s X - B||_F^2 + 0.5 lam^2 ||X||_F^2."""
    X, Bd = _f64(X), _f64(Bd)
    m, n = X.shape
    C, p, D, q = _prof(ka)
    return float(_native.lib().orc_objective(X, Bd, m, n, ka.r, C, p, ka.cr, D, q,
                                             ka.cc, ka.bc, lam))


def sfista(Bd, ka, L, lam, iters, project=False, k0=0, X_start=None,
           Xprev_start=None, return_prev=False, mu=0.0):
    """Alg. 2 from X_0 = 0 (or resumed at iteration k0 from (X_k0, X_k0-1)).

    mu > 0 adds mu ||X||_1 to the regulariser: Step 1 becomes the minimiser
    of Q_L (Sec. 3.1), S_mu(L Y - grad f(Y)) / (L + lam^2) element by element."""
    Bd = _f64(Bd)
    m, n = Bd.shape
    C, p, D, q = _prof(ka)
    X = np.empty_like(Bd)
    Xp = np.empty_like(Bd)
    xs = _f64(X_start) if X_start is not None else None
    xps = _f64(Xprev_start) if Xprev_start is not None else None
    _native.lib().orc_sfista(
        Bd, m, n, ka.r, C, p, ka.cr, D, q, ka.cc, ka.bc, float(L), float(lam),
        int(iters), int(bool(project)), float(mu), int(k0),
        xs.ctypes.data if xs is not None else None,
        xps.ctypes.data if xps is not None else None,
        X, Xp.ctypes.data)
    return (X, Xp) if return_prev else X


def fista_dense(A, b, L, lam, iters, mu=0.0):
    """Alg. 1 (vector FISTA) on an explicit matrix, x_0 = 0 (mu: l1 weight)."""
    A, b = _f64(A), _f64(b)
    x = np.empty_like(b)
    _native.lib().orc_fista_dense(A, b, b.shape[0], float(L), float(lam), float(mu), int(iters), x)
    return x


def fista_exact(Bd, P, cr, cc, bc, L, lam, iters):
    """Alg. 1 (vector FISTA) on the exact blur A of Eq. (1.1), x_0 = 0: the
    comparison system of Sec. 4 (no Kronecker approximation)."""
    Bd, P = _f64(Bd), _f64(P)
    m, n = Bd.shape
    X = np.empty_like(Bd)
    _native.lib().orc_fista_exact(Bd, m, n, P, P.shape[0], P.shape[1], int(cr), int(cc), int(bc), float(L),
                                  float(lam), int(iters), X)
    return X


def lipschitz_exact(P, cr, cc, bc, X0, tol=1e-13, maxit=2000):
    """lambda_max(A^T A) of the exact blur by power iteration from X0; returns (L, iterations)."""
    X, P = _f64(X0).copy(), _f64(P)
    m, n = X.shape
    it = ctypes.c_int(0)
    L = _native.lib().orc_power_lipschitz_exact(X, m, n, P, P.shape[0], P.shape[1], int(cr), int(cc), int(bc),
                                                tol, maxit, ctypes.byref(it))
    return float(L), int(it.value)


def t_schedule(iters):
    """t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 (Alg. 2, Step 2); returns t_1..t_{iters+1}."""
    t = [1.0]
    for _ in range(iters):
        t.append(0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t[-1] * t[-1])))
    return np.array(t)


def rel_fro(X, Xref):
    """||X - Xref||_F / ||Xref||_F."""
    X = np.asarray(X, dtype=np.float64)
    Xref = np.asarray(Xref, dtype=np.float64)
    return float(np.linalg.norm(X - Xref) / np.linalg.norm(Xref))


def psnr(X, Xtrue, peak=1.0):
    """10 log10(peak^2 / MSE(X, Xtrue))."""
    X = np.asarray(X, dtype=np.float64)
    mse = float(np.mean((X - np.asarray(Xtrue, dtype=np.float64)) ** 2))
    return 10.0 * np.log10(peak * peak / mse)
