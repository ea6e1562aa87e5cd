"""Pins of the oracle's reverse mode: FP64 central finite differences of the
unrolled solve on tiny problems (every entry of the gradient), and agreement
of its forward with the convolution-based oracle solve (Alg. 2)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, kron
from paper_1901_00913_gb300 import workloads as W


def _setup(seed=41, m=7, n=6, r=2, bc=1):
    g = W.rng(seed)
    P = W.random_psf(g, 5, 5)
    ka = kron.kron_approx(P, 2, 2, m, n, bc, r)
    Bf, Af = kron.dense_factors(ka)
    x = g.uniform(size=(m, n))
    Bd = oracle.blur(x, P, 2, 2, bc) + 0.01 * g.standard_normal((m, n))
    return ka, Af, Bf, Bd, x


def test_dense_forward_matches_convolution_oracle():
    ka, A, B, Bd, x = _setup()
    X = adjoint.unrolled_forward(Bd, A, B, 1.3, 0.07, 9)[0]
    np.testing.assert_allclose(X, oracle.sfista(Bd, ka, 1.3, 0.07, 9), atol=1e-13)


@pytest.mark.parametrize("K", [1, 2, 5])
def test_reverse_mode_matches_central_differences(K):
    ka, A, B, Bd, x = _setup(seed=42 + K)
    L, lam = 1.2, 0.1

    def f(Bd_, A_, B_, lam_):
        return adjoint.loss_true(Bd_, A_, B_, L, lam_, K, x)[0]

    gX = adjoint.loss_true(Bd, A, B, L, lam, K, x)[1]
    gB, glam, gA, gBf = adjoint.unrolled_grad(Bd, A, B, L, lam, K, gX)
    eps = 1e-6
    fd = np.zeros_like(Bd)
    for idx in np.ndindex(Bd.shape):
        E = np.zeros_like(Bd)
        E[idx] = eps
        fd[idx] = (f(Bd + E, A, B, lam) - f(Bd - E, A, B, lam)) / (2 * eps)
    np.testing.assert_allclose(gB, fd, rtol=1e-6, atol=1e-9)
    fdl = (f(Bd, A, B, lam + eps) - f(Bd, A, B, lam - eps)) / (2 * eps)
    assert abs(glam - fdl) <= 1e-6 * max(1.0, abs(fdl))
    for F, G, which in ((A, gA, "A"), (B, gBf, "B")):
        for idx in list(np.ndindex(F.shape))[::3]:
            E = np.zeros_like(F)
            E[idx] = eps
            if which == "A":
                fdv = (f(Bd, F + E, B, lam) - f(Bd, F - E, B, lam)) / (2 * eps)
            else:
                fdv = (f(Bd, A, F + E, lam) - f(Bd, A, F - E, lam)) / (2 * eps)
            assert abs(G[idx] - fdv) <= 1e-6 * max(1e-3, abs(fdv)), (which, idx, G[idx], fdv)


def test_reverse_mode_catches_a_dropped_momentum_term():
    """Planted mistake: dropping the x_bar_{k-2} update changes the gradient well beyond FD error."""
    ka, A, B, Bd, x = _setup(seed=47)
    L, lam, K = 1.2, 0.1, 5
    gX = adjoint.loss_true(Bd, A, B, L, lam, K, x)[1]
    gB = adjoint.unrolled_grad(Bd, A, B, L, lam, K, gX)[0]
    orig = adjoint.unrolled_grad

    def broken(Bd_, A_, B_, L_, lam_, K_, gX_):
        Xs = adjoint.unrolled_forward(Bd_, A_, B_, L_, lam_, K_)
        betas = Xs[3]
        xbar = {K_: gX_.copy()}
        gB_ = np.zeros_like(Bd_)
        for k in range(K_, 0, -1):
            V = xbar.pop(k, np.zeros_like(Bd_))
            W_ = adjoint._As(V, A_, B_)
            ybar = (L_ * V - adjoint._AsT(W_, A_, B_)) / (L_ + lam_ ** 2)
            gB_ += W_ / (L_ + lam_ ** 2)
            if k >= 2:
                xbar[k - 1] = xbar.get(k - 1, 0.0) + (1.0 + betas[k - 2]) * ybar
        return gB_

    assert orig is adjoint.unrolled_grad
    assert np.linalg.norm(broken(Bd, A, B, L, lam, K, gX) - gB) > 1e-4 * np.linalg.norm(gB)
