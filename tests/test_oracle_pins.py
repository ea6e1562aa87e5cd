"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed examples, brute-force matrices built from the definition of the blur,
a library routine for a special case, a theorem of the paper, or a closed form.
"""
import os

import numpy as np
import pytest
import scipy.ndimage

import oracle
from oracle import kron
from paper_1901_00913_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), dtype=int, comments="#")


def _from_index(idx, c):
    return np.where(idx > 0, np.asarray(c)[np.maximum(idx, 1) - 1], 0.0)


# ------------------------------------------------------------------ Sec. 2 structure
def test_toep_matches_paper_example():
    """toep(c, 4) printed in Sec. 2 == zero-boundary 1-D factor with centre 4 (1-based)."""
    c = np.array([2.0, 3.0, 5.0, 7.0, 11.0])
    M = kron.operator_matrix_1d(c, 3, 5, bc=0)
    np.testing.assert_array_equal(M, _from_index(_golden("toep_c_j4_5x5.txt"), c))


def test_hank_matches_paper_example():
    """hank(c, 3) printed in Sec. 2 == reflective factor minus its Toeplitz part (centre 3)."""
    c = np.array([2.0, 3.0, 5.0, 7.0, 11.0])
    H = kron.operator_matrix_1d(c, 2, 5, bc=1) - kron.operator_matrix_1d(c, 2, 5, bc=0)
    np.testing.assert_array_equal(H, _from_index(_golden("hank_c_j3_5x5.txt"), c))


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape,centre,img", [((5, 5), (2, 2), (7, 6)),
                                              ((3, 4), (0, 2), (6, 5)),
                                              ((4, 3), (3, 1), (5, 7))])
def test_blur_matches_point_source_matrix(bc, shape, centre, img):
    """Eq. (1.1): column t of A is the PSF image of a point source at pixel t (Sec. 2)."""
    g = W.rng(11)
    P = W.random_psf(g, *shape)
    m, n = img
    A = kron.explicit_blur_matrix(P, centre[0], centre[1], m, n, bc)
    X = g.standard_normal((m, n))
    Y = oracle.blur(X, P, centre[0], centre[1], bc)
    np.testing.assert_allclose(Y.flatten(order="F"), A @ X.flatten(order="F"), atol=1e-14)
    Z = oracle.blur_T(X, P, centre[0], centre[1], bc)
    np.testing.assert_allclose(Z.flatten(order="F"), A.T @ X.flatten(order="F"), atol=1e-14)


@pytest.mark.parametrize("bc,mode", [(0, "constant"), (1, "reflect")])
def test_blur_matches_scipy_convolve(bc, mode):
    """Centred odd PSF: zero / reflective blur == scipy.ndimage.convolve constant / reflect."""
    g = W.rng(12)
    X = g.uniform(size=(40, 33))
    P = W.rotated_gaussian_psf(9, 2.5, 1.0, 0.4)
    Y = oracle.blur(X, P, 4, 4, bc)
    Ys = scipy.ndimage.convolve(X, P, mode=mode, cval=0.0)
    np.testing.assert_allclose(Y, Ys, rtol=0, atol=1e-14)


# ------------------------------------------------------------------ Theorem 1
@pytest.mark.parametrize("m,p", [(9, 5), (16, 7), (40, 11)])
def test_gram_zero_bc_is_W_squared(m, p):
    """Zero boundary: Gram = diag(n - |i - l|) = W_a^2 of Theorem 1."""
    for cr in (0, p // 2, p - 1):
        G = kron.gram_matrix(p, cr, m, 0)
        np.testing.assert_array_equal(G, np.diag([m - abs(i - cr) for i in range(p)]))


@pytest.mark.parametrize("m,p", [(9, 5), (16, 7), (40, 11)])
def test_gram_reflective_is_paper_toeplitz(m, p):
    """Reflective boundary: Gram = symmetric Toeplitz with first row [n, 1, 0, 1, 0, ...] (Theorem 1)."""
    row = np.array([m] + [1.0 if k % 2 else 0.0 for k in range(1, p)])
    T = scipy.linalg.toeplitz(row)
    for cr in (0, p // 2, p - 1):
        np.testing.assert_array_equal(kron.gram_matrix(p, cr, m, 1), T)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_theorem1_equality(bc, r):
    """||A - sum_k A_k kron B_k||_F == ||P_bar - sum_k sigma_k u_k v_k^T||_F (Theorem 1)."""
    g = W.rng(13 + r)
    P = W.random_psf(g, 5, 5)
    m, n = 9, 8
    A = kron.explicit_blur_matrix(P, 2, 2, m, n, bc)
    ka = kron.kron_approx(P, 2, 2, m, n, bc, r)
    err = np.linalg.norm(A - kron.explicit_kron_matrix(ka))
    assert abs(err - ka.approx_err) <= 1e-12 * max(1.0, err)


@pytest.mark.parametrize("bc", [0, 1])
def test_theorem1_catches_literal_factor_orientation(bc):
    """Planted mistake: the paper's literal (K from u, H from v) assignment breaks Theorem 1."""
    g = W.rng(17)
    P = W.random_psf(g, 5, 5)
    A = kron.explicit_blur_matrix(P, 2, 2, 8, 8, bc)
    ka = kron.kron_approx(P, 2, 2, 8, 8, bc, 2, swap_orientation=True)
    err = np.linalg.norm(A - kron.explicit_kron_matrix(ka))
    assert err > 1.5 * ka.approx_err


@pytest.mark.parametrize("bc", [0, 1])
def test_full_rank_decomposition_is_exact(bc):
    """Eq. (kron1): keeping all min(p, q) terms reproduces A exactly."""
    g = W.rng(18)
    P = W.random_psf(g, 4, 5)
    A = kron.explicit_blur_matrix(P, 1, 2, 7, 9, bc)
    ka = kron.kron_approx(P, 1, 2, 7, 9, bc, 4)
    assert np.linalg.norm(A - kron.explicit_kron_matrix(ka)) < 1e-13
    assert ka.approx_err < 1e-13


@pytest.mark.parametrize("bc", [0, 1])
def test_separable_psf_rank_one_is_exact(bc):
    """A separable PSF (Gaussian) needs one term: A_1 = A, to rounding."""
    P = W.gaussian_psf(9, 2.0)
    ka = kron.kron_approx(P, 4, 4, 24, 20, bc, 1)
    assert ka.approx_err < 1e-15
    g = W.rng(19)
    X = g.uniform(size=(24, 20))
    np.testing.assert_allclose(oracle.kron_apply(X, ka), oracle.blur(X, P, 4, 4, bc), atol=1e-15)


# ------------------------------------------------------------------ operator
@pytest.mark.parametrize("bc", [0, 1])
def test_kron_apply_matches_explicit_kron(bc):
    """sum_k B_k X A_k^T == (sum_k A_k kron B_k) vec(X) with column-stacked vec (Eq. matrix equation)."""
    g = W.rng(20)
    P = W.random_psf(g, 5, 3)
    ka = kron.kron_approx(P, 2, 1, 8, 7, bc, 3)
    As = kron.explicit_kron_matrix(ka)
    X = g.standard_normal((8, 7))
    np.testing.assert_allclose(oracle.kron_apply(X, ka).flatten(order="F"),
                               As @ X.flatten(order="F"), atol=1e-14)
    np.testing.assert_allclose(oracle.kron_apply_T(X, ka).flatten(order="F"),
                               As.T @ X.flatten(order="F"), atol=1e-14)


@pytest.mark.parametrize("bc", [0, 1])
def test_adjoint_identity(bc):
    """<A_s X, Y> == <X, A_s^T Y> (Theorem 3's transpose property) at a moderate size."""
    g = W.rng(21)
    P = W.rotated_gaussian_psf(15, 3.0, 1.0, 0.5)
    ka = kron.kron_approx(P, 7, 7, 96, 80, bc, 3)
    X = g.standard_normal((96, 80))
    Y = g.standard_normal((96, 80))
    lhs = np.vdot(oracle.kron_apply(X, ka), Y)
    rhs = np.vdot(X, oracle.kron_apply_T(Y, ka))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ------------------------------------------------------------------ Alg. 2 / theorems
def _tiny_problem(bc=1, r=2, m=8, n=7, seed=22):
    g = W.rng(seed)
    P = W.random_psf(g, 5, 5)
    ka = kron.kron_approx(P, 2, 2, m, n, bc, r)
    x = g.uniform(size=(m, n))
    Bd = oracle.blur(x, P, 2, 2, bc) + 0.01 * g.standard_normal((m, n))
    As = kron.explicit_kron_matrix(ka)
    L = float(np.linalg.eigvalsh(As.T @ As).max())
    return ka, Bd, As, L


def test_lipschitz_power_iteration_matches_eig():
    ka, Bd, As, L = _tiny_problem()
    Lp, _ = oracle.lipschitz(ka, W.rng(1).uniform(size=Bd.shape), tol=1e-15, maxit=20000)
    assert abs(Lp - L) <= 1e-10 * L


@pytest.mark.parametrize("bc", [0, 1])
def test_theorem3_sfista_equals_vector_fista(bc):
    """Theorem 3: sFISTA on the matrix model == FISTA (Alg. 1) on A_s, iterate for iterate."""
    ka, Bd, As, L = _tiny_problem(bc=bc)
    for iters in (1, 2, 7, 40):
        X = oracle.sfista(Bd, ka, L, 0.05, iters)
        x = oracle.fista_dense(As, Bd.flatten(order="F"), L, 0.05, iters)
        np.testing.assert_allclose(X.flatten(order="F"), x, atol=1e-13)


def _tikhonov_minimiser(As, Bd, lam):
    N = As.shape[1]
    x = np.linalg.solve(As.T @ As + lam * lam * np.eye(N), As.T @ Bd.flatten(order="F"))
    return x.reshape(Bd.shape, order="F")


def test_theorem2_rate_bound():
    """Theorem 2: Phi_s(X_k) - Phi_s* <= 2 L ||X_0 - X*||^2 / (k+1)^2 for every k."""
    ka, Bd, As, L = _tiny_problem(seed=23)
    lam = 0.02
    Xs = _tikhonov_minimiser(As, Bd, lam)
    Fs = oracle.objective(Xs, Bd, ka, lam)
    c = 2.0 * L * np.sum(Xs * Xs)
    for k in range(1, 60):
        Fk = oracle.objective(oracle.sfista(Bd, ka, L, lam, k), Bd, ka, lam)
        assert Fk - Fs <= c / (k + 1) ** 2 + 1e-14


@pytest.mark.parametrize("bc", [0, 1])
def test_objective_matches_explicit_formula(bc):
    """Phi_s(X) = 1/2 ||A_s vec X - vec B||^2 + 1/2 lam^2 ||X||^2 (Eq. matrix minimization model),
    with A_s the explicit sum of Kronecker products acting on the column-stacked vec."""
    ka, Bd, As, _ = _tiny_problem(bc=bc, seed=27)
    g = W.rng(28)
    for lam in (0.0, 0.07, 0.6):
        X = g.standard_normal(Bd.shape)
        e = As @ X.flatten(order="F") - Bd.flatten(order="F")
        want = 0.5 * float(e @ e) + 0.5 * lam * lam * float(np.sum(X * X))
        assert abs(oracle.objective(X, Bd, ka, lam) - want) <= 1e-13 * want


def test_objective_at_and_around_the_minimiser():
    """At X* = (A_s^T A_s + lam^2 I)^{-1} A_s^T b:  Phi_s(X*) = 1/2 <B - A_s X*, B>, and for any D,
    Phi_s(X* + D) - Phi_s(X*) = 1/2 ||A_s D||^2 + 1/2 lam^2 ||D||^2 (the quadratic's expansion about its
    minimiser).  A dropped 1/2, lam in place of lam^2 or a sign error breaks one of the two."""
    ka, Bd, As, _ = _tiny_problem(seed=29)
    g = W.rng(30)
    for lam in (0.05, 0.4):
        Xs = _tikhonov_minimiser(As, Bd, lam)
        Fs = oracle.objective(Xs, Bd, ka, lam)
        r = Bd.flatten(order="F") - As @ Xs.flatten(order="F")
        assert abs(Fs - 0.5 * float(r @ Bd.flatten(order="F"))) <= 1e-12 * Fs
        for _ in range(3):
            D = g.standard_normal(Bd.shape)
            AD = As @ D.flatten(order="F")
            want = 0.5 * float(AD @ AD) + 0.5 * lam * lam * float(np.sum(D * D))
            got = oracle.objective(Xs + D, Bd, ka, lam) - Fs
            assert abs(got - want) <= 1e-11 * want


def test_converges_to_closed_form_tikhonov():
    """With enough iterations X_k -> X* = (A_s^T A_s + lam^2 I)^{-1} A_s^T b, and X* is a fixed point of Step 1."""
    ka, Bd, As, L = _tiny_problem(seed=24)
    lam = 0.3
    Xs = _tikhonov_minimiser(As, Bd, lam)
    X = oracle.sfista(Bd, ka, L, lam, 3000)
    assert oracle.rel_fro(X, Xs) < 1e-10
    G = oracle.kron_apply_T(oracle.kron_apply(Xs, ka) - Bd, ka)
    step = (L * Xs - G) / (L + lam * lam)
    np.testing.assert_allclose(step, Xs, atol=1e-13)


def test_rank_one_closed_form_at_moderate_size():
    """r = 1, any n: X* = V_H[(V_H^T B^T Bd A V_K) ./ (mu nu^T + lam^2)] V_K^T; sFISTA reaches it."""
    g = W.rng(25)
    n = 64
    P = W.gaussian_psf(9, 1.5)
    ka = kron.kron_approx(P, 4, 4, n, n, 1, 1)
    Bf, Af = kron.dense_factors(ka)
    B, A = Bf[0], Af[0]
    x = W.rectangles_image(g, n, n)
    Bd = oracle.blur(x, P, 4, 4, 1) + 0.01 * g.standard_normal((n, n))
    lam = 0.4
    mu, VH = np.linalg.eigh(B.T @ B)
    nu, VK = np.linalg.eigh(A.T @ A)
    Xs = VH @ ((VH.T @ B.T @ Bd @ A @ VK) / (np.outer(mu, nu) + lam * lam)) @ VK.T
    L = float(mu.max() * nu.max())
    X = oracle.sfista(Bd, ka, L, lam, 400)
    assert oracle.rel_fro(X, Xs) < 1e-10


def test_prox_form_equals_gradient_form():
    """Step 1's prox form equals a gradient step of size 1/(L + lam^2) on Phi_s (Sec. 3.2 derivation)."""
    ka, Bd, As, L = _tiny_problem(seed=26)
    lam = 0.1
    Y = W.rng(3).uniform(size=Bd.shape)
    G = oracle.kron_apply_T(oracle.kron_apply(Y, ka) - Bd, ka)
    prox = (L * Y - G) / (L + lam * lam)
    grad = Y - (G + lam * lam * Y) / (L + lam * lam)
    np.testing.assert_allclose(prox, grad, atol=1e-15)
    X1 = oracle.sfista(Bd, ka, L, lam, 1, X_start=Y, Xprev_start=Y)
    np.testing.assert_allclose(X1, prox, atol=1e-15)


def test_t_schedule_identities():
    """t_{k+1}^2 - t_{k+1} = t_k^2 and t_k >= (k+1)/2 (Beck-Teboulle sequence of Step 2)."""
    t = oracle.t_schedule(500)
    assert t[0] == 1.0
    np.testing.assert_allclose(t[1:] ** 2 - t[1:], t[:-1] ** 2, rtol=1e-13)
    assert np.all(t >= (np.arange(1, 502) + 1) / 2.0 - 1e-12)


def test_resume_matches_uninterrupted_run():
    """State (X_k, X_{k-1}, k) is all Alg. 2 carries: resuming reproduces the uninterrupted run."""
    ka, Bd, As, L = _tiny_problem(seed=27)
    X30 = oracle.sfista(Bd, ka, L, 0.05, 30)
    X20, X19 = oracle.sfista(Bd, ka, L, 0.05, 20, return_prev=True)
    Xr = oracle.sfista(Bd, ka, L, 0.05, 10, k0=20, X_start=X20, Xprev_start=X19)
    np.testing.assert_allclose(Xr, X30, atol=1e-14)


def test_projection_is_nonnegative_prox():
    """max(0, .) after the shrink: the iterates stay non-negative and match the clipped step."""
    ka, Bd, As, L = _tiny_problem(seed=28)
    X = oracle.sfista(Bd - 0.2, ka, L, 0.05, 25, project=True)
    assert X.min() >= 0.0
    Y = np.abs(W.rng(4).standard_normal(Bd.shape))
    G = oracle.kron_apply_T(oracle.kron_apply(Y, ka) - Bd, ka)
    X1 = oracle.sfista(Bd, ka, L, 0.05, 1, project=True, X_start=Y, Xprev_start=Y)
    np.testing.assert_allclose(X1, np.maximum((L * Y - G) / (L + 0.0025), 0.0), atol=1e-15)


def test_theorem4_error_falls_with_rank():
    """Theorem 4 / Tables 1-4 trend: the Kronecker error eps_s and the restoration error fall as r grows."""
    g = W.rng(29)
    n = 48
    P = W.rotated_gaussian_psf(11, 2.5, 0.8, np.deg2rad(35))
    x = W.shapes_image(g, n, n, rects=4, ellipses=4)
    Bd = oracle.blur(x, P, 5, 5, 1)
    errs, etas = [], []
    for r in (1, 2, 3, 5, 11):
        ka = kron.kron_approx(P, 5, 5, n, n, 1, r)
        L, _ = oracle.lipschitz(ka, np.ones((n, n)), tol=1e-10, maxit=3000)
        X = oracle.sfista(Bd, ka, L, 0.01, 100)
        errs.append(ka.approx_err)
        etas.append(oracle.rel_fro(X, x))
    assert all(a >= b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-13
    assert etas[-1] <= etas[0]
    assert all(b <= a * 1.02 for a, b in zip(etas, etas[1:]))


# ------------------------------------------------------------------ l1 variant of Step 1
def _soft(v, mu):
    return np.sign(v) * np.maximum(np.abs(v) - mu, 0.0)


def test_l1_step_with_identity_operator_is_closed_form():
    """A 1x1 unit PSF gives A_s = I; with L = 1 the first step from Y_1 = 0 is already the
    minimiser of 1/2||X - B||^2 + lam^2/2 ||X||^2 + mu ||X||_1: S_mu(B) / (1 + lam^2)."""
    g = W.rng(31)
    B = g.standard_normal((13, 11))
    ka = kron.kron_approx(np.ones((1, 1)), 0, 0, 13, 11, 0, 1)
    lam, mu = 0.3, 0.45
    X1 = oracle.sfista(B, ka, 1.0, lam, 1, mu=mu)
    np.testing.assert_allclose(X1, _soft(B, mu) / (1.0 + lam * lam), atol=1e-15)
    assert np.count_nonzero(X1 == 0.0) > 0      # the threshold does set entries to zero
    X40 = oracle.sfista(B, ka, 1.0, lam, 40, mu=mu)    # and it is a fixed point
    np.testing.assert_allclose(X40, X1, atol=1e-14)


def test_l1_limit_satisfies_optimality_conditions():
    """At the limit X* of Step 1 with the l1 term: for X*_j != 0,
    (grad f + lam^2 X*)_j = -mu sign(X*_j); for X*_j = 0, |(grad f + lam^2 X*)_j| <= mu."""
    ka, Bd, As, L = _tiny_problem(seed=32)
    lam, mu = 0.1, 0.2
    X = oracle.sfista(Bd, ka, L, lam, 6000, mu=mu)
    G = oracle.kron_apply_T(oracle.kron_apply(X, ka) - Bd, ka) + lam * lam * X
    nz = X != 0.0
    assert 0 < nz.sum() < X.size                # both cases occur
    np.testing.assert_allclose(G[nz], -mu * np.sign(X[nz]), atol=1e-9)
    assert np.abs(G[~nz]).max() <= mu + 1e-9


def test_l1_sfista_equals_vector_fista():
    """Theorem 3 carries over: the element-wise threshold commutes with vec."""
    ka, Bd, As, L = _tiny_problem(seed=33)
    for iters in (1, 5, 30):
        X = oracle.sfista(Bd, ka, L, 0.05, iters, mu=0.01)
        x = oracle.fista_dense(As, Bd.flatten(order="F"), L, 0.05, iters, mu=0.01)
        np.testing.assert_allclose(X.flatten(order="F"), x, atol=1e-13)


# ------------------------------------------------------------------ Alg. 1 on the exact blur
@pytest.mark.parametrize("bc", [0, 1])
def test_fista_exact_equals_alg1_on_explicit_blur_matrix(bc):
    """Alg. 1 with A applied by the exact blur == Alg. 1 on the explicit N x N matrix whose columns are
    point-source images (Sec. 2), iterate for iterate; non-symmetric, non-centred PSF."""
    g = W.rng(40)
    P = W.random_psf(g, 5, 4)
    m, n = 9, 8
    A = kron.explicit_blur_matrix(P, 1, 3, m, n, bc)
    x = g.uniform(size=(m, n))
    Bd = oracle.blur(x, P, 1, 3, bc) + 0.01 * g.standard_normal((m, n))
    L = float(np.linalg.eigvalsh(A.T @ A).max())
    for iters in (1, 3, 25):
        X = oracle.fista_exact(Bd, P, 1, 3, bc, L, 0.05, iters)
        xd = oracle.fista_dense(A, Bd.flatten(order="F"), L, 0.05, iters)
        np.testing.assert_allclose(X.flatten(order="F"), xd, atol=1e-13)


@pytest.mark.parametrize("bc", [0, 1])
def test_lipschitz_exact_matches_eig(bc):
    g = W.rng(41)
    P = W.random_psf(g, 5, 5)
    A = kron.explicit_blur_matrix(P, 2, 2, 10, 9, bc)
    L = float(np.linalg.eigvalsh(A.T @ A).max())
    Lp, _ = oracle.lipschitz_exact(P, 2, 2, bc, W.rng(1).uniform(size=(10, 9)), tol=1e-15, maxit=20000)
    assert abs(Lp - L) <= 1e-10 * L


def test_fista_exact_is_sfista_for_a_separable_psf():
    """A separable PSF is its own rank-1 Kronecker approximation (Theorem 1 with sigma_2 = 0), so Alg. 1 on
    the exact blur and Alg. 2 with r = 1 produce the same iterates."""
    g = W.rng(42)
    P = W.gaussian_psf(9, 1.7)
    x = W.rectangles_image(g, 48, 40)
    for bc in (0, 1):
        Bd = oracle.blur(x, P, 4, 4, bc) + 0.01 * g.standard_normal(x.shape)
        ka = kron.kron_approx(P, 4, 4, 48, 40, bc, 1)
        assert ka.approx_err < 1e-12
        X1 = oracle.fista_exact(Bd, P, 4, 4, bc, 1.0, 0.02, 30)
        X2 = oracle.sfista(Bd, ka, 1.0, 0.02, 30)
        np.testing.assert_allclose(X1, X2, atol=1e-12)
