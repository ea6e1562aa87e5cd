"""The FFT form of the operator (SFISTA_OP_FFT) and the exact-blur context of
Alg. 1 (sfista_setup_exact) against the FP64 oracle, through the C ABI.

The FFT form applies sum_i B_i X A_i^T as one 2-D convolution of the
boundary-extended image with the rank-r kernel sum_i c_i d_i^T; the exact
context applies the blur of Eq. (1.1) with the PSF itself.  Both are FP32:
operator results are held to 2e-6 relative Frobenius error (a few FP32
rounding steps through transforms of length <= 8192), solves to the FP32
path's 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import kron
from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape,psf,centre,r", [((200, 176), (13, 11), (4, 7), 3), ((64, 64), (9, 9), (4, 4), 1),
                                                ((37, 45), (13, 11), (12, 0), 2), ((96, 100), (41, 9), (20, 4), 4),
                                                ((1, 40), (1, 7), (0, 3), 1)])
def test_fft_apply_matches_oracle(bc, shape, psf, centre, r):
    """A_s X and A_s^T X by the FFT form on ragged sizes, non-square and non-centred PSFs."""
    m, n = shape
    g = W.rng(300 + m + n + bc)
    P = W.random_psf(g, *psf)
    ka = kron.kron_approx(P, centre[0], centre[1], m, n, bc, r)
    s = api.Sfista(P, (m, n), bc, r, center=centre, prec="fp32", op="fft", lipschitz=1.0)
    assert s.info()["op"] == "fft"
    X = g.standard_normal((m, n)).astype(np.float32)
    for tr in (False, True):
        Y = s.apply(_cuda(X), transpose=tr).cpu().numpy()
        Yo = (oracle.kron_apply_T if tr else oracle.kron_apply)(X.astype(np.float64), ka)
        assert oracle.rel_fro(Y, Yo) < OP_TOL, (tr, oracle.rel_fro(Y, Yo))
    s.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_fft_apply_wide_psf(bc):
    """256^2 image, 63 x 63 PSF (wider than n/8, where the FFT form is meant to win), r = 4."""
    n = 256
    g = W.rng(310 + bc)
    P = W.mixture_moffat_psf(g, 63)
    ka = kron.kron_approx(P, 31, 31, n, n, bc, 4)
    s = api.Sfista(P, (n, n), bc, 4, prec="fp32", op="fft", lipschitz=1.0)
    X = W.shapes_image(g, n, n).astype(np.float32)
    for tr in (False, True):
        Y = s.apply(_cuda(X), transpose=tr).cpu().numpy()
        Yo = (oracle.kron_apply_T if tr else oracle.kron_apply)(X.astype(np.float64), ka)
        assert oracle.rel_fro(Y, Yo) < OP_TOL
    s.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_fft_apply_long_lines(bc):
    """2100 x 2104 image with a 31 x 27 PSF: both extended axes (2130) take 2160-point lines, whose
    plan has the in-register radix-16 and radix-9 stages (16, 9, 3, 5); A_s X and A_s^T X against the
    oracle."""
    m, n = 2100, 2104
    g = W.rng(320 + bc)
    P = W.random_psf(g, 31, 27)
    ka = kron.kron_approx(P, 15, 13, m, n, bc, 2)
    s = api.Sfista(P, (m, n), bc, 2, center=(15, 13), prec="fp32", op="fft", lipschitz=1.0)
    X = g.standard_normal((m, n)).astype(np.float32)
    for tr in (False, True):
        Y = s.apply(_cuda(X), transpose=tr).cpu().numpy()
        Yo = (oracle.kron_apply_T if tr else oracle.kron_apply)(X.astype(np.float64), ka)
        assert oracle.rel_fro(Y, Yo) < OP_TOL, (tr, oracle.rel_fro(Y, Yo))
    s.close()


def _observation(x, P, cr, cc, bc, g, level=0.01):
    bx = oracle.blur(x, P, cr, cc, bc)
    return (bx + W.noise_scale(bx, g.standard_normal(x.shape), level)).astype(np.float32)


def test_fft_solve_config2_matches_oracle():
    """The 512^2 workload (31 x 31 rotated Gaussian, reflective, r = 3, 200 iterations) in the FFT form."""
    pr = W.config2()
    cr, cc = pr.centre
    n = 512
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
    L, _ = oracle.lipschitz(ka, np.ones((n, n)), tol=1e-9, maxit=300)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, pr.lam, pr.iters)
    s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="fp32", op="fft", lipschitz=L)
    X = s.solve_device(_cuda(b), pr.lam, pr.iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-5
    s.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_fft_solve_ragged_with_options(bc):
    """Ragged 120 x 98 image, non-centred PSF, projection and the l1 term, 60 iterations."""
    m, n = 120, 98
    g = W.rng(320 + bc)
    P = W.random_psf(g, 11, 9)
    x = W.shapes_image(g, m, n, rects=5, ellipses=5)
    b = _observation(x, P, 3, 5, bc, g)
    ka = kron.kron_approx(P, 3, 5, m, n, bc, 3)
    L, _ = oracle.lipschitz(ka, np.ones((m, n)), tol=1e-10, maxit=500)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.01, 60, project=True, mu=1e-4)
    s = api.Sfista(P, (m, n), bc, 3, center=(3, 5), prec="fp32", op="fft", lipschitz=L, project=True, l1=1e-4)
    X = s.solve_device(_cuda(b), 0.01, 60).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-5
    s.close()


# ------------------------------------------------------------------ exact blur (Alg. 1)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape,psf,centre", [((200, 176), (13, 11), (4, 7)), ((37, 45), (7, 14), (3, 0)),
                                              ((128, 128), (31, 31), (15, 15))])
def test_exact_apply_matches_oracle_blur(bc, shape, psf, centre):
    """A x and A^T x of Eq. (1.1) (no approximation) against the oracle's exact blur and its transpose."""
    m, n = shape
    g = W.rng(330 + m + bc)
    P = W.random_psf(g, *psf) if psf[0] < 31 else W.rotated_gaussian_psf(31, 3.0, 1.0, np.deg2rad(30))
    s = api.Sfista(P, (m, n), bc, 1, center=centre, exact=True, lipschitz=1.0)
    assert s.info()["op"] == "exact_fft"
    X = g.standard_normal((m, n)).astype(np.float32)
    for tr in (False, True):
        Y = s.apply(_cuda(X), transpose=tr).cpu().numpy()
        Yo = (oracle.blur_T if tr else oracle.blur)(X.astype(np.float64), P, centre[0], centre[1], bc)
        assert oracle.rel_fro(Y, Yo) < OP_TOL, (tr, oracle.rel_fro(Y, Yo))
    s.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_exact_lipschitz_matches_oracle(bc):
    g = W.rng(340 + bc)
    P = W.rotated_gaussian_psf(15, 2.5, 1.0, 0.4)
    s = api.Sfista(P, (96, 80), bc, 1, exact=True)
    Lo, _ = oracle.lipschitz_exact(P, 7, 7, bc, np.ones((96, 80)), tol=1e-12, maxit=3000)
    # FP32 applications: the power iteration stops once its Rayleigh quotient changes by < 2e-7 per
    # step, short of lambda_max where the top eigenvalues cluster (as the paper's Lanczos estimate)
    assert abs(s.info()["lipschitz"] / Lo - 1.0) < 1e-4
    s.close()
    del g


@pytest.mark.parametrize("bc", [0, 1])
def test_exact_solve_matches_oracle_alg1(bc):
    """Alg. 1 on the exact blur: 256^2 shapes image, 31 x 31 rotated Gaussian (non-separable), 100 iterations."""
    n = 256
    g = W.rng(350 + bc)
    P = W.rotated_gaussian_psf(31, 3.0, 1.0, np.deg2rad(30))
    x = W.shapes_image(g, n, n)
    b = _observation(x, P, 15, 15, bc, g)
    L, _ = oracle.lipschitz_exact(P, 15, 15, bc, np.ones((n, n)), tol=1e-9, maxit=300)
    Xo = oracle.fista_exact(b.astype(np.float64), P, 15, 15, bc, L, 0.005, 100)
    s = api.Sfista(P, (n, n), bc, 1, exact=True, lipschitz=L)
    X = s.solve_device(_cuda(b), 0.005, 100).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-5
    s.close()


def test_fft_forms_reject_what_they_do_not_support():
    P = W.gaussian_psf(9, 2.0)
    with pytest.raises(api.SfistaError) as ei:
        api.Sfista(P, (64, 64), 1, 1, prec="bf16x3", op="fft", lipschitz=1.0)
    assert ei.value.status == api.ENOTSUP
    with pytest.raises(api.SfistaError) as ei:          # transforms longer than 8192
        api.Sfista(P, (8192, 64), 1, 1, prec="fp32", op="fft", lipschitz=1.0)
    assert ei.value.status == api.ENOTSUP
    e = api.Sfista(P, (64, 64), 1, 1, exact=True, lipschitz=1.0)
    with pytest.raises(api.SfistaError) as ei:
        e.tune()
    assert ei.value.status == api.ENOTSUP
    with pytest.raises(api.SfistaError) as ei:
        e.factors()
    assert ei.value.status == api.ENOTSUP
    f = api.Sfista(P, (64, 64), 1, 1, prec="fp32", op="fft", lipschitz=1.0)
    with pytest.raises(api.SfistaError) as ei:
        api.Batch([f])
    assert ei.value.status == api.ENOTSUP
    e.close()
    f.close()


def test_tuner_times_the_fft_form():
    """With the operator form left to the library, the tuner also times the FFT form."""
    P = W.mixture_moffat_psf(W.rng(360), 63)
    s = api.Sfista(P, (256, 256), 1, 3, prec="fp32", lipschitz=1.0)
    entries = s.tune(iters=3)
    assert any(e["op"] == "fft" for e in entries)
    X = _cuda(W.rng(361).standard_normal((256, 256)))
    ka = kron.kron_approx(P, 31, 31, 256, 256, 1, 3)
    Y = s.apply(X).cpu().numpy()
    assert oracle.rel_fro(Y, oracle.kron_apply(X.double().cpu().numpy(), ka)) < OP_TOL
    s.close()
