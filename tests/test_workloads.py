"""The seeded workload generators: PSF families, noise kinds and the
Example 2 stand-in set (checked against their definitions, on the CPU)."""
import numpy as np
import pytest

from paper_1901_00913_gb300 import diagnostics as D, workloads as W


@pytest.mark.parametrize("p,R", [(7, 2.0), (11, 4.0), (17, 7.0)])
def test_defocus_psf_is_normalised_disk(p, R):
    P = W.defocus_psf(p, R)
    assert abs(P.sum() - 1.0) < 1e-14
    h = (p - 1) / 2
    y, x = np.mgrid[0:p, 0:p] - h
    inside = x * x + y * y <= R * R
    np.testing.assert_allclose(P[inside], 1.0 / inside.sum())
    assert np.all(P[~inside] == 0.0)
    np.testing.assert_array_equal(P, P.T)


def test_shake_psf_is_a_normalised_seeded_walk():
    P1 = W.shake_psf(W.rng(7), 15, 30)
    P2 = W.shake_psf(W.rng(7), 15, 30)
    np.testing.assert_array_equal(P1, P2)
    assert P1.min() >= 0.0 and abs(P1.sum() - 1.0) < 1e-14
    sv = D.psf_singular_values(P1)
    assert sv[1] / sv[0] > 1e-3          # not separable


def test_laplace_draw_has_unit_variance_and_laplace_tails():
    d = W.laplace_noise_draw(W.rng(8), 1000, 1000)
    assert abs(d.mean()) < 5e-3 and abs(d.var() - 1.0) < 1e-2
    kurt = np.mean(d ** 4) / np.mean(d ** 2) ** 2 - 3.0
    assert abs(kurt - 3.0) < 0.15         # Laplace excess kurtosis is 3 (Gaussian: 0)


@pytest.mark.parametrize("kind", ["gauss", "laplace", "multiplicative"])
def test_noise_kinds_have_the_requested_level(kind):
    g = W.rng(9)
    bx = np.zeros((40, 50))
    bx[5:30, 10:45] = g.uniform(0.1, 1.0, size=(25, 35))
    draw = W.laplace_noise_draw(g, 40, 50) if kind == "laplace" else W.noise_draw(g, 40, 50)
    e = W.noise_of_kind(kind, bx, draw, 0.02)
    assert abs(np.linalg.norm(e) / np.linalg.norm(bx) - 0.02) < 1e-14
    if kind == "multiplicative":
        assert np.all(e[bx == 0.0] == 0.0)
        on = bx != 0.0
        c = e[on] / (bx[on] * draw[on])            # one positive constant: e = c * bx * draw
        assert c.min() > 0.0 and np.ptp(c) <= 1e-12 * c.max()
    else:
        c = e / draw                               # e = c * draw
        assert c.min() > 0.0 and np.ptp(c) <= 1e-12 * c.max()


def test_example2_cases():
    cs = W.example2_cases(n=48)
    assert len(cs) == 18 and len({c.name for c in cs}) == 18
    assert {c.extra["noise"] for c in cs} == set(W.EX2_NOISES)
    assert {(c.extra["family"], c.extra["level"]) for c in cs} == {(f, l) for f in ("defocus", "shake")
                                                                   for l in W.EX2_LEVELS}
    for c in cs:
        assert c.x_true.shape == (48, 48) and 0.0 <= c.x_true.min() and c.x_true.max() <= 1.0
        assert c.psf.shape[0] % 2 == 1 and abs(c.psf.sum() - 1.0) < 1e-12
        assert c.r == min(5, *c.psf.shape) and c.iters == 50 and c.bc == 1


def test_decay_ratios():
    sep = W.gaussian_psf(9, 1.5)                 # separable: rank one
    r = D.decay_ratios(D.psf_singular_values(sep))
    assert r[2] < 1e-12
    disk = D.decay_ratios(D.psf_singular_values(W.defocus_psf(17, 7.0)))
    assert 1.0 > disk[2] > disk[6] > 0.0
