"""C-ABI library: loads, exports what include/sfista.h declares, host setup
matches the oracle, argument errors come back as status codes (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from oracle import kron
from paper_1901_00913_gb300 import api, build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sfista_\w+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("case", [((15, 15), (7, 7), (64, 60), 3),
                                  ((9, 13), (2, 9), (40, 33), 4),
                                  ((31, 31), (15, 15), (128, 128), 5)])
def test_factorize_matches_oracle(lib, bc, case):
    """The library's own FP64 Jacobi SVD / Cholesky / Gram setup == the oracle's (Theorem 1)."""
    (p, q), (cr, cc), (m, n), r = case
    g = W.rng(p * 100 + q + bc)
    P = W.rotated_gaussian_psf(max(p, q), 3.0, 1.2, 0.6)[:p, :q] + 0.05 * g.uniform(size=(p, q))
    sig, C, D, err = api.sfista_factorize(P, m, n, bc, r, center=(cr, cc))
    ka = kron.kron_approx(P, cr, cc, m, n, bc, r)
    np.testing.assert_allclose(sig, ka.sigma, rtol=0, atol=1e-13 * ka.sigma[0])
    assert abs(err - ka.approx_err) <= 1e-12 * ka.sigma[0]
    for k in range(r):
        np.testing.assert_allclose(np.outer(C[k], D[k]), np.outer(ka.C[k], ka.D[k]), rtol=0,
                                   atol=1e-12 * np.abs(np.outer(ka.C[0], ka.D[0])).max())


def test_factorize_sign_rule(lib):
    """Largest-|u| entry positive: with distinct singular values the profiles themselves agree."""
    P = W.rotated_gaussian_psf(15, 3.0, 1.0, np.deg2rad(30))
    sig, C, D, err = api.sfista_factorize(P, 64, 64, 1, 3)
    ka = kron.kron_approx(P, 7, 7, 64, 64, 1, 3)
    np.testing.assert_allclose(C, ka.C, atol=1e-12)
    np.testing.assert_allclose(D, ka.D, atol=1e-12)


@pytest.mark.parametrize("args,status", [
    (dict(m=10, n=10, bc=1, r=3), api.EINVAL),        # PSF larger than the image
    (dict(m=64, n=64, bc=2, r=3), api.ENOTSUP),       # periodic boundary
    (dict(m=64, n=64, bc=7, r=3), api.EINVAL),        # unknown boundary
    (dict(m=64, n=64, bc=1, r=0), api.EINVAL),        # rank too small
    (dict(m=64, n=64, bc=1, r=16), api.EINVAL),       # rank > min(p, q)
    (dict(m=64, n=64, bc=1, r=3, center=(15, 0)), api.EINVAL),   # centre outside
])
def test_argument_errors(lib, args, status):
    P = W.gaussian_psf(15, 2.0)
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_factorize(P, args["m"], args["n"], args["bc"], args["r"], center=args.get("center", (-1, -1)))
    assert ei.value.status == status
    o = api.default_opts()
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_setup(P, args["m"], args["n"], args["bc"], args["r"], args.get("center", (-1, -1)), o)
    assert ei.value.status == status


def test_nonfinite_psf_rejected(lib):
    P = W.gaussian_psf(9, 2.0)
    P[3, 4] = np.nan
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_factorize(P, 32, 32, 0, 1)
    assert ei.value.status == api.EINVAL


def test_tied_singular_values_rejected(lib):
    """A PSF whose weighted singular values tie at the truncation point has no unique rank-r sum."""
    P = np.zeros((5, 5))
    P[1, 1] = P[3, 3] = 1.0       # two equal separable bumps -> sigma_1 == sigma_2 (zero BC weights equal)
    P[1, 3] = P[3, 1] = 0.0
    sig, C, D, err = api.sfista_factorize(P, 32, 32, 0, 2, center=(2, 2))
    assert err < 1e-14
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_factorize(P, 32, 32, 0, 1, center=(2, 2))
    assert ei.value.status == api.EINVAL


def test_default_opts(lib):
    o = api.default_opts()
    assert o.prec == 0 and o.op == 0 and o.use_graph == 1 and o.device == -1
    assert o.lipschitz == 0.0 and o.lipschitz_maxit > 0
    assert o.l1 == 0.0 and o.refine_every == 0
    assert o.tile_override == 0 and o.gemm_bn == 0 and o.gemm_resident_panels == 0


@pytest.mark.parametrize("field,value", [("refine_every", -1), ("l1", -0.5), ("prec", 9), ("tile_override", 30),
                                         ("gemm_bn", 192), ("gemm_bn", 32), ("gemm_resident_panels", 2)])
def test_option_errors(lib, field, value):
    o = api.default_opts()
    setattr(o, field, value)
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_setup(W.gaussian_psf(9, 2.0), 64, 64, 1, 2, (-1, -1), o)
    assert ei.value.status == api.EINVAL


def _dense_from_band(band, lo):
    """F_k[c][c + lo + t] = band[k, t, c] (entries outside the axis are 0 by contract)."""
    r, w, length = band.shape
    F = np.zeros((r, length, length))
    for k in range(r):
        for t in range(w):
            for c in range(length):
                j = c + lo + t
                if 0 <= j < length:
                    F[k, c, j] = band[k, t, c]
                else:
                    assert band[k, t, c] == 0.0
    return F


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("psf_shape,centre,shape,r", [((9, 7), (4, 3), (40, 36), 2), ((6, 11), (0, 10), (33, 50), 3),
                                                      ((15, 15), (7, 7), (64, 64), 4)])
def test_factor_bands_are_the_oracle_factors(lib, bc, psf_shape, centre, shape, r):
    """The band tables the kernels read hold the factors T + H of Sec. 2 /
    Theorem 1 (A_k acting on columns, B_k on rows, and their transposes),
    as the oracle builds them densely."""
    g = W.rng(900 + psf_shape[0] * 7 + psf_shape[1] + bc)
    P = W.random_psf(g, *psf_shape)
    m, n = shape
    ka = kron.kron_approx(P, centre[0], centre[1], m, n, bc, r)
    Bo, Ao = kron.dense_factors(ka)
    ref = {0: Ao, 1: np.transpose(Ao, (0, 2, 1)), 2: Bo, 3: np.transpose(Bo, (0, 2, 1))}
    for which in range(4):
        band, lo, _ = api.sfista_factor_bands(P, m, n, bc, r, which, center=centre)
        F = _dense_from_band(band, lo)
        scale = np.abs(ref[which]).max()
        np.testing.assert_allclose(F, ref[which], rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("psf_shape,centre,shape", [((9, 9), (4, 4), (64, 72)), ((7, 12), (1, 9), (64, 72)),
                                                    ((13, 5), (12, 0), (64, 72)), ((9, 9), (4, 4), (12, 9)),
                                                    ((5, 7), (2, 6), (8, 16))])
def test_factor_band_interior_rows(lib, bc, psf_shape, centre, shape):
    """Interior rows: every row in [i0, i1) holds the middle row's FP32 values
    bit for bit, the run is maximal, and it covers every row whose taps all
    land inside the axis (no boundary term), where the factor is Toeplitz.
    Small images, where few or no rows are free of the boundary, included."""
    g = W.rng(950 + psf_shape[0] + 3 * psf_shape[1] + bc)
    P = W.random_psf(g, *psf_shape)
    (m, n), r = shape, 2
    for which in range(4):
        band, lo, (i0, i1) = api.sfista_factor_bands(P, m, n, bc, r, which, center=centre)
        f = band.astype(np.float32).reshape(-1, band.shape[-1])   # (r * w) x len
        length = f.shape[1]
        mid = length // 2
        assert i0 <= mid < i1
        for row in range(i0, i1):
            assert np.array_equal(f[:, row].view(np.uint32), f[:, mid].view(np.uint32))
        for row in (i0 - 1, i1):
            if 0 <= row < length:
                assert not np.array_equal(f[:, row].view(np.uint32), f[:, mid].view(np.uint32))
        p = psf_shape[1] if which < 2 else psf_shape[0]
        c = centre[1] if which < 2 else centre[0]
        # Rows free of the boundary.  Row a of F_k takes taps a - t + c,
        # t < p: all inside the axis for a in [p-1-c, len-1-c].  Row e of
        # F_k^T gathers rows a = e + t - c of F_k (all must exist: e in
        # [c, len-p+c]) and, with reflection, taps of rows near the ends that
        # reflect onto e (none for e in [p-1-c, len-1-c]).
        if which % 2 == 0:
            first, last = p - 1 - c, length - 1 - c
        else:
            first, last = max(c, p - 1 - c), min(length - p + c, length - 1 - c)
        if first <= mid <= last:   # the middle row is free of the boundary: so is the whole free run
            assert i0 <= first and i1 >= last + 1, (which, i0, i1, first, last)


def test_factor_bands_argument_errors(lib):
    P = W.gaussian_psf(9, 2.0)
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_factor_bands(P, 32, 32, 1, 2, 4)
    assert ei.value.status == api.EINVAL
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_factor_bands(P, 32, 32, 2, 2, 0)
    assert ei.value.status == api.ENOTSUP
