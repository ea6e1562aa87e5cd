"""Degenerate and extreme inputs through the C ABI vs the FP64 oracle (needs a
GB300): lambda = 0, a unit PSF (A_s = I), single-row images, an image larger
than any workload, and the full 64-problem batch in the bench's tuned launch
configuration (checked on sampled problems)."""
import numpy as np
import pytest

import oracle
from oracle import kron
from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("op,prec,tol", [("banded", "fp32", 1e-5), ("banded_fused", "fp32", 1e-5),
                                         ("gemm_band", "bf16x3", 1e-4)])
def test_lambda_zero_is_plain_least_squares(op, prec, tol):
    g = W.rng(601)
    P = W.rotated_gaussian_psf(11, 2.0, 1.0, 0.5)
    x = W.shapes_image(g, 96, 80, rects=5, ellipses=5)
    b = oracle.blur(x, P, 5, 5, 1).astype(np.float32)
    ka = kron.kron_approx(P, 5, 5, 96, 80, 1, 3)
    L, _ = oracle.lipschitz(ka, np.ones((96, 80)), tol=1e-10, maxit=500)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.0, 40)
    s = api.Sfista(P, (96, 80), 1, 3, op=op, prec=prec, lipschitz=L)
    X = s.solve_device(_cuda(b), 0.0, 40).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= tol
    s.close()


@pytest.mark.parametrize("op", ["banded", "banded_fused", "banded_persistent"])
def test_unit_psf_step_is_closed_form(op):
    """A 1 x 1 unit PSF: A_s = I, L = 1, and X_1 = B / (1 + lambda^2), a fixed point."""
    g = W.rng(602)
    B = g.uniform(size=(40, 56)).astype(np.float32)
    s = api.Sfista(np.ones((1, 1)), (40, 56), 0, 1, op=op, lipschitz_tol=1e-14)
    assert abs(s.info()["lipschitz"] - 1.0) < 1e-12
    lam = 0.3
    X1 = s.solve_device(_cuda(B), lam, 1).cpu().numpy()
    np.testing.assert_allclose(X1, B / (1.0 + lam * lam), rtol=1e-6)
    X9 = s.solve_device(_cuda(B), lam, 9).cpu().numpy()
    np.testing.assert_allclose(X9, X1, rtol=1e-6, atol=1e-7)
    s.close()


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("op", ["banded", "banded_fused"])
def test_single_row_image(bc, op):
    """m = 1 with a 1 x 7 horizontal blur (one 32-row tile, 31 rows outside the image)."""
    g = W.rng(603)
    P = g.uniform(0.1, 1.0, size=(1, 7))
    P /= P.sum()
    x = g.uniform(size=(1, 200))
    b = oracle.blur(x, P, 0, 3, bc).astype(np.float32)
    ka = kron.kron_approx(P, 0, 3, 1, 200, bc, 1)
    L, _ = oracle.lipschitz(ka, np.ones((1, 200)), tol=1e-12, maxit=5000)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.02, 30)
    s = api.Sfista(P, (1, 200), bc, 1, op=op, lipschitz=L)
    X = s.solve_device(_cuda(b), 0.02, 30).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-5
    s.close()


def test_image_larger_than_any_workload():
    """4096^2, r = 2, 15 x 15 PSF: the operator and three iterations against the oracle."""
    n = 4096
    g = W.rng(604)
    P = W.rotated_gaussian_psf(15, 3.0, 1.5, 0.7)
    X = g.uniform(size=(n, n)).astype(np.float32)
    ka = kron.kron_approx(P, 7, 7, n, n, 1, 2)
    s = api.Sfista(P, (n, n), 1, 2, op="auto", lipschitz=1.0)
    Y = s.apply(_cuda(X)).cpu().numpy()
    assert oracle.rel_fro(Y, oracle.kron_apply(X.astype(np.float64), ka)) < 1e-6
    X3 = s.solve_device(_cuda(X), 0.01, 3).cpu().numpy()
    assert oracle.rel_fro(X3, oracle.sfista(X.astype(np.float64), ka, 1.0, 0.01, 3)) <= 1e-5
    s.close()
