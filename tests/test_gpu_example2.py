"""The Example 2 stand-in set (defocus and shake blur at three levels, three
noise kinds) through the library vs the FP64 oracle, and the library's P_bar
singular values vs the oracle's (needs a GB300)."""
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


@pytest.mark.parametrize("case", range(18))
def test_example2_case_matches_oracle(case):
    pr = W.example2_cases(n=64)[case]
    n = 64
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_of_kind(pr.extra["noise"], bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
    L, _ = oracle.lipschitz(ka, np.ones((n, n)), tol=1e-10, maxit=2000)
    iters = 20
    Xo = oracle.sfista(b.astype(np.float64), ka, L, pr.lam, iters)
    s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="fp32", lipschitz=L)
    X = s.solve_device(torch.from_numpy(b).cuda(), pr.lam, iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-5
    k = min(pr.psf.shape)
    sig = s.info()["sigma"][:k]
    np.testing.assert_allclose(sig, ka.sigma[:k], rtol=1e-10, atol=1e-14 * ka.sigma[0])
    s.close()
