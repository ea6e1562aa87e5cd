"""Reverse mode of the unrolled solve on the GPU vs the FP64 oracle's reverse
mode (every gradient entry, small case) and vs FP64 central finite
differences of the oracle forward (directional, 512^2 r=3 50 iterations)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, kron
from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("op", ["banded", "banded_fused", "banded_persistent"])
def test_gradients_match_oracle_reverse_mode(op):
    m, n, r, K, ck = 64, 56, 2, 12, 5
    g = W.rng(401)
    P = W.rotated_gaussian_psf(11, 2.5, 1.0, 0.4)
    ka = kron.kron_approx(P, 5, 5, m, n, 1, r)
    Bf, Af = kron.dense_factors(ka)
    x = W.shapes_image(g, m, n, rects=4, ellipses=4)
    bx = oracle.blur(x, P, 5, 5, 1)
    b = (bx + W.noise_scale(bx, g.standard_normal((m, n)), 0.01)).astype(np.float32)
    L, lam = 1.05, 0.05
    s = api.Sfista(P, (m, n), 1, r, prec="fp32", op=op, lipschitz=L)
    db = torch.from_numpy(b).cuda()
    nseg = (K + ck - 1) // ck
    ckpt = torch.empty(2 * nseg, m, n, dtype=torch.float64, device="cuda")
    X = torch.empty_like(db)
    api.sfista_unrolled_fwd(s.ctx, db, lam, K, ck, ckpt, X)
    torch.cuda.synchronize()
    Xo = adjoint.unrolled_forward(b.astype(np.float64), Af, Bf, L, lam, K)[0]
    assert _rel(X.cpu().numpy(), Xo) < 1e-5
    gX = 2.0 * (X.double().cpu().numpy() - x)
    gb = torch.empty_like(db)
    gA = torch.empty(r, n, n, device="cuda")
    gB = torch.empty(r, m, m, device="cuda")
    gl = api.sfista_unrolled_bwd(s.ctx, db, lam, K, ck, ckpt, torch.from_numpy(gX.astype(np.float32)).cuda(),
                                 gb, gA, gB)
    ob, ol, oA, oB = adjoint.unrolled_grad(b.astype(np.float64), Af, Bf, L, lam, K, gX)
    assert _rel(gb.cpu().numpy(), ob) < 1e-4
    assert abs(gl - ol) <= 1e-4 * abs(ol)
    assert _rel(gA.cpu().numpy(), oA) < 1e-4
    assert _rel(gB.cpu().numpy(), oB) < 1e-4
    s.close()


def test_autograd_function_matches_abi():
    m, n, r, K = 48, 40, 2, 9
    P = W.rotated_gaussian_psf(9, 2.0, 1.0, 0.3)
    g = W.rng(402)
    s = api.Sfista(P, (m, n), 1, r, prec="fp32", lipschitz=1.0)
    A, B = s.factors()
    b = torch.from_numpy(g.uniform(size=(m, n)).astype(np.float32)).cuda().requires_grad_(True)
    lam = torch.tensor(0.03, dtype=torch.float64, device="cuda", requires_grad=True)
    At = torch.from_numpy(A.astype(np.float32)).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B.astype(np.float32)).cuda().requires_grad_(True)
    xt = torch.from_numpy(g.uniform(size=(m, n)).astype(np.float32)).cuda()
    X = api.unrolled_solve(s, b, lam, K, ckpt_every=4, A=At, B=Bt)
    loss = ((X - xt) ** 2).sum()
    loss.backward()
    assert b.grad.shape == (m, n) and At.grad.shape == (r, n, n) and Bt.grad.shape == (r, m, m)
    ob, ol, oA, oB = adjoint.unrolled_grad(b.detach().double().cpu().numpy(), A, B, 1.0, 0.03, K,
                                           2.0 * (X.detach().double().cpu().numpy() - xt.double().cpu().numpy()))
    assert _rel(b.grad.cpu().numpy(), ob) < 1e-4
    assert abs(lam.grad.item() - ol) <= 1e-4 * abs(ol)
    assert _rel(At.grad.cpu().numpy(), oA) < 1e-4
    assert _rel(Bt.grad.cpu().numpy(), oB) < 1e-4
    s.close()


def test_config5_gradients_vs_central_differences():
    """512^2, r=3, 50 unrolled iterations, checkpoint every 10, loss ||X_50 - X_true||^2:
    directional derivatives along b, lambda, A and B vs FP64 central differences (<= 1e-3)."""
    pr = W.config5()
    n, r, K, ck = 512, pr.r, pr.iters, pr.extra["ckpt_every"]
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, r)
    Bf, Af = kron.dense_factors(ka)
    L, _ = oracle.lipschitz(ka, np.ones((n, n)), tol=1e-9, maxit=300)
    lam = pr.lam
    s = api.Sfista(pr.psf, (n, n), pr.bc, r, prec="fp32", lipschitz=L)
    db = torch.from_numpy(b).cuda()
    ckpt = torch.empty(2 * ((K + ck - 1) // ck), n, n, dtype=torch.float64, device="cuda")
    X = torch.empty_like(db)
    api.sfista_unrolled_fwd(s.ctx, db, lam, K, ck, ckpt, X)
    torch.cuda.synchronize()
    gX = 2.0 * (X.double() - torch.from_numpy(pr.x_true).cuda())
    gb = torch.empty_like(db)
    gA = torch.empty(r, n, n, device="cuda")
    gB = torch.empty(r, n, n, device="cuda")
    gl = api.sfista_unrolled_bwd(s.ctx, db, lam, K, ck, ckpt, gX.float().contiguous(), gb, gA, gB)
    b64 = b.astype(np.float64)

    def loss(bb=b64, AA=Af, BB=Bf, ll=lam):
        return adjoint.loss_true(bb, AA, BB, L, ll, K, pr.x_true)[0]

    g = W.rng(403)
    Db = g.standard_normal((n, n))
    DA = g.standard_normal(Af.shape) * (Af != 0)
    DB = g.standard_normal(Bf.shape) * (Bf != 0)
    checks = []
    e = 1e-3
    checks.append((np.vdot(gb.double().cpu().numpy(), Db), (loss(bb=b64 + e * Db) - loss(bb=b64 - e * Db)) / (2 * e)))
    e = 1e-6
    checks.append((gl, (loss(ll=lam + e) - loss(ll=lam - e)) / (2 * e)))
    e = 1e-5
    checks.append((np.vdot(gA.double().cpu().numpy(), DA), (loss(AA=Af + e * DA) - loss(AA=Af - e * DA)) / (2 * e)))
    checks.append((np.vdot(gB.double().cpu().numpy(), DB), (loss(BB=Bf + e * DB) - loss(BB=Bf - e * DB)) / (2 * e)))
    for k, (ad, fd) in enumerate(checks):
        assert abs(ad - fd) <= 1e-3 * abs(fd), (k, ad, fd)
    s.close()


def _band_mask(F):
    """Entries of the stacked factors F that lie inside their band (the band of the setup's factors)."""
    rows, cols = np.nonzero(np.any(F != 0.0, axis=0))
    lo, hi = int((cols - rows).min()), int((cols - rows).max())
    idx = np.arange(F.shape[1])
    off = idx[None, :] - idx[:, None]
    return (off >= lo) & (off <= hi)


@pytest.mark.parametrize("op", ["banded", "banded_persistent"])
def test_autograd_follows_the_factors_passed(op):
    """Perturbed factors (inside the band) passed to the autograd function change the forward, and forward and
    gradients then match the oracle's reverse mode run with those same factors; a factor with an entry outside
    the band is refused."""
    m, n, r, K = 48, 40, 2, 9
    P = W.rotated_gaussian_psf(9, 2.0, 1.0, 0.3)
    g = W.rng(403)
    s = api.Sfista(P, (m, n), 1, r, prec="fp32", op=op, lipschitz=1.0)
    A0, B0 = s.factors()
    A = A0 + 0.05 * g.standard_normal(A0.shape) * _band_mask(A0)[None] * (A0 != 0).any(axis=0)[None]
    B = B0 + 0.05 * g.standard_normal(B0.shape) * _band_mask(B0)[None] * (B0 != 0).any(axis=0)[None]
    b = torch.from_numpy(g.uniform(size=(m, n)).astype(np.float32)).cuda()
    xt = torch.from_numpy(g.uniform(size=(m, n)).astype(np.float32)).cuda()
    lam = torch.tensor(0.03, dtype=torch.float64, device="cuda", requires_grad=True)
    X0 = api.unrolled_solve(s, b, lam, K, ckpt_every=4).detach()
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    X = api.unrolled_solve(s, b, lam, K, ckpt_every=4, A=At, B=Bt)
    b64 = b.double().cpu().numpy()
    Xo = adjoint.unrolled_forward(b64, A, B, 1.0, 0.03, K)[0]
    assert _rel(X.detach().cpu().numpy(), Xo) < 1e-5
    assert _rel(X0.cpu().numpy(), Xo) > 1e-3          # the perturbation matters
    loss = ((X - xt) ** 2).sum()
    loss.backward()
    ob, ol, oA, oB = adjoint.unrolled_grad(b64, A, B, 1.0, 0.03, K,
                                           2.0 * (X.detach().double().cpu().numpy() - xt.double().cpu().numpy()))
    assert abs(lam.grad.item() - ol) <= 1e-4 * abs(ol)
    assert _rel(At.grad.cpu().numpy(), oA) < 1e-4
    assert _rel(Bt.grad.cpu().numpy(), oB) < 1e-4
    np.testing.assert_allclose(s.factors()[0], A.astype(np.float64), rtol=0, atol=0)
    bad = A.copy()
    bad[0, 0, n - 1] = 1.0                              # far outside the band
    with pytest.raises(api.SfistaError) as ei:
        s.set_factors(bad, None)
    assert ei.value.status == api.EINVAL
    with pytest.raises(api.SfistaError) as ei:
        s.profiles()
    assert ei.value.status == api.ENOTSUP
    s.close()
