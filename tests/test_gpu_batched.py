"""Batched solves (grouped launches over problems of uneven size, PSF and rank)
vs the FP64 oracle and vs one-at-a-time solves, through the C ABI."""
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


def _problems():
    """Uneven sizes (with ragged 128-tile tails), PSF widths, ranks and centres."""
    g = W.rng(301)
    specs = [(64, 64, 9, 1), (96, 136, 15, 2), (200, 176, 13, 3), (128, 128, 21, 4), (56, 80, 7, 2)]
    out = []
    for m, n, p, r in specs:
        P = W.gaussian_mixture_psf(g, p)
        x = W.shapes_image(g, m, n, rects=4, ellipses=4)
        cr, cc = (p - 1) // 2, (p - 1) // 2
        bx = oracle.blur(x, P, cr, cc, 1)
        b = (bx + W.noise_scale(bx, g.standard_normal((m, n)), 0.01)).astype(np.float32)
        ka = kron.kron_approx(P, cr, cc, m, n, 1, r)
        L, _ = oracle.lipschitz(ka, np.ones((m, n)), tol=1e-9, maxit=300)
        out.append((P, b, ka, L, 0.005 + 0.001 * r))
    return out


@pytest.fixture(scope="module")
def probs():
    pr = _problems()
    iters = 40
    refs = [oracle.sfista(b.astype(np.float64), ka, L, lam, iters) for P, b, ka, L, lam in pr]
    return pr, iters, refs


@pytest.mark.parametrize("prec,op,tol", [("fp32", "banded", 1e-5), ("fp32", "auto", 1e-5),
                                         ("bf16x3", "gemm_band", 1e-4), ("tf32x3", "gemm_band", 1e-4)])
def test_batched_matches_oracle_and_single(probs, prec, op, tol):
    """A batch runs the grouped kernels whatever form its contexts chose (FP32
    auto: the one-launch fused solver for the single solves here), with the
    same arithmetic in the same order."""
    pr, iters, refs = probs
    solvers = [api.Sfista(P, b.shape, 1, ka.r, prec=prec, op=op, lipschitz=L) for P, b, ka, L, lam in pr]
    d_bs = [torch.from_numpy(b).cuda() for P, b, ka, L, lam in pr]
    lams = [lam for *_, lam in pr]
    batch = api.Batch(solvers)
    for rep in range(2):     # second solve replays the cached graph
        outs = batch.solve(d_bs, lams, iters)
        for k, (X, ref) in enumerate(zip(outs, refs)):
            err = oracle.rel_fro(X.cpu().numpy(), ref)
            assert err <= tol, (prec, k, err)
    singles = [s.solve_device(db, lam, iters) for s, db, lam in zip(solvers, d_bs, lams)]
    for X, Y in zip(outs, singles):
        assert torch.equal(X, Y)     # same tiles, same arithmetic, same order
    batch.close()
    for s in solvers:
        s.close()


def test_solve_batched_one_shot(probs):
    pr, iters, refs = probs
    solvers = [api.Sfista(P, b.shape, 1, ka.r, prec="bf16x3", lipschitz=L) for P, b, ka, L, lam in pr[:3]]
    d_bs = [torch.from_numpy(b).cuda() for P, b, ka, L, lam in pr[:3]]
    outs = [torch.empty_like(d) for d in d_bs]
    api.sfista_solve_batched([s.ctx for s in solvers], d_bs, [lam for *_, lam in pr[:3]], iters, outs)
    torch.cuda.synchronize()
    for X, ref in zip(outs, refs[:3]):
        assert oracle.rel_fro(X.cpu().numpy(), ref) <= 1e-4


def test_batch_rejects_mixed_families():
    P = W.gaussian_psf(9, 2.0)
    a = api.Sfista(P, (64, 64), 1, 1, prec="fp32", lipschitz=1.0)
    b = api.Sfista(P, (64, 64), 1, 1, prec="bf16x3", lipschitz=1.0)
    with pytest.raises(api.SfistaError) as ei:
        api.Batch([a, b])
    assert ei.value.status == api.EINVAL
    with pytest.raises(api.SfistaError):
        api.Batch([a, a])
    a.close()
    b.close()


@pytest.mark.parametrize("prec,op,tol", [("fp32", "banded", 1e-5), ("bf16x3", "gemm_band", 1e-4)])
def test_batched_l1_per_problem(probs, prec, op, tol):
    """Each problem keeps its own l1 weight inside the grouped launches."""
    pr, iters, _ = probs
    mus = [0.0, 0.02, 0.05, 0.01, 0.03]
    refs = [oracle.sfista(b.astype(np.float64), ka, L, lam, iters, mu=mu)
            for (P, b, ka, L, lam), mu in zip(pr, mus)]
    solvers = [api.Sfista(P, b.shape, 1, ka.r, prec=prec, op=op, lipschitz=L, l1=mu)
               for (P, b, ka, L, lam), mu in zip(pr, mus)]
    d_bs = [torch.from_numpy(b).cuda() for P, b, ka, L, lam in pr]
    batch = api.Batch(solvers)
    outs = batch.solve(d_bs, [lam for *_, lam in pr], iters)
    for k, (X, ref) in enumerate(zip(outs, refs)):
        assert oracle.rel_fro(X.cpu().numpy(), ref) <= tol, (k, mus[k])
    batch.close()
    for s in solvers:
        s.close()


def test_batch_table_refresh_and_aliasing(probs):
    """Repeated solves of one batch (FP32 auto: the one-launch form, which
    reads each B in place and writes each X itself) follow every change of
    observations, weights and outputs, and an output may be its own input."""
    pr, iters, _ = probs
    solvers = [api.Sfista(P, b.shape, 1, ka.r, prec="fp32", lipschitz=L) for P, b, ka, L, lam in pr]
    d_bs = [torch.from_numpy(b).cuda() for P, b, ka, L, lam in pr]
    lams = [lam for *_, lam in pr]
    batch = api.Batch(solvers)
    outs = [torch.empty_like(d) for d in d_bs]

    def singles(bs, ls):
        return [s.solve_device(db, lam, iters) for s, db, lam in zip(solvers, bs, ls)]

    for rep in range(2):    # same buffers: the second solve reuses the device table
        batch.solve(d_bs, lams, iters, outs=outs)
        for X, Y in zip(outs, singles(d_bs, lams)):
            assert torch.equal(X, Y)
    d_bs2 = [0.5 * d + 0.1 for d in d_bs]
    lams2 = [2.0 * lam for lam in lams]
    batch.solve(d_bs2, lams2, iters, outs=outs)
    ref2 = singles(d_bs2, lams2)
    for X, Y in zip(outs, ref2):
        assert torch.equal(X, Y)
    inplace = [d.clone() for d in d_bs2]
    batch.solve(inplace, lams2, iters, outs=inplace)
    for X, Y in zip(inplace, ref2):
        assert torch.equal(X, Y)
    batch.close()
    for s in solvers:
        s.close()
