"""The autotuner (sfista_tune): every candidate it keeps must still match the
FP64 oracle, term chunking must not change the arithmetic (bitwise equal to
the untuned two-pass result), and batches must pick up the tuned chunks."""
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


def _problem(m, n, p, r, seed):
    g = W.rng(seed)
    P = W.gaussian_mixture_psf(g, p)
    x = W.shapes_image(g, m, n, rects=4, ellipses=4)
    c = (p - 1) // 2
    bx = oracle.blur(x, P, c, c, 1)
    b = (bx + W.noise_scale(bx, g.standard_normal((m, n)), 0.01)).astype(np.float32)
    ka = kron.kron_approx(P, c, c, m, n, 1, r)
    L, _ = oracle.lipschitz(ka, np.ones((m, n)), tol=1e-9, maxit=300)
    return P, b, ka, L


def test_tune_keeps_explicit_banded_form_and_its_arithmetic():
    P, b, ka, L = _problem(200, 176, 15, 4, 501)
    lam, iters = 0.006, 40
    db = torch.from_numpy(b).cuda()
    ref = api.Sfista(P, b.shape, 1, 4, prec="fp32", op="banded", lipschitz=L)
    X0 = ref.solve_device(db, lam, iters)
    s = api.Sfista(P, b.shape, 1, 4, prec="fp32", op="banded", lipschitz=L)
    log = s.tune(iters=5)
    assert s.info()["op"] == "banded"
    stages = {e["stage"] for e in log if e["stage"] >= 0}
    assert stages == {0, 1, 2, 3}
    assert all(e["ms"] > 0 for e in log)
    for st in range(4):     # every chunk 1..r was tried for every stage (all fit at this width)
        assert sorted(e["chunk"] for e in log if e["stage"] == st) == [1, 2, 3, 4]
    X1 = s.solve_device(db, lam, iters)
    assert torch.equal(X0, X1)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, lam, iters)
    assert oracle.rel_fro(X1.cpu().numpy(), Xo) <= 1e-5
    s.close()
    ref.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-4)])
def test_tune_auto_form_matches_oracle(prec, tol):
    P, b, ka, L = _problem(128, 160, 13, 3, 502)
    lam, iters = 0.005, 40
    s = api.Sfista(P, b.shape, 1, 3, prec=prec, op="auto", lipschitz=L)
    log = s.tune(iters=5)
    whole = {e["op"] for e in log if e["stage"] == -1}
    if prec == "fp32":
        # 4 x 5 tiles: the one-launch fused solver fits as well; the FFT form is always timed
        assert whole == {"banded", "banded_fused", "banded_persistent", "fft"}
        assert s.info()["op"] in whole
    else:
        assert whole == {"gemm_band", "gemm_dense"}
        assert s.info()["op"] in whole
    X = s.solve_device(torch.from_numpy(b).cuda(), lam, iters).cpu().numpy()
    Xo = oracle.sfista(b.astype(np.float64), ka, L, lam, iters)
    assert oracle.rel_fro(X, Xo) <= tol
    s.close()


def test_batch_uses_tuned_chunks():
    specs = [(96, 128, 11, 2, 503), (128, 96, 17, 3, 504), (64, 64, 9, 1, 505)]
    pr = [_problem(*sp) for sp in specs]
    lam, iters = 0.005, 30
    solvers = [api.Sfista(P, b.shape, 1, ka.r, prec="fp32", op="banded", lipschitz=L) for P, b, ka, L in pr]
    for s in solvers:
        s.tune(iters=3)
    d_bs = [torch.from_numpy(b).cuda() for _, b, _, _ in pr]
    batch = api.Batch(solvers)
    outs = batch.solve(d_bs, [lam] * len(pr), iters)
    for X, (P, b, ka, L), s, db in zip(outs, pr, solvers, d_bs):
        Xo = oracle.sfista(b.astype(np.float64), ka, L, lam, iters)
        assert oracle.rel_fro(X.cpu().numpy(), Xo) <= 1e-5
        assert torch.equal(X, s.solve_device(db, lam, iters))
    batch.close()
    for s in solvers:
        s.close()


def test_batch_tune_keeps_results():
    specs = [(96, 128, 11, 2, 506), (128, 96, 17, 3, 507), (64, 64, 9, 1, 508), (200, 176, 23, 4, 509)]
    pr = [_problem(*sp) for sp in specs]
    lam, iters = 0.005, 30
    solvers = [api.Sfista(P, b.shape, 1, ka.r, prec="fp32", op="banded", lipschitz=L) for P, b, ka, L in pr]
    d_bs = [torch.from_numpy(b).cuda() for _, b, _, _ in pr]
    batch = api.Batch(solvers)
    before = [X.clone() for X in batch.solve(d_bs, [lam] * len(pr), iters)]
    log = batch.tune(iters=3)
    assert log and all(e["ms"] > 0 for e in log)
    plans = [(e["op"], e["budget_kb"]) for e in log]
    assert len(set(plans)) == len(plans)    # distinct plans only
    # 4 + 4x3 + 2x2 + 7x6 tiles of 32 x 32: the one-launch plan is a candidate
    assert ("banded_persistent", 0) in plans
    after = batch.solve(d_bs, [lam] * len(pr), iters)
    for X0, X1, (P, b, ka, L) in zip(before, after, pr):
        assert torch.equal(X0, X1)     # chunking regroups terms, not the arithmetic
        Xo = oracle.sfista(b.astype(np.float64), ka, L, lam, iters)
        assert oracle.rel_fro(X1.cpu().numpy(), Xo) <= 1e-5
    batch.close()
    for s in solvers:
        s.close()
