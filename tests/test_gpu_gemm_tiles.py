"""Tile shapes of the tensor-core stages.

The summed stages (1, 3) run with N tiles of 64, 128 or 256 columns, the
stacked stages (0, 2) with 64 or 128 (gemm_bn = 64 sets every stage), and
the stacked stages either stream each tile's factor panel or keep it
resident in shared memory for the tiles that share it.  None of this may
change the result beyond summation order: every shape matches the FP64
oracle (Sec. 2 products, Alg. 2 solves) and the resident panel is bit-exact
against the streamed one (the same MMAs on the same operands in the same
order)."""
import numpy as np
import pytest

import oracle
from oracle import kron
from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Per-application bounds of the operator (as in the GEMM parity tests).
OP_TOL = {"bf16x3": 2e-5, "tf32x3": 2e-6, "bf16": 1e-2}
# 392 x 520: 4 row tiles (the last ragged) and column tiles of 64, 128 or 256
# (the last ragged); a 31 x 25 non-centred PSF, r = 3.
M, N = 392, 520


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _shapes():
    return [(bn, stream) for bn in (64, 128, 256) for stream in (False, True)]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32x3"])
@pytest.mark.parametrize("bc", [0, 1])
def test_tile_shapes_apply_match_oracle(prec, bc):
    g = W.rng(601 + bc)
    P = W.random_psf(g, 31, 25)
    cr, cc = 12, 9
    ka = kron.kron_approx(P, cr, cc, M, N, bc, 3)
    X = g.standard_normal((M, N)).astype(np.float32)
    ref = {tr: (oracle.kron_apply_T if tr else oracle.kron_apply)(X.astype(np.float64), ka) for tr in (False, True)}
    out = {}
    for bn, stream in _shapes():
        s = api.Sfista(P, (M, N), bc, 3, center=(cr, cc), prec=prec, op="gemm_band", lipschitz=1.0, gemm_bn=bn,
                       gemm_resident_panels=not stream)
        for tr in (False, True):
            Y = s.apply(_cuda(X), transpose=tr)
            out[(bn, stream, tr)] = Y
            assert oracle.rel_fro(Y.cpu().numpy(), ref[tr]) < OP_TOL[prec], (bn, stream, tr)
        s.close()
    for bn in (64, 128, 256):
        for tr in (False, True):
            # resident panel == streamed panel, bit for bit
            assert torch.equal(out[(bn, False, tr)], out[(bn, True, tr)]), (bn, tr)
    for bn in (64, 256):
        for tr in (False, True):
            a, b = out[(128, False, tr)].double(), out[(bn, False, tr)].double()
            assert (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item() < 1e-6


def _problem(seed, p=31, q=25):
    g = W.rng(seed)
    P = W.random_psf(g, p, q)
    x = W.shapes_image(g, M, N, rects=5, ellipses=5)
    cr, cc = (p - 1) // 2 - 3, (q - 1) // 2 + 2
    bx = oracle.blur(x, P, cr, cc, 1)
    b = (bx + W.noise_scale(bx, g.standard_normal((M, N)), 0.01)).astype(np.float32)
    ka = kron.kron_approx(P, cr, cc, M, N, 1, 3)
    L, _ = oracle.lipschitz(ka, np.ones((M, N)), tol=1e-9, maxit=300)
    return P, (cr, cc), x, b, ka, L


@pytest.fixture(scope="module")
def solved():
    P, c, x, b, ka, L = _problem(611)
    lam, iters = 0.004, 60
    Xo = oracle.sfista(b.astype(np.float64), ka, L, lam, iters)
    return P, c, x, b, ka, L, lam, iters, Xo


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tile_shapes_solve_match_oracle(solved, prec):
    """60 iterations of Alg. 2 with every tile shape: <= 1e-4 and 0.01 dB against the oracle."""
    P, c, x, b, ka, L, lam, iters, Xo = solved
    res = {}
    for bn, stream in _shapes():
        s = api.Sfista(P, (M, N), 1, 3, center=c, prec=prec, op="gemm_band", lipschitz=L, gemm_bn=bn,
                       gemm_resident_panels=not stream)
        X = s.solve_device(_cuda(b), lam, iters)
        res[(bn, stream)] = X
        Xn = X.cpu().numpy()
        assert oracle.rel_fro(Xn, Xo) <= 1e-4, (bn, stream)
        assert abs(oracle.psnr(Xn, x) - oracle.psnr(Xo, x)) <= 0.01
        s.close()
    for bn in (64, 128, 256):
        assert torch.equal(res[(bn, False)], res[(bn, True)])


def test_wide_band_streams_its_panels():
    """A band wider than three K blocks (71 taps: up to 205 columns per row tile) cannot keep its panel
    resident; the default then streams it, and the tuner offers only streamed shapes for stages 0 and 2."""
    P, c, x, b, ka, L = _problem(612, p=71, q=71)
    lam, iters = 0.004, 20
    Xo = oracle.sfista(b.astype(np.float64), ka, L, lam, iters)
    s = api.Sfista(P, (M, N), 1, 3, center=c, prec="bf16x3", op="gemm_band", lipschitz=L)
    log = s.tune(iters=2)
    assert sorted(e["chunk"] for e in log if e["stage"] == 0) == [64, 128]   # no resident-panel entries
    assert sorted(e["chunk"] for e in log if e["stage"] == 1) == [64, 128, 256]
    X = s.solve_device(_cuda(b), lam, iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-4
    s.close()


def test_tune_times_every_tile_shape(solved):
    P, c, x, b, ka, L, lam, iters, Xo = solved
    s = api.Sfista(P, (M, N), 1, 3, center=c, prec="bf16x3", op="gemm_band", lipschitz=L)
    log = s.tune(iters=3)
    by_stage = {st: sorted(e["chunk"] for e in log if e["stage"] == st) for st in range(4)}
    assert by_stage == {0: [64, 65, 128, 129], 1: [64, 128, 256], 2: [64, 65, 128, 129], 3: [64, 128, 256]}
    assert all(e["ms"] > 0 for e in log)
    assert s.info()["op"] == "gemm_band"
    X = s.solve_device(_cuda(b), lam, iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= 1e-4
    s.close()


def test_batch_resident_panels_bit_exact():
    """Grouped stages 0 and 2 with resident and with streamed panels give the same bits; the batch
    tuner times both."""
    specs = [(256, 384, 15, 2, 621), (384, 256, 21, 3, 622), (128, 128, 9, 1, 623)]
    probs = []
    for m, n, p, r, seed in specs:
        g = W.rng(seed)
        P = W.gaussian_mixture_psf(g, p)
        xx = W.shapes_image(g, m, n, rects=3, ellipses=3)
        cc = (p - 1) // 2
        bx = oracle.blur(xx, P, cc, cc, 1)
        bb = (bx + W.noise_scale(bx, g.standard_normal((m, n)), 0.01)).astype(np.float32)
        ka = kron.kron_approx(P, cc, cc, m, n, 1, r)
        L, _ = oracle.lipschitz(ka, np.ones((m, n)), tol=1e-9, maxit=300)
        probs.append((P, bb, ka, L))
    lam, iters = 0.005, 30
    d_bs = [_cuda(bb) for _, bb, _, _ in probs]
    outs = {}
    for stream in (False, True):
        solvers = [api.Sfista(P, bb.shape, 1, ka.r, prec="bf16x3", op="gemm_band", lipschitz=L,
                              gemm_resident_panels=not stream) for P, bb, ka, L in probs]
        batch = api.Batch(solvers)
        outs[stream] = [X.clone() for X in batch.solve(d_bs, [lam] * len(probs), iters)]
        if not stream:
            log = batch.tune(iters=2)
            assert len(log) == 2 and all(e["ms"] > 0 for e in log)
            after = batch.solve(d_bs, [lam] * len(probs), iters)
            for X0, X1 in zip(outs[stream], after):
                assert torch.equal(X0, X1)
        batch.close()
        for s in solvers:
            s.close()
    for X0, X1, (P, bb, ka, L) in zip(outs[False], outs[True], probs):
        assert torch.equal(X0, X1)
        Xo = oracle.sfista(bb.astype(np.float64), ka, L, lam, iters)
        assert oracle.rel_fro(X0.cpu().numpy(), Xo) <= 1e-4
