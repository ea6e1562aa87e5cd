"""Full-length runs of the two largest workloads against stored FP64 oracle results.

The 2048^2 workload (r = 5, 63 x 63 PSF, 300 iterations) and the largest
problems of the batched workload (up to 1024^2, 150 iterations) take the FP64
oracle minutes, so committed scripts in tests/golden/ ran it once and stored,
for each result X_ref, its values at seeded pixels, a CountSketch S X_ref and
||X_ref||_F (plus the oracle's L, which both sides take as Alg. 2's step
input).  Each test here rebuilds the same observation b with the oracle's
exact blur and the seeded noise draw, solves on the GPU with the stored L,
and checks
  - the sampled pixels element by element: the root-mean-square difference
    over the samples relative to that of X_ref (an unbiased estimate of the
    relative Frobenius error), and the largest single difference;
  - ||S (X - X_ref)|| / ||X_ref||, which estimates the relative Frobenius
    error of the whole image (a CountSketch preserves squared norms in
    expectation, relative spread about sqrt(2 / buckets));
  - for the split-precision forms, PSNR against x_true within 0.01 dB of the
    oracle's.
Tolerances: 1e-5 for the FP32 operator, 1e-4 for BF16x3 / TF32x3.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = {"fp32": 1e-5, "tf32x3": 1e-4, "bf16x3": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _observation(pr):
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    return (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)


def check_against_summary(X, idx, vals, sketch, x_norm, sketch_seed, tol, label):
    X = np.asarray(X, dtype=np.float64)
    d = X.ravel()[idx] - vals
    sampled = float(np.sqrt(np.mean(d * d)) / np.sqrt(np.mean(vals * vals)))
    worst = float(np.max(np.abs(d)) / (x_norm / np.sqrt(X.size)))
    est = float(np.linalg.norm(W.count_sketch(X, len(sketch), sketch_seed) - sketch) / x_norm)
    assert sampled <= tol, "%s: sampled rel. error %.3e" % (label, sampled)
    assert est <= tol, "%s: sketched rel. Frobenius error %.3e" % (label, est)
    assert worst <= 20 * tol, "%s: largest sampled difference %.3e (in RMS units)" % (label, worst)
    assert abs(np.linalg.norm(X) / x_norm - 1.0) <= tol
    return sampled, est


@pytest.fixture(scope="module")
def cfg3():
    ref = np.load(os.path.join(GOLDEN, "config3_oracle_300.npz"))
    pr = W.config3()
    b = _observation(pr)
    b64 = b.astype(np.float64)
    assert abs(np.linalg.norm(b64) / float(ref["b_norm"]) - 1.0) < 1e-12
    assert abs(b64.sum() / float(ref["b_sum"]) - 1.0) < 1e-10
    return pr, _cuda(b), ref


@pytest.mark.parametrize("prec,op", [("fp32", "auto"), ("fp32", "fft"), ("bf16x3", "gemm_band"),
                                     ("tf32x3", "gemm_band"), ("bf16x3", "gemm_dense")])
def test_config3_300_iterations(cfg3, prec, op):
    """2048^2, r = 5, 63 x 63 mixture + Moffat PSF, reflective, lambda 0.002: all 300 iterations of Alg. 2."""
    pr, db, ref = cfg3
    L = float(ref["L"])
    s = api.Sfista(pr.psf, (2048, 2048), pr.bc, pr.r, prec=prec, op=op, lipschitz=L)
    tol = TOL[prec]
    X10 = s.solve_device(db, pr.lam, 10).cpu().numpy()
    check_against_summary(X10, ref["idx"], ref["vals10"], ref["sketch10"], float(ref["x_norm10"]),
                          int(ref["sketch_seed"]), tol, "%s X_10" % prec)
    X = s.solve_device(db, pr.lam, int(ref["iters"])).cpu().numpy()
    check_against_summary(X, ref["idx"], ref["vals"], ref["sketch"], float(ref["x_norm"]),
                          int(ref["sketch_seed"]), tol, "%s X_300" % prec)
    if prec != "fp32":
        assert abs(oracle.psnr(X, pr.x_true) - float(ref["psnr"])) <= 0.01
    s.close()


@pytest.mark.parametrize("prec,op", [("fp32", "banded"), ("bf16x3", "gemm_band")])
def test_config4_every_size_class(prec, op):
    """The batched workload (64 problems, 256^2 .. 1024^2, r 1..4, 150 iterations) in one batch;
    the checked problem of every size class (most terms, widest PSF) against the oracle."""
    ref = np.load(os.path.join(GOLDEN, "config4_oracle_150.npz"))
    probs = W.config4()
    iters = probs[0].iters
    checked = {int(ref["k%d" % j]): j for j in range(int(ref["count"]))}
    assert sorted({probs[k].x_true.shape[0] for k in checked}) == [256, 384, 512, 768, 1024]
    d_bs, solvers = [], []
    for k, pr in enumerate(probs):
        if k in checked:
            j = checked[k]
            b = _observation(pr)
            assert abs(np.linalg.norm(b.astype(np.float64)) / float(ref["b_norm%d" % j]) - 1.0) < 1e-12
            d_bs.append(_cuda(b))
            L = float(ref["L%d" % j])
        else:
            # Problems that are not checked only need to be of the right shape
            # and scale: their data come from the library.
            xt = _cuda(pr.x_true)
            bx = api.sfista_blur(pr.psf, xt, pr.bc).double().cpu().numpy()
            d_bs.append(_cuda(bx + W.noise_scale(bx, pr.noise, pr.noise_level)))
            L = 1.05   # above lambda_max(A_s^T A_s) (about 1 for these normalised PSFs)
        solvers.append(api.Sfista(pr.psf, pr.x_true.shape, pr.bc, pr.r, prec=prec, op=op, lipschitz=L))
    for sv in solvers:
        sv.tune(iters=2)
    batch = api.Batch(solvers)
    batch.tune(iters=2)
    outs = batch.solve(d_bs, [pr.lam for pr in probs], iters)
    for k, j in checked.items():
        check_against_summary(outs[k].cpu().numpy(), ref["idx%d" % j], ref["vals%d" % j], ref["sketch%d" % j],
                              float(ref["x_norm%d" % j]), int(ref["sketch_seed"]) + k, TOL[prec],
                              "%s %s" % (prec, probs[k].name))
    batch.close()
    for sv in solvers:
        sv.close()
