"""FP32 refinement of the tensor-core forms (option refine_every): every
k_ref-th iteration runs all of Step 1 of Alg. 2 (the residual and the adjoint
product) with the FP32 band kernels instead of the low-precision GEMMs.
Checked against the FP64 oracle, for a lower error than the same form without
refinement, for bit-exact resume and graph replay, and for its rejection in
batches."""
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


M, N, R, LAM, ITERS = 96, 128, 2, 0.01, 40


@pytest.fixture(scope="module")
def case():
    g = W.rng(611)
    P = W.rotated_gaussian_psf(15, 2.5, 1.2, 0.4)
    x = W.shapes_image(g, M, N, rects=6, ellipses=6)
    bx = oracle.blur(x, P, 7, 7, 1)
    b = (bx + W.noise_scale(bx, g.standard_normal((M, N)), 0.01)).astype(np.float32)
    ka = kron.kron_approx(P, 7, 7, M, N, 1, R)
    L, _ = oracle.lipschitz(ka, np.ones((M, N)), tol=1e-9, maxit=300)
    ref = oracle.sfista(b.astype(np.float64), ka, L, LAM, ITERS)
    return P, b, L, ref


def _solve(case, prec, every, **kw):
    P, b, L, _ = case
    s = api.Sfista(P, (M, N), 1, R, prec=prec, op="gemm_band", lipschitz=L, refine_every=every, **kw)
    X = s.solve_device(torch.from_numpy(b).cuda(), LAM, ITERS)
    s.close()
    return X


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-4), ("tf32x3", 1e-4), ("tf32", 2e-2), ("bf16", 5e-2)])
@pytest.mark.parametrize("every", [1, 3])
def test_refined_solve_matches_oracle(case, prec, tol, every):
    ref = case[3]
    err = oracle.rel_fro(_solve(case, prec, every).cpu().numpy(), ref)
    assert err <= tol, (prec, every, err)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_refined_resume_and_graph_are_bit_exact(case, prec):
    """The refined iterations are fixed by the absolute k, so a solve split at
    k = 18 (not a multiple of k_ref = 4) continues from the same state, and the
    stream-ordered loop gives the graph's result bit for bit.  The BF16x3 form
    keeps an FP32 state and resumes bit for bit; TF32x3 keeps a double-float
    state, which crosses the FP64 boundary of sfista_solve_state rounded where
    a pair's low word lies more than 29 bits below its high word, so its
    resumed solve agrees to the last bits of FP64 (1e-13 relative)."""
    P, b, L, _ = case
    db = torch.from_numpy(b).cuda()
    s = api.Sfista(P, (M, N), 1, R, prec=prec, op="gemm_band", lipschitz=L, refine_every=4)
    X = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    Xp = torch.zeros_like(X)
    s.solve_state(db, LAM, 0, 30, X, Xp)
    whole = X.clone()
    X.zero_()
    Xp.zero_()
    s.solve_state(db, LAM, 0, 18, X, Xp)
    s.solve_state(db, LAM, 18, 12, X, Xp)
    if prec == "bf16x3":
        assert torch.equal(X, whole)
    else:
        assert (torch.linalg.norm(X - whole) / torch.linalg.norm(whole)).item() <= 1e-13
    s.close()
    assert torch.equal(_solve(case, prec, 4), _solve(case, prec, 4, use_graph=False))


def test_refinement_changes_the_iterates(case):
    assert not torch.equal(_solve(case, "bf16x3", 2), _solve(case, "bf16x3", 0))


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
def test_refinement_lowers_the_error(case, prec):
    """Refined iterations carry no low-precision product error, so the error against the FP64 oracle
    falls as k_ref falls: for the single-product forms, whose error is all product error, refining
    every second iteration at least roughly halves it; refining every iteration reaches the FP32
    operator's level (these forms keep an FP32 state, so 1e-5), below BF16x3's own, which the FP32
    state bounds from below."""
    ref = case[3]
    e0 = oracle.rel_fro(_solve(case, prec, 0).cpu().numpy(), ref)
    e2 = oracle.rel_fro(_solve(case, prec, 2).cpu().numpy(), ref)
    e1 = oracle.rel_fro(_solve(case, prec, 1).cpu().numpy(), ref)
    assert e1 < e2 < e0, (prec, e0, e2, e1)
    if prec != "bf16x3":
        assert e2 < 0.7 * e0, (prec, e0, e2)
    assert e1 <= 1e-5, (prec, e1)


def test_batches_reject_refined_tensor_forms(case):
    P, b, L, _ = case
    a = api.Sfista(P, (M, N), 1, R, prec="bf16x3", op="gemm_band", lipschitz=L, refine_every=2)
    c = api.Sfista(P, (M, N), 1, R, prec="bf16x3", op="gemm_band", lipschitz=L)
    with pytest.raises(api.SfistaError) as ei:
        api.Batch([c, a])
    assert ei.value.status == api.ENOTSUP
    a.close()
    c.close()
