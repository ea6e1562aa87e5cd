"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Inputs are seeded and synthetic; the oracle computes its own factorisation,
operator and iterations in FP64, and both sides take the same FP32 b and the
same L (an input of Alg. 2, computed by the oracle).  Tolerances are relative
Frobenius errors: 1e-5 for the FP32 operator, 1e-4 (and 0.01 dB PSNR) for the
split-precision tensor-core operators.
"""
import numpy as np
import pytest

import oracle
from oracle import kron
from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-4, "bf16x3": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


def _problem(m, n, psf, bc, seed, noise=0.01, centre=None):
    g = W.rng(seed)
    x = W.shapes_image(g, m, n, rects=6, ellipses=6)
    cr, cc = centre if centre else ((psf.shape[0] - 1) // 2, (psf.shape[1] - 1) // 2)
    bx = oracle.blur(x, psf, cr, cc, bc)
    b = (bx + W.noise_scale(bx, g.standard_normal((m, n)), noise)).astype(np.float32)
    return x, b, (cr, cc)


def _oracle_L(ka, maxit=300):
    L, _ = oracle.lipschitz(ka, np.ones((ka.m, ka.n)), tol=1e-9, maxit=maxit)
    return L


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


# ------------------------------------------------------------------ exact blur
@pytest.mark.parametrize("bc", [0, 1])
def test_blur_exact_matches_oracle(bc):
    g = W.rng(101)
    P = W.random_psf(g, 7, 5)
    X = g.uniform(size=(200, 176))
    Y = api.sfista_blur(P, _cuda(X), bc, center=(2, 3)).cpu().numpy()
    Yo = oracle.blur(X.astype(np.float32).astype(np.float64), P.astype(np.float32).astype(np.float64), 2, 3, bc)
    assert oracle.rel_fro(Y, Yo) < 1e-6


# ------------------------------------------------------------------ operator
@pytest.mark.parametrize("op", ["banded", "banded_fused"])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("shape", [(200, 176), (64, 64), (37, 45)])
def test_apply_matches_oracle(bc, transpose, shape, op):
    """A_s X and A_s^T X on ragged sizes with a non-centred, non-square PSF."""
    m, n = shape
    g = W.rng(102 + m)
    P = W.random_psf(g, 13, 11)
    ka = kron.kron_approx(P, 4, 7, m, n, bc, 3)
    s = api.Sfista(P, (m, n), bc, 3, center=(4, 7), prec="fp32", op=op, lipschitz=1.0)
    X = g.standard_normal((m, n)).astype(np.float32)
    Y = s.apply(_cuda(X), transpose=transpose).cpu().numpy()
    Yo = (oracle.kron_apply_T if transpose else oracle.kron_apply)(X.astype(np.float64), ka)
    assert oracle.rel_fro(Y, Yo) < 1e-6
    s.close()


@pytest.mark.parametrize("psf_shape,centre,r", [((41, 9), (20, 4), 2), ((9, 10), (2, 6), 3), ((12, 13), (5, 5), 5),
                                               ((7, 14), (3, 0), 4), ((10, 7), (9, 6), 1), ((6, 11), (0, 10), 6)])
@pytest.mark.parametrize("shape", [(96, 100), (45, 38)])
def test_fused_apply_band_offsets(psf_shape, centre, r, shape):
    """The one-kernel operator over PSF widths and centres that give every
    column-offset class of the band (mod 4), term counts split 4 + rest, a
    column band wider than 32 rows, and aligned / unaligned image widths."""
    m, n = shape
    g = W.rng(110 + psf_shape[0] * 16 + psf_shape[1])
    P = W.random_psf(g, *psf_shape)
    ka = kron.kron_approx(P, centre[0], centre[1], m, n, 1, r)
    s = api.Sfista(P, (m, n), 1, r, center=centre, prec="fp32", op="banded_fused", lipschitz=1.0)
    assert s.info()["op"] == "banded_fused"
    X = g.standard_normal((m, n)).astype(np.float32)
    for transpose in (False, True):
        Y = s.apply(_cuda(X), transpose=transpose).cpu().numpy()
        Yo = (oracle.kron_apply_T if transpose else oracle.kron_apply)(X.astype(np.float64), ka)
        assert oracle.rel_fro(Y, Yo) < 1e-6
    s.close()


def test_adjoint_identity_gpu():
    g = W.rng(103)
    P = W.rotated_gaussian_psf(31, 3.0, 1.0, np.deg2rad(30))
    s = api.Sfista(P, (256, 240), 1, 3, prec="fp32", op="banded", lipschitz=1.0)
    X = _cuda(g.standard_normal((256, 240)))
    Y = _cuda(g.standard_normal((256, 240)))
    lhs = torch.sum(s.apply(X).double() * Y.double()).item()
    rhs = torch.sum(X.double() * s.apply(Y, transpose=True).double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    s.close()


def test_factors_match_oracle_dense():
    P = W.rotated_gaussian_psf(15, 3.0, 1.0, 0.4)
    s = api.Sfista(P, (48, 40), 1, 3, lipschitz=1.0)
    A, B = s.factors()
    ka = kron.kron_approx(P, 7, 7, 48, 40, 1, 3)
    Bo, Ao = kron.dense_factors(ka)
    np.testing.assert_allclose(A, Ao, atol=1e-12)
    np.testing.assert_allclose(B, Bo, atol=1e-12)
    s.close()


# ------------------------------------------------------------------ Lipschitz constant
@pytest.mark.parametrize("bc,r", [(0, 1), (1, 2), (1, 3)])
def test_lipschitz_matches_oracle(bc, r):
    P = W.rotated_gaussian_psf(9, 2.0, 1.0, 0.3)
    ka = kron.kron_approx(P, 4, 4, 24, 20, bc, r)
    As = kron.explicit_kron_matrix(ka)
    Lx = float(np.linalg.eigvalsh(As.T @ As).max())
    s = api.Sfista(P, (24, 20), bc, r, lipschitz_tol=1e-14, lipschitz_maxit=20000)
    L = s.info()["lipschitz"]
    assert abs(L - Lx) <= 1e-9 * Lx
    s.close()


# ------------------------------------------------------------------ Alg. 2
def test_solve_config1_fp32():
    """64^2, separable Gaussian (r=1 exact), zero boundary, 100 iterations."""
    pr = W.config1()
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, 64, 64, pr.bc, pr.r)
    L = _oracle_L(ka, maxit=3000)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, pr.lam, pr.iters)
    s = api.Sfista(pr.psf, (64, 64), pr.bc, pr.r, prec="fp32", lipschitz=L)
    Xd = s.solve_device(_cuda(b), pr.lam, pr.iters).cpu().numpy()
    Xh = s.solve(b, pr.lam, pr.iters)
    assert oracle.rel_fro(Xd, Xo) <= TOL["fp32"]
    np.testing.assert_array_equal(Xd, Xh)
    s.close()


@pytest.fixture(scope="module")
def cfg2():
    pr = W.config2()
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, 512, 512, pr.bc, pr.r)
    L = _oracle_L(ka)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, pr.lam, pr.iters)
    return pr, b, ka, L, Xo


@pytest.mark.parametrize("op", ["banded", "banded_fused", "banded_persistent"])
def test_solve_config2_fp32(cfg2, op):
    """512^2, rotated Gaussian, reflexive, r=3, 200 iterations: rel err <= 1e-5."""
    pr, b, ka, L, Xo = cfg2
    s = api.Sfista(pr.psf, (512, 512), pr.bc, pr.r, prec="fp32", op=op, lipschitz=L)
    X = s.solve_device(_cuda(b), pr.lam, pr.iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= TOL["fp32"]
    assert abs(oracle.psnr(X, pr.x_true) - oracle.psnr(Xo, pr.x_true)) <= 0.01
    s.close()


@pytest.mark.parametrize("op", ["banded", "banded_fused", "banded_persistent"])
@pytest.mark.parametrize("bc", [0, 1])
def test_solve_ragged(bc, op):
    m, n = 200, 176
    g = W.rng(104)
    P = W.random_psf(g, 11, 9)
    x, b, (cr, cc) = _problem(m, n, P, bc, 105, centre=(3, 5))
    ka = kron.kron_approx(P, cr, cc, m, n, bc, 3)
    L = _oracle_L(ka)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.01, 60)
    s = api.Sfista(P, (m, n), bc, 3, center=(cr, cc), prec="fp32", op=op, lipschitz=L)
    X = s.solve_device(_cuda(b), 0.01, 60).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= TOL["fp32"]
    s.close()


@pytest.mark.parametrize("m,n", [(200, 176), (202, 178), (640, 512)])
def test_persistent_forms_match_oracle(m, n):
    """The one-launch solver takes the fused form (band tiles and state resident)
    when m, n are multiples of 4 and every tile has a co-resident block
    (200 x 176: 16-row tiles, the last strip ragged), else the two-pass form
    (202 x 178: not multiples of 4; 640 x 512: 320 tiles of 32 rows, more than
    two per SM).  Both against the oracle, and a resumed solve against the
    uninterrupted one."""
    P = W.rotated_gaussian_psf(31, 3.0, 1.0, 0.5)
    x, b, _ = _problem(m, n, P, 1, 108)
    ka = kron.kron_approx(P, 15, 15, m, n, 1, 3)
    L = _oracle_L(ka)
    iters = 24
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.005, iters)
    s = api.Sfista(P, (m, n), 1, 3, prec="fp32", op="banded_persistent", lipschitz=L)
    db = _cuda(b)
    X = s.solve_device(db, 0.005, iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= TOL["fp32"]
    ref = torch.zeros(m, n, dtype=torch.float64, device="cuda")
    s.solve_state(db, 0.005, 0, iters, ref, torch.zeros_like(ref))
    Xs, Xp = torch.zeros_like(ref), torch.zeros_like(ref)
    s.solve_state(db, 0.005, 0, 10, Xs, Xp)
    s.solve_state(db, 0.005, 10, iters - 10, Xs, Xp)
    assert torch.max(torch.abs(Xs - ref)).item() <= 1e-12
    assert oracle.rel_fro(ref.cpu().numpy(), Xo) <= TOL["fp32"]
    s.close()


@pytest.mark.parametrize("psf_shape,centre,r", [((9, 9), (4, 4), 3), ((7, 14), (3, 0), 4), ((10, 7), (9, 6), 1),
                                               ((41, 37), (20, 18), 2), ((6, 11), (0, 10), 5)])
def test_one_launch_solver_band_offsets(psf_shape, centre, r):
    """The one-launch fused solver over PSF widths and centres that give every
    column-offset class of both operators' bands (mod 4), term counts split
    4 + rest, and bands wider than 32 rows (two row groups in the row pass),
    against the oracle and the two-launch fused form."""
    m, n = 96, 100
    g = W.rng(140 + psf_shape[0] * 16 + psf_shape[1])
    P = W.random_psf(g, *psf_shape)
    x, b, _ = _problem(m, n, P, 1, 141, centre=centre)
    ka = kron.kron_approx(P, centre[0], centre[1], m, n, 1, r)
    L = _oracle_L(ka)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.01, 20)
    db = _cuda(b)
    outs = {}
    for op in ("banded_persistent", "banded_fused"):
        s = api.Sfista(P, (m, n), 1, r, center=centre, prec="fp32", op=op, lipschitz=L)
        outs[op] = s.solve_device(db, 0.01, 20).cpu().numpy()
        s.close()
    assert oracle.rel_fro(outs["banded_persistent"], Xo) <= TOL["fp32"]
    # the same arithmetic in the same order: the two forms agree bit for bit
    assert np.array_equal(outs["banded_persistent"], outs["banded_fused"])


@pytest.mark.parametrize("shape,th", [((512, 512), 28), ((512, 512), 60), ((512, 512), 64), ((200, 176), 16),
                                      ((200, 176), 36), ((200, 176), 48), ((200, 176), 64)])
def test_one_launch_solver_every_tile_height(shape, th):
    """Tile heights of both block sizes of the one-launch solver (256 threads up to 32 rows, 512 threads
    above; 200 x 176 leaves a ragged last strip) against the oracle, and bit for bit against the
    two-launch fused form (every pixel's sums are formed in the same order whatever the tiling)."""
    m, n = shape
    P = W.rotated_gaussian_psf(31, 3.0, 1.0, np.deg2rad(30))
    x, b, _ = _problem(m, n, P, 1, 150 + th)
    ka = kron.kron_approx(P, 15, 15, m, n, 1, 3)
    L = _oracle_L(ka)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.005, 30)
    db = _cuda(b)
    s = api.Sfista(P, (m, n), 1, 3, prec="fp32", op="banded_persistent", lipschitz=L, tile_override=th)
    X = s.solve_device(db, 0.005, 30).cpu().numpy()
    s.close()
    f = api.Sfista(P, (m, n), 1, 3, prec="fp32", op="banded_fused", lipschitz=L)
    Xf = f.solve_device(db, 0.005, 30).cpu().numpy()
    f.close()
    assert oracle.rel_fro(X, Xo) <= TOL["fp32"]
    assert np.array_equal(X, Xf)


def test_earlier_contexts_keep_their_launch_limits():
    """Kernel attributes are per kernel, not per context or batch: creating a
    context (and a batch) with a smaller shared-memory layout after a larger
    one must leave the larger one launchable, for the one-launch solver, the
    two-launch fused form and the grouped batch."""
    g = W.rng(150)
    big = W.rotated_gaussian_psf(31, 3.0, 1.0, 0.5)
    small = W.random_psf(g, 5, 5)
    m, n = 96, 128
    x, b, _ = _problem(m, n, big, 1, 151)
    ka = kron.kron_approx(big, 15, 15, m, n, 1, 3)
    L = _oracle_L(ka)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.005, 15)
    db = _cuda(b)
    for op in ("banded_persistent", "banded_fused"):
        s_big = api.Sfista(big, (m, n), 1, 3, prec="fp32", op=op, lipschitz=L)
        s_small = api.Sfista(small, (64, 64), 1, 1, prec="fp32", op=op, lipschitz=1.0)
        X = s_big.solve_device(db, 0.005, 15).cpu().numpy()
        assert oracle.rel_fro(X, Xo) <= TOL["fp32"], op
        s_small.close()
        s_big.close()
    s_big = api.Sfista(big, (m, n), 1, 3, prec="fp32", op="banded", lipschitz=L)
    s_small = api.Sfista(small, (64, 64), 1, 1, prec="fp32", op="banded", lipschitz=1.0)
    batch_big = api.Batch([s_big])
    batch_small = api.Batch([s_small])
    X = batch_big.solve([db], [0.005], 15)[0].cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= TOL["fp32"]
    batch_small.close()
    batch_big.close()
    s_small.close()
    s_big.close()


def test_graph_and_direct_launch_agree():
    P = W.rotated_gaussian_psf(15, 2.0, 1.0, 0.3)
    x, b, _ = _problem(96, 80, P, 1, 106)
    outs = []
    for graph in (True, False):
        s = api.Sfista(P, (96, 80), 1, 2, lipschitz=1.0, use_graph=graph)
        outs.append(s.solve_device(_cuda(b), 0.01, 40).cpu().numpy())
        s.close()
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("op,prec,tol", [("banded", "fp32", 1e-6), ("banded_fused", "fp32", 1e-6),
                                         ("banded_persistent", "fp32", 1e-6), ("gemm_band", "tf32x3", 1e-6),
                                         ("gemm_band", "bf16x3", 1e-4)])
def test_resume_state_matches_uninterrupted(op, prec, tol):
    """A solve split at k = 20 continues bit for bit; TF32x3 keeps the
    double-float state, BF16x3 iterates on an FP32 state."""
    P = W.rotated_gaussian_psf(15, 2.0, 1.0, 0.3)
    x, b, _ = _problem(96, 80, P, 1, 107)
    s = api.Sfista(P, (96, 80), 1, 2, lipschitz=1.0, op=op, prec=prec)
    db = _cuda(b)
    X = torch.zeros(96, 80, dtype=torch.float64, device="cuda")
    Xp = torch.zeros_like(X)
    s.solve_state(db, 0.01, 0, 30, X, Xp)
    ref = X.clone()
    X.zero_()
    Xp.zero_()
    s.solve_state(db, 0.01, 0, 20, X, Xp)
    s.solve_state(db, 0.01, 20, 10, X, Xp)
    assert torch.max(torch.abs(X - ref)).item() <= 1e-12
    ka = kron.kron_approx(P, 7, 7, 96, 80, 1, 2)
    Xo = oracle.sfista(b.astype(np.float64), ka, 1.0, 0.01, 30)
    assert oracle.rel_fro(ref.cpu().numpy(), Xo) <= tol
    s.close()


@pytest.mark.parametrize("op,prec,tol", [("banded", "fp32", 1e-5), ("banded_fused", "fp32", 1e-5),
                                          ("banded_persistent", "fp32", 1e-5), ("gemm_band", "bf16x3", 1e-4)])
def test_projection_matches_oracle(op, prec, tol):
    P = W.rotated_gaussian_psf(15, 2.0, 1.0, 0.3)
    x, b, _ = _problem(96, 80, P, 1, 108)
    b = b - 0.1
    ka = kron.kron_approx(P, 7, 7, 96, 80, 1, 2)
    Xo = oracle.sfista(b.astype(np.float64), ka, 1.0, 0.01, 40, project=True)
    s = api.Sfista(P, (96, 80), 1, 2, lipschitz=1.0, project=True, op=op, prec=prec)
    X = s.solve_device(_cuda(b), 0.01, 40).cpu().numpy()
    assert X.min() >= 0.0
    assert oracle.rel_fro(X, Xo) <= tol
    s.close()


@pytest.mark.parametrize("op,prec,tol", [("banded", "fp32", 1e-5), ("banded_fused", "fp32", 1e-5),
                                         ("banded_persistent", "fp32", 1e-5), ("gemm_band", "bf16x3", 1e-4),
                                         ("gemm_dense", "tf32x3", 1e-4)])
@pytest.mark.parametrize("project", [False, True])
def test_l1_threshold_matches_oracle(op, prec, tol, project):
    """Step 1 with the l1 term (soft threshold tau = mu / (L + lambda^2)), optionally projected."""
    P = W.rotated_gaussian_psf(15, 2.0, 1.0, 0.3)
    x, b, _ = _problem(96, 80, P, 1, 109)
    ka = kron.kron_approx(P, 7, 7, 96, 80, 1, 2)
    L = _oracle_L(ka)
    mu = 0.03
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.01, 40, project=project, mu=mu)
    nz_o = np.count_nonzero(Xo == 0.0)
    assert 0.02 * Xo.size < nz_o < 0.98 * Xo.size      # the threshold is active
    s = api.Sfista(P, (96, 80), 1, 2, lipschitz=L, project=project, op=op, prec=prec, l1=mu)
    X = s.solve_device(_cuda(b), 0.01, 40).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= tol
    assert abs(np.count_nonzero(X == 0.0) - nz_o) <= 0.01 * Xo.size
    if project:
        assert X.min() >= 0.0
    s.close()


def test_l1_rejected_by_reverse_mode():
    P = W.gaussian_psf(7, 1.5)
    s = api.Sfista(P, (32, 32), 1, 1, lipschitz=1.0, l1=0.01)
    db = torch.zeros(32, 32, device="cuda")
    ck = torch.empty(2, 32, 32, dtype=torch.float64, device="cuda")
    with pytest.raises(api.SfistaError) as e:
        api.sfista_unrolled_fwd(s.ctx, db, 0.01, 5, 5, ck, torch.empty_like(db))
    assert e.value.status == 4     # SFISTA_ENOTSUP
    s.close()


@pytest.mark.parametrize("op,prec,tol", [("banded", "fp32", 1e-6), ("banded_fused", "fp32", 1e-6),
                                         ("gemm_band", "bf16x3", 1e-4)])
def test_objective_matches_oracle(op, prec, tol):
    """Phi_s(X) = 1/2 ||A_s X - B||^2 + 1/2 lam^2 ||X||^2 on the device vs the FP64 oracle."""
    P = W.rotated_gaussian_psf(15, 2.0, 1.0, 0.3)
    x, b, _ = _problem(96, 80, P, 1, 111)
    ka = kron.kron_approx(P, 7, 7, 96, 80, 1, 2)
    s = api.Sfista(P, (96, 80), 1, 2, lipschitz=1.0, op=op, prec=prec)
    X = W.rng(112).uniform(size=(96, 80)).astype(np.float32)
    phi = s.objective(_cuda(b), _cuda(X), 0.05)
    phio = oracle.objective(X.astype(np.float64), b.astype(np.float64), ka, 0.05)
    assert abs(phi - phio) <= tol * abs(phio)
    s.close()


@pytest.mark.parametrize("op,prec", [("banded", "fp32"), ("banded_fused", "fp32"), ("banded_persistent", "fp32"),
                                     ("gemm_band", "bf16x3"), ("gemm_dense", "tf32x3")])
def test_solves_are_bit_reproducible(op, prec):
    """Two solves of the same input give bit-identical results (no atomics in the reductions)."""
    P = W.rotated_gaussian_psf(15, 2.0, 1.0, 0.3)
    x, b, _ = _problem(128, 96, P, 1, 113)
    db = _cuda(b)
    s1 = api.Sfista(P, (128, 96), 1, 2, op=op, prec=prec)
    s2 = api.Sfista(P, (128, 96), 1, 2, op=op, prec=prec)
    assert s1.info()["lipschitz"] == s2.info()["lipschitz"]
    X1 = s1.solve_device(db, 0.01, 30)
    X2 = s1.solve_device(db, 0.01, 30)
    X3 = s2.solve_device(db, 0.01, 30)
    assert torch.equal(X1, X2) and torch.equal(X1, X3)
    s1.close()
    s2.close()


def test_zero_iterations_returns_zero():
    P = W.gaussian_psf(9, 2.0)
    s = api.Sfista(P, (40, 40), 0, 1, lipschitz=1.0)
    X = s.solve_device(_cuda(np.ones((40, 40))), 0.01, 0)
    assert torch.count_nonzero(X).item() == 0
    s.close()


def test_nonfinite_input_reported():
    P = W.gaussian_psf(9, 2.0)
    s = api.Sfista(P, (40, 40), 0, 1, lipschitz=1.0)
    b = np.ones((40, 40), dtype=np.float32)
    b[3, 3] = np.inf
    with pytest.raises(api.SfistaError) as ei:
        s.solve(b, 0.01, 5)
    assert ei.value.status == api.EINVAL
    with pytest.raises(api.SfistaError) as ei:
        s.solve_device(_cuda(b), 0.01, 5)
    assert ei.value.status == api.ENUMERIC
    X = s.solve_device(_cuda(np.ones((40, 40))), 0.01, 5)     # context still usable
    assert torch.isfinite(X).all().item()
    s.close()


# ------------------------------------------------------------------ full size
def test_config3_full_size_operator_and_steps():
    """2048^2, r=5, 63x63 mixture PSF: the operator, its adjoint and 2 iterations vs the oracle."""
    pr = W.config3()
    cr, cc = pr.centre
    n = 2048
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
    s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="fp32", lipschitz=1.0)
    assert s.info()["op"] == "banded"          # automatic choice at 2048^2 with a 63-wide band
    X = pr.x_true.astype(np.float32)
    for tr in (False, True):
        Y = s.apply(_cuda(X), transpose=tr).cpu().numpy()
        Yo = (oracle.kron_apply_T if tr else oracle.kron_apply)(X.astype(np.float64), ka)
        assert oracle.rel_fro(Y, Yo) < 1e-6
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    Xo = oracle.sfista(b.astype(np.float64), ka, 1.0, pr.lam, 2)
    Xg = s.solve_device(_cuda(b), pr.lam, 2).cpu().numpy()
    assert oracle.rel_fro(Xg, Xo) <= TOL["fp32"]
    s.close()


# ------------------------------------------------------------------ tensor-core operator
# Per-application relative error bounds of the operator by precision (the
# split forms are near FP32; single BF16 / TF32 keep 8 / 11 significant bits).
OP_TOL = {"bf16x3": 2e-5, "tf32x3": 2e-6, "bf16": 1e-2, "tf32": 2e-3}


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "bf16", "tf32"])
@pytest.mark.parametrize("op", ["gemm_band", "gemm_dense"])
@pytest.mark.parametrize("bc", [0, 1])
def test_gemm_apply_matches_oracle(prec, op, bc):
    """tcgen05 GEMM operator (A_s and A_s^T) on a ragged 200x176 image, r=3, non-centred PSF."""
    m, n = 200, 176
    g = W.rng(201 + bc)
    P = W.random_psf(g, 13, 11)
    ka = kron.kron_approx(P, 4, 7, m, n, bc, 3)
    s = api.Sfista(P, (m, n), bc, 3, center=(4, 7), prec=prec, op=op, lipschitz=1.0)
    assert s.info()["op"] == op and s.info()["prec"] == prec
    X = g.standard_normal((m, n)).astype(np.float32)
    for tr in (False, True):
        Y = s.apply(_cuda(X), transpose=tr).cpu().numpy()
        Yo = (oracle.kron_apply_T if tr else oracle.kron_apply)(X.astype(np.float64), ka)
        assert oracle.rel_fro(Y, Yo) < OP_TOL[prec], (prec, op, tr)
    s.close()


def test_gemm_band_and_dense_agree():
    """Skipping K tiles outside the band changes nothing but summation order."""
    P = W.rotated_gaussian_psf(31, 3.0, 1.0, np.deg2rad(30))
    X = _cuda(W.rng(202).standard_normal((384, 256)))
    ys = []
    for op in ("gemm_band", "gemm_dense"):
        s = api.Sfista(P, (384, 256), 1, 3, prec="bf16x3", op=op, lipschitz=1.0)
        ys.append(s.apply(X).double())
        s.close()
    assert (torch.linalg.norm(ys[0] - ys[1]) / torch.linalg.norm(ys[1])).item() < 1e-6


def test_gemm_rejects_unaligned_sizes():
    P = W.gaussian_psf(9, 2.0)
    with pytest.raises(api.SfistaError) as ei:
        api.Sfista(P, (100, 60), 1, 1, prec="bf16x3", op="gemm_band", lipschitz=1.0)
    assert ei.value.status == api.ENOTSUP


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_solve_config2_split_precision(cfg2, prec):
    """512^2, r=3, 200 iterations, split-precision tensor-core operator: <= 1e-4 and 0.01 dB."""
    pr, b, ka, L, Xo = cfg2
    s = api.Sfista(pr.psf, (512, 512), pr.bc, pr.r, prec=prec, op="gemm_band", lipschitz=L)
    X = s.solve_device(_cuda(b), pr.lam, pr.iters).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= TOL[prec]
    assert abs(oracle.psnr(X, pr.x_true) - oracle.psnr(Xo, pr.x_true)) <= 0.01
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_solve_config2_single_precision_reported(cfg2, prec):
    """Single-product BF16 / TF32 are reported, not held to 1e-4: bounded and finite."""
    pr, b, ka, L, Xo = cfg2
    s = api.Sfista(pr.psf, (512, 512), pr.bc, pr.r, prec=prec, op="gemm_band", lipschitz=L)
    X = s.solve_device(_cuda(b), pr.lam, pr.iters).cpu().numpy()
    err = oracle.rel_fro(X, Xo)
    assert np.isfinite(err) and err < 0.1
    s.close()


def test_gemm_solve_ragged_matches_oracle():
    m, n = 200, 176
    g = W.rng(203)
    P = W.random_psf(g, 11, 9)
    x, b, (cr, cc) = _problem(m, n, P, 1, 204, centre=(3, 5))
    ka = kron.kron_approx(P, cr, cc, m, n, 1, 3)
    L = _oracle_L(ka)
    Xo = oracle.sfista(b.astype(np.float64), ka, L, 0.01, 60)
    s = api.Sfista(P, (m, n), 1, 3, center=(cr, cc), prec="bf16x3", lipschitz=L)
    X = s.solve_device(_cuda(b), 0.01, 60).cpu().numpy()
    assert oracle.rel_fro(X, Xo) <= TOL["bf16x3"]
    s.close()


def test_config3_full_size_tensor_core():
    """2048^2, r=5, 63x63 PSF: BF16x3 operator and 2 iterations vs the oracle."""
    pr = W.config3()
    cr, cc = pr.centre
    n = 2048
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
    s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="bf16x3", op="gemm_band", lipschitz=1.0)
    X = pr.x_true.astype(np.float32)
    Y = s.apply(_cuda(X)).cpu().numpy()
    assert oracle.rel_fro(Y, oracle.kron_apply(X.astype(np.float64), ka)) < OP_TOL["bf16x3"]
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    Xo = oracle.sfista(b.astype(np.float64), ka, 1.0, pr.lam, 2)
    Xg = s.solve_device(_cuda(b), pr.lam, 2).cpu().numpy()
    assert oracle.rel_fro(Xg, Xo) <= TOL["bf16x3"]
    s.close()


def test_bounded_wait_times_out_and_context_survives():
    """A device wait that nothing satisfies gives up after ~1 s: ETIMEOUT, then the context still solves."""
    import time
    P = W.gaussian_psf(9, 2.0)
    s = api.Sfista(P, (40, 40), 0, 1, prec="bf16x3", lipschitz=1.0)
    t0 = time.perf_counter()
    st = api.sfista_selftest_wait_timeout(s.ctx)
    dt = time.perf_counter() - t0
    assert st == api.ETIMEOUT
    assert 0.2 < dt < 30.0
    X = s.solve_device(_cuda(np.ones((40, 40))), 0.01, 5)
    assert torch.isfinite(X).all().item()
    s.close()
