"""Seeded synthetic inputs for the sFISTA workloads.

Images in [0, 1], point spread functions and standard-normal noise draws with
the shapes and statistics of the paper's experiments (square images,
reflective or zero boundary, Gaussian noise of 0.5-1 %, Kronecker rank up to
5).  The paper's own test images and PSFs (IR Tools, Sec. 4) are not
available, so these stand in for them.

This module holds none of the method's arithmetic: it only draws random
numbers and evaluates closed-form PSF shapes.  Blurring the true image is
left to the caller (the library's exact-blur kernel, or the oracle in tests),
and ``noise_scale`` only rescales a noise draw to a relative level
(NoiseLevel = ||noise|| / ||b||, Sec. 4).

Every generator takes a seed; config k of the workload table uses
``SEED_BASE + k`` with numpy's PCG64 ``default_rng``.
"""
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 19010913


def rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- images
def rectangles_image(g, m, n, count=10, side=(4, 24)):
    """Axis-aligned rectangles, later ones overwrite, background 0, intensities U[0,1]."""
    X = np.zeros((m, n))
    for _ in range(count):
        h = int(g.integers(side[0], side[1] + 1))
        w = int(g.integers(side[0], side[1] + 1))
        a = int(g.integers(0, max(1, m - h + 1)))
        b = int(g.integers(0, max(1, n - w + 1)))
        X[a:a + h, b:b + w] = g.uniform(0.0, 1.0)
    return X


def shapes_image(g, m, n, rects=12, ellipses=12):
    """Rectangles and rotated ellipses, intensities U[0,1], later ones overwrite."""
    X = np.zeros((m, n))
    aa, bb = np.mgrid[0:m, 0:n].astype(np.float64)
    smax = max(8, min(m, n) // 8)
    for _ in range(rects):
        h = int(g.integers(8, 2 * smax + 1))
        w = int(g.integers(8, 2 * smax + 1))
        a = int(g.integers(0, max(1, m - h + 1)))
        b = int(g.integers(0, max(1, n - w + 1)))
        X[a:a + h, b:b + w] = g.uniform(0.0, 1.0)
    for _ in range(ellipses):
        ra, rb = g.uniform(8, smax, size=2)
        th = g.uniform(0.0, np.pi)
        a0, b0 = g.uniform(0, m), g.uniform(0, n)
        u = (bb - b0) * np.cos(th) + (aa - a0) * np.sin(th)
        v = -(bb - b0) * np.sin(th) + (aa - a0) * np.cos(th)
        X[(u / rb) ** 2 + (v / ra) ** 2 <= 1.0] = g.uniform(0.0, 1.0)
    return X


def dots_image(g, m, n, count=None, sigma=(1.0, 3.0)):
    """Small Gaussian-shaped dots of peak U[0.3, 1] at uniform positions (a
    stand-in for the 'dot' test images of Example 2); count defaults to n/2."""
    count = max(1, n // 2) if count is None else count
    X = np.zeros((m, n))
    aa, bb = np.mgrid[0:m, 0:n].astype(np.float64)
    for _ in range(count):
        a0, b0 = g.uniform(0, m), g.uniform(0, n)
        s = g.uniform(*sigma)
        X = np.maximum(X, g.uniform(0.3, 1.0) * np.exp(-((aa - a0) ** 2 + (bb - b0) ** 2) / (2.0 * s * s)))
    return X


def smooth_edges_image(g, m, n, sigma=32.0, rects=40):
    """Gaussian-filtered white noise scaled to [0, 0.6] plus rectangles of step U[0.2,0.4], clipped."""
    from scipy.ndimage import gaussian_filter

    F = gaussian_filter(g.standard_normal((m, n)), sigma, mode="reflect")
    F = 0.6 * (F - F.min()) / max(F.max() - F.min(), 1e-300)
    smax = max(8, min(m, n) // 8)
    for _ in range(rects):
        h = int(g.integers(8, 2 * smax + 1))
        w = int(g.integers(8, 2 * smax + 1))
        a = int(g.integers(0, max(1, m - h + 1)))
        b = int(g.integers(0, max(1, n - w + 1)))
        F[a:a + h, b:b + w] += g.uniform(0.2, 0.4)
    return np.clip(F, 0.0, 1.0)


# ---------------------------------------------------------------- PSFs
def _grid(p):
    h = (p - 1) / 2.0
    y, x = np.mgrid[0:p, 0:p].astype(np.float64)
    return x - h, y - h   # x = column offset, y = row offset (downwards)


def gaussian_psf(p, sigma):
    """Isotropic Gaussian exp(-(x^2+y^2)/(2 sigma^2)), normalised to sum 1 (separable)."""
    x, y = _grid(p)
    P = np.exp(-(x * x + y * y) / (2.0 * sigma * sigma))
    return P / P.sum()


def rotated_gaussian_psf(p, sx, sy, theta):
    """Anisotropic Gaussian with axes rotated by theta, normalised to sum 1."""
    x, y = _grid(p)
    u = x * np.cos(theta) + y * np.sin(theta)
    v = -x * np.sin(theta) + y * np.cos(theta)
    P = np.exp(-u * u / (2.0 * sx * sx) - v * v / (2.0 * sy * sy))
    return P / P.sum()


def moffat_psf(p, alpha, beta):
    x, y = _grid(p)
    P = (1.0 + (x * x + y * y) / (alpha * alpha)) ** (-beta)
    return P / P.sum()


def mixture_moffat_psf(g, p):
    """0.3/0.25/0.25 of three rotated Gaussians plus 0.2 of a Moffat tail (alpha 4, beta 2.5)."""
    P = np.zeros((p, p))
    for wgt in (0.3, 0.25, 0.25):
        sx = g.uniform(1.5, 6.0)
        sy = g.uniform(1.0, 4.0)
        P += wgt * rotated_gaussian_psf(p, sx, sy, g.uniform(0.0, np.pi))
    P += 0.2 * moffat_psf(p, 4.0, 2.5)
    return P / P.sum()


def gaussian_mixture_psf(g, p):
    """A mixture of 1-3 rotated Gaussians with sigma in U[1, p/6], normalised."""
    k = int(g.integers(1, 4))
    P = np.zeros((p, p))
    for _ in range(k):
        sx, sy = g.uniform(1.0, max(1.0001, p / 6.0), size=2)
        P += g.uniform(0.2, 1.0) * rotated_gaussian_psf(p, sx, sy, g.uniform(0.0, np.pi))
    return P / P.sum()


def defocus_psf(p, radius):
    """Out-of-focus blur: a uniform disk of the given radius (pixel centres with
    x^2 + y^2 <= radius^2), normalised to sum 1 (the defocus family of Example 2)."""
    x, y = _grid(p)
    P = (x * x + y * y <= radius * radius).astype(np.float64)
    return P / P.sum()


def shake_psf(g, p, steps):
    """Camera-shake blur: a seeded random walk from the centre (steps of
    N(0, 1) px in each axis, kept inside the p x p support), its visits
    accumulated with bilinear weights and normalised to sum 1 (the shake
    family of Example 2)."""
    P = np.zeros((p, p))
    c = (p - 1) / 2.0
    pos = np.array([c, c])
    for _ in range(steps):
        pos = np.clip(pos + g.standard_normal(2), 0.0, p - 1.0)
        i0, j0 = int(np.floor(pos[0])), int(np.floor(pos[1]))
        fi, fj = pos[0] - i0, pos[1] - j0
        for di, wi in ((0, 1.0 - fi), (1, fi)):
            for dj, wj in ((0, 1.0 - fj), (1, fj)):
                if i0 + di < p and j0 + dj < p:
                    P[i0 + di, j0 + dj] += wi * wj
    return P / P.sum()


def random_psf(g, p, q):
    """Dense non-symmetric positive PSF (small test cases)."""
    P = g.uniform(0.05, 1.0, size=(p, q))
    return P / P.sum()


# ---------------------------------------------------------------- noise
def noise_draw(g, m, n):
    return g.standard_normal((m, n))


def laplace_noise_draw(g, m, n):
    """Laplace draw of unit variance (scale 1/sqrt(2))."""
    return g.laplace(0.0, 1.0 / np.sqrt(2.0), size=(m, n))


def noise_scale(blurred, draw, level):
    """Scale a noise draw so that ||noise|| / ||blurred|| = level (NoiseLevel of Sec. 4)."""
    nb = float(np.linalg.norm(blurred))
    nd = float(np.linalg.norm(draw))
    return draw * (level * nb / nd)


def noise_of_kind(kind, blurred, draw, level):
    """Noise e with ||e|| / ||blurred|| = level: 'gauss' and 'laplace' add the
    scaled draw; 'multiplicative' scales it by the blurred image first
    (e proportional to blurred * draw, zero where the signal is zero)."""
    if kind == "multiplicative":
        return noise_scale(blurred, blurred * draw, level)
    return noise_scale(blurred, draw, level)


# ---------------------------------------------------------------- configs
@dataclass
class Problem:
    """One restoration problem: true image, PSF (centre = middle pixel), settings."""
    name: str
    x_true: np.ndarray
    psf: np.ndarray
    bc: int            # 0 zero, 1 reflective
    r: int
    lam: float
    noise_level: float
    iters: int
    noise: np.ndarray  # standard-normal draw, same shape as x_true
    extra: dict = field(default_factory=dict)

    @property
    def centre(self):
        return (self.psf.shape[0] - 1) // 2, (self.psf.shape[1] - 1) // 2


def config1(seed=SEED_BASE + 1, n=64):
    """64^2 rectangles, separable 9x9 Gaussian sigma=2 (r=1 exact), zero BC, lam 0.01, 1 %, 100 its."""
    g = rng(seed)
    x = rectangles_image(g, n, n)
    return Problem("cfg1_64_r1_zero", x, gaussian_psf(9, 2.0), 0, 1, 0.01, 0.01, 100,
                   noise_draw(g, n, n))


def config2(seed=SEED_BASE + 2, n=512):
    """512^2 shapes, 31x31 rotated Gaussian (3, 1, 30 deg), reflective, r=3, lam 0.005, 1 %, 200 its."""
    g = rng(seed)
    x = shapes_image(g, n, n)
    return Problem("cfg2_512_r3_reflexive", x,
                   rotated_gaussian_psf(31, 3.0, 1.0, np.deg2rad(30.0)), 1, 3, 0.005,
                   0.01, 200, noise_draw(g, n, n))


def config3(seed=SEED_BASE + 3, n=2048):
    """2048^2 smooth field + edges, 63x63 mixture + Moffat PSF, reflective, r=5, lam 0.002, 0.5 %, 300 its."""
    g = rng(seed)
    x = smooth_edges_image(g, n, n)
    return Problem("cfg3_2048_r5_reflexive", x, mixture_moffat_psf(g, 63), 1, 5, 0.002,
                   0.005, 300, noise_draw(g, n, n))


def config4(seed=SEED_BASE + 4, count=64, sizes=(256, 384, 512, 768, 1024)):
    """64 problems of uneven size, PSF width and rank; reflective, lam 0.005, 1 %, 150 its."""
    g = rng(seed)
    out = []
    for k in range(count):
        n = int(g.choice(sizes))
        p = int(g.choice(np.arange(15, 42, 2)))
        r = int(g.integers(1, 5))
        x = shapes_image(g, n, n)
        out.append(Problem("cfg4_%02d_%d_p%d_r%d" % (k, n, p, r), x,
                           gaussian_mixture_psf(g, p), 1, r, 0.005, 0.01, 150,
                           noise_draw(g, n, n)))
    return out


def wide_psf(seed=SEED_BASE + 7, n=512, p=127):
    """Config 2's image with a p x p mixture + Moffat PSF (p about n / 4: a PSF wide enough that the
    band forms' cost per pixel, which grows with p, exceeds the FFT form's), reflective, r=3,
    lam 0.005, 1 %, 200 its."""
    pr = config2(n=n)
    g = rng(seed)
    pr.name = "wide_%d_p%d_r3" % (n, p)
    pr.psf = mixture_moffat_psf(g, p)
    pr.noise = noise_draw(g, n, n)
    return pr


def config5(seed=SEED_BASE + 2, n=512):
    """Config 2's problem (same seed) unrolled for 50 iterations (checkpoint every 10) for gradients."""
    pr = config2(seed=seed, n=n)
    pr.name = "cfg5_512_r3_unrolled"
    pr.iters = 50
    pr.extra["ckpt_every"] = 10
    return pr


EX2_LEVELS = ("mild", "medium", "severe")
EX2_NOISES = ("gauss", "laplace", "multiplicative")


def example2_cases(seed=SEED_BASE + 6, n=256, r=5, iters=50, level=0.01, lam=0.005):
    """Example 2 stand-in: two blur families (defocus disk, camera shake) at
    three blur levels, each with three noise types, on images cycling through
    the geometric, dots and smooth stand-ins; reflective boundary, r terms,
    50 iterations (the paper's fixed count).  18 problems; the noise type is
    in extra['noise'] and the noise draw matches it (Laplace draw for
    'laplace', standard normal otherwise)."""
    g = rng(seed)
    radii = {"mild": 2.0, "medium": 4.0, "severe": 7.0}
    shake = {"mild": (9, 12), "medium": (15, 30), "severe": (21, 60)}
    out = []
    k = 0
    for fam in ("defocus", "shake"):
        for lev in EX2_LEVELS:
            if fam == "defocus":
                R = radii[lev]
                P = defocus_psf(2 * int(np.ceil(R)) + 3, R)
            else:
                p, steps = shake[lev]
                P = shake_psf(g, p, steps)
            for noise in EX2_NOISES:
                kind = k % 3
                x = (shapes_image(g, n, n), dots_image(g, n, n), smooth_edges_image(g, n, n, sigma=n / 16.0,
                                                                                   rects=8))[kind]
                draw = laplace_noise_draw(g, n, n) if noise == "laplace" else noise_draw(g, n, n)
                pr = Problem("ex2_%s_%s_%s" % (fam, lev, noise), x, P, 1, min(r, *P.shape), lam, level, iters,
                             draw, {"noise": noise, "family": fam, "level": lev})
                out.append(pr)
                k += 1
    return out


# ---------------------------------------------------------------- comparison of large results
# A full 2048^2 result is too large to keep beside the tests, so a long
# reference run is stored as a summary that any later result can be compared
# with: the values at a seeded set of pixels, and a CountSketch (each pixel
# added with a random sign into one of k buckets).  For a difference image d,
# ||S d||^2 has expectation ||d||_F^2 and relative standard deviation about
# sqrt(2 / k) (Charikar, Chen, Farach-Colton 2002; a sparse Johnson-
# Lindenstrauss embedding), so ||S x - S x_ref|| / ||x_ref|| estimates the
# relative Frobenius error without the reference image.  Only seeded draws
# and sums: none of the method's arithmetic.
def sample_pixels(shape, count, seed):
    """Flat indices of `count` seeded pixels plus the four corners and the
    middle of every edge (the boundary rows and columns matter for the
    boundary condition)."""
    m, n = shape
    g = rng(seed)
    idx = g.choice(m * n, size=count, replace=False)
    edge = [0, n - 1, (m - 1) * n, m * n - 1, n // 2, (m - 1) * n + n // 2, (m // 2) * n, (m // 2) * n + n - 1]
    return np.unique(np.concatenate([idx, np.asarray(edge)])).astype(np.int64)


def count_sketch(X, k, seed):
    """CountSketch of the flattened image X into k buckets (FP64)."""
    X = np.asarray(X, dtype=np.float64).ravel()
    g = rng(seed)
    bucket = g.integers(0, k, size=X.size)
    sign = g.integers(0, 2, size=X.size) * 2.0 - 1.0
    return np.bincount(bucket, weights=sign * X, minlength=k)
