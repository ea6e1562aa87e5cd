"""Writes the stored FP64 oracle result of the 2048^2 workload (300 iterations).

The 2048 x 2048 problem (smooth field plus edges, 63 x 63 mixture + Moffat
PSF, reflective boundary, r = 5 Kronecker terms, lambda = 0.002, 0.5 %
noise) takes the FP64 oracle several minutes per hundred iterations, so its
300-iteration result is computed once by this script and kept as a summary:

  L           lambda_max(A_s^T A_s) by the oracle's power iteration (the
              step size of Alg. 2; both sides take it as an input)
  b_norm, b_sum
              of the observation b = A x_true + e (exact blur of Eq. 1.1
              by the oracle, noise from the seeded draw), so a test can
              check that it rebuilt the same b
  idx, vals   X_300 at seeded pixels (and the corners and edge middles)
  sketch      CountSketch of X_300 (k buckets, seeded): estimates the
              relative Frobenius error of another result (see
              workloads.count_sketch)
  x_norm      ||X_300||_F
  psnr        PSNR(X_300, x_true), peak 1
  vals10, sketch10, x_norm10
              the same for X_10 (a short check)

Only oracle/ and the seeded input module are called.  Run from the
repository root:  python tests/golden/make_config3_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import kron  # noqa: E402
from paper_1901_00913_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "config3_oracle_300.npz")
SAMPLE_SEED = W.SEED_BASE + 300
SKETCH_SEED = W.SEED_BASE + 301
SKETCH_K = 4096
SAMPLES = 4096


def observation(pr):
    """b = A x_true + e with the oracle's exact blur (Eq. 1.1)."""
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    return bx + W.noise_scale(bx, pr.noise, pr.noise_level)


def main():
    t0 = time.time()
    pr = W.config3()
    n = pr.x_true.shape[0]
    cr, cc = pr.centre
    b = observation(pr)
    # Both sides solve with the FP32 observation, as the library receives it.
    b32 = b.astype(np.float32).astype(np.float64)
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
    L, lit = oracle.lipschitz(ka, np.ones((n, n)), tol=1e-12, maxit=400)
    print("L = %.17g after %d power steps (%.0f s)" % (L, lit, time.time() - t0), flush=True)
    idx = W.sample_pixels((n, n), SAMPLES, SAMPLE_SEED)
    X10 = oracle.sfista(b32, ka, L, pr.lam, 10)
    print("10 iterations done (%.0f s)" % (time.time() - t0), flush=True)
    X = oracle.sfista(b32, ka, L, pr.lam, pr.iters)
    print("%d iterations done (%.0f s)" % (pr.iters, time.time() - t0), flush=True)
    np.savez_compressed(
        OUT, L=L, lam=pr.lam, iters=pr.iters, b_norm=np.linalg.norm(b32), b_sum=b32.sum(),
        idx=idx, vals=X.ravel()[idx], sketch=W.count_sketch(X, SKETCH_K, SKETCH_SEED),
        x_norm=np.linalg.norm(X), psnr=oracle.psnr(X, pr.x_true),
        vals10=X10.ravel()[idx], sketch10=W.count_sketch(X10, SKETCH_K, SKETCH_SEED),
        x_norm10=np.linalg.norm(X10), sample_seed=SAMPLE_SEED, sketch_seed=SKETCH_SEED)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
