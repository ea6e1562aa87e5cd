"""Writes the stored FP64 oracle results of the batched workload's checked problems.

The batched workload has 64 problems of sizes 256^2 .. 1024^2 (reflective
boundary, Gaussian-mixture PSFs of 15-41 px, r in 1..4, lambda = 0.005, 1 %
noise, 150 iterations).  One problem of every size class is checked against
the oracle: the one with the most Kronecker terms (ties: the widest PSF).
For each, this script stores

  k           the problem's index in the workload
  L           lambda_max(A_s^T A_s) by the oracle's power iteration
  b_norm      ||b|| of the observation b = A x_true + e (oracle exact blur)
  idx, vals   X_150 at seeded pixels (and the corners and edge middles)
  sketch      CountSketch of X_150 (see workloads.count_sketch)
  x_norm      ||X_150||_F

Only oracle/ and the seeded input module are called.  Run from the
repository root:  python tests/golden/make_config4_reference.py
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

OUT = os.path.join(HERE, "config4_oracle_150.npz")
SAMPLE_SEED = W.SEED_BASE + 400
SKETCH_SEED = W.SEED_BASE + 401
SKETCH_K = 2048
SAMPLES = 2048


def checked_problems(probs):
    """Index of the checked problem of each size class (most terms, then widest PSF)."""
    best = {}
    for k, pr in enumerate(probs):
        n = pr.x_true.shape[0]
        key = (pr.r, pr.psf.shape[0])
        if n not in best or key > best[n][0]:
            best[n] = (key, k)
    return [best[n][1] for n in sorted(best)]


def observation(pr):
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    return bx + W.noise_scale(bx, pr.noise, pr.noise_level)


def main():
    t0 = time.time()
    probs = W.config4()
    out = {}
    ks = checked_problems(probs)
    for j, k in enumerate(ks):
        pr = probs[k]
        n = pr.x_true.shape[0]
        cr, cc = pr.centre
        b32 = observation(pr).astype(np.float32).astype(np.float64)
        ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
        L, lit = oracle.lipschitz(ka, np.ones((n, n)), tol=1e-10, maxit=400)
        X = oracle.sfista(b32, ka, L, pr.lam, pr.iters)
        idx = W.sample_pixels((n, n), SAMPLES, SAMPLE_SEED + k)
        out.update({"k%d" % j: k, "L%d" % j: L, "b_norm%d" % j: np.linalg.norm(b32), "idx%d" % j: idx,
                    "vals%d" % j: X.ravel()[idx], "sketch%d" % j: W.count_sketch(X, SKETCH_K, SKETCH_SEED + k),
                    "x_norm%d" % j: np.linalg.norm(X)})
        print("%s: L = %.12g (%d steps), %.0f s" % (pr.name, L, lit, time.time() - t0), flush=True)
    np.savez_compressed(OUT, count=len(ks), sample_seed=SAMPLE_SEED, sketch_seed=SKETCH_SEED, sketch_k=SKETCH_K,
                        **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
