"""Host diagnostics of a problem (not on the solver's path).

The paper motivates small Kronecker ranks by how fast the singular values of
the PSF P and of its weighted rearrangement P_bar decay (Sec. 3.2, the ratios
of the 6th and 10th singular values to the largest).  P_bar's values come from
the library's FP64 setup (``Sfista.info()['sigma']``); P's are computed here.
"""
import numpy as np


def psf_singular_values(psf):
    """Singular values of the PSF matrix P (FP64, descending)."""
    return np.linalg.svd(np.asarray(psf, dtype=np.float64), compute_uv=False)


def decay_ratios(sigma, ks=(2, 6, 10)):
    """sigma_k / sigma_1 for each k in ks that exists (1-based k)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.size == 0 or sigma[0] == 0.0:
        return {}
    return {int(k): float(sigma[k - 1] / sigma[0]) for k in ks if k <= sigma.size}
