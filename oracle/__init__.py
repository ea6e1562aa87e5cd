"""FP64 CPU oracle for structured FISTA (arXiv 1901.00913).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_1901_00913_gb300/`` never does, and the two share no code.  The one
module both sides use is the seeded input generator
``paper_1901_00913_gb300.workloads``, which holds none of the method's
arithmetic.

Modules
-------
``_native``  builds and loads ``sfista_oracle.c`` (exact blur, the Kronecker
             operator as 1-D boundary-aware convolutions, Alg. 1 on an explicit
             matrix and on the exact blur, Alg. 2, power iteration for L).
``kron``     Kronecker approximation of Sec. 2 / Theorem 1 (Gram weights,
             Cholesky, SVD of the weighted PSF, factor profiles, dense
             toep/hank factors for small checks).
``solve``    sFISTA driver, t-schedule, objective and metrics.
"""
from . import _native  # noqa: F401
from .kron import (  # noqa: F401
    KronApprox,
    gram_matrix,
    kron_approx,
    operator_matrix_1d,
    dense_factors,
    explicit_blur_matrix,
    explicit_kron_matrix,
)
from .solve import (  # noqa: F401
    blur,
    blur_T,
    kron_apply,
    kron_apply_T,
    lipschitz,
    sfista,
    fista_dense,
    fista_exact,
    lipschitz_exact,
    objective,
    t_schedule,
    rel_fro,
    psnr,
)
