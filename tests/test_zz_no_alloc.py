"""sfista_apply_static, the operator entry point that allocates nothing.

Callers that cannot allocate device memory (a plugin whose host framework
owns all GPU memory through its own arena, or a latency-critical loop that
cannot afford an allocation's synchronisation or failure) use this call; its
intermediate images live in a fixed 32 MiB device array inside the library.
This test builds the band tables from the context's dense factors, calls the
entry point twice in a row through the C ABI and compares each result with
sfista_apply on the same context.  It sits in its own file, collected last.
"""
import numpy as np
import pytest

from paper_1901_00913_gb300 import api, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _band(F):
    """Band table (r, w, len) and lo of a stack of square banded matrices F[i][row][col]."""
    r, n, _ = F.shape
    rows, cols = np.nonzero(np.any(F != 0.0, axis=0))
    off = cols - rows
    lo, hi = int(off.min()), int(off.max())
    w = hi - lo + 1
    T = np.zeros((r, w, n))
    for k in range(w):
        for row in range(n):
            col = row + lo + k
            if 0 <= col < n:
                T[:, k, row] = F[:, row, col]
    return torch.from_numpy(T.astype(np.float32)).cuda(), lo


def _host_bands(P, m, n, r, transpose):
    """Band tables of the right and left factors from the library's host-only
    factorisation (no dense factors: used at 2048^2)."""
    bc = api.BC["reflexive"]
    right, lo_r, _ = api.sfista_factor_bands(P, m, n, bc, r, 1 if transpose else 0)
    left, lo_l, _ = api.sfista_factor_bands(P, m, n, bc, r, 3 if transpose else 2)
    dev = lambda T: torch.from_numpy(T.astype(np.float32)).cuda()   # noqa: E731
    return dev(right), lo_r, dev(left), lo_l


# 200 x 176: the 16-byte kernels with 32-row tiles; 201 x 177: sizes that are
# not multiples of 4 take the scalar kernels; 2048 x 2048 with r = 2 fills the
# static array exactly (r * m * n = 8,388,608 floats) and takes the 128-row
# column pass.
@pytest.mark.parametrize("m,n,r,transpose", [(200, 176, 3, False), (200, 176, 3, True), (201, 177, 3, False),
                                             (201, 177, 2, True), (2048, 2048, 2, False)])
def test_static_scratch_operator_matches_context_operator(m, n, r, transpose):
    import __graft_entry__ as g
    g.build()
    P = W.rotated_gaussian_psf(15, 3.0, 1.0, np.deg2rad(30))
    s = api.Sfista(P, (m, n), "reflexive", r, prec="fp32", op="banded", lipschitz=1.0)
    if m * n > 1 << 20:
        bandA, loA, bandB, loB = _host_bands(P, m, n, r, transpose)
    else:
        A, B = s.factors()
        if transpose:
            A, B = A.transpose(0, 2, 1), B.transpose(0, 2, 1)
        bandA, loA = _band(A)
        bandB, loB = _band(B)
    gen = W.rng(2024)
    for call in range(2):
        x = torch.from_numpy(gen.standard_normal((m, n)).astype(np.float32)).cuda()
        ref = s.apply(x, transpose=transpose)
        y = torch.full_like(x, float("nan"))
        api.sfista_apply_static(x, y, r, bandA, loA, bandB, loB)
        torch.cuda.synchronize()
        err = (torch.linalg.norm((y - ref).double()) / torch.linalg.norm(ref.double())).item()
        assert err <= 1e-6, "call %d: rel err %.3e" % (call, err)
    s.close()


def test_static_scratch_rejects_oversize_and_bad_offsets():
    import __graft_entry__ as g
    g.build()
    x = torch.zeros(16, 16, device="cuda")
    y = torch.zeros_like(x)
    band = torch.zeros(1, 3, 16, device="cuda")
    # beyond the static array (r * m * n = 32769 * 256 = 8,388,864 > 8 Mi floats); no kernel runs
    with pytest.raises(api.SfistaError) as ei:
        api.sfista_apply_static(x, y, 32769, band, -1, band, -1)
    assert ei.value.status == api.EINVAL
    # band offsets that place the band wholly outside the image (and whose
    # index arithmetic would overflow int) are refused before any launch
    for lo_r, lo_l in ((-(1 << 30), -1), (-1, 1 << 30), (17, -1), (-1, -33)):
        with pytest.raises(api.SfistaError) as ei:
            api.sfista_apply_static(x, y, 1, band, lo_r, band, lo_l)
        assert ei.value.status == api.EINVAL
    # the extremes of the accepted range run
    api.sfista_apply_static(x, y, 1, band, -32, band, 16)
    torch.cuda.synchronize()
    assert float(torch.count_nonzero(y)) == 0.0
