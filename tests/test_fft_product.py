"""The FFT structured product that bench.py times against the library's
operator forms (`--workload fft`): each 1-D factor applied as a correlation
of the zero- or reflectively extended line with the reversed profile (toep,
toep + hank of Sec. 2), by real FFTs.  Checked here on the CPU, in FP64,
against the oracle's operator, so the timed alternative computes the same
A_s as the forms it is compared with."""
import numpy as np
import pytest

import bench
import oracle
from oracle import kron
from paper_1901_00913_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("m,n,psf,centre,r", [(40, 36, (7, 9), (3, 4), 2), (33, 50, (11, 5), (2, 4), 3),
                                               (24, 24, (9, 9), (4, 4), 1)])
def test_fft_product_matches_oracle_operator(bc, m, n, psf, centre, r):
    g = W.rng(801 + m + n + bc)
    P = W.random_psf(g, *psf)
    ka = kron.kron_approx(P, centre[0], centre[1], m, n, bc, r)
    Y = g.standard_normal((m, n))
    out = bench.fft_kron_apply(torch, torch.from_numpy(Y), torch.from_numpy(ka.C), ka.cr, torch.from_numpy(ka.D),
                               ka.cc, bc).numpy()
    assert oracle.rel_fro(out, oracle.kron_apply(Y, ka)) <= 1e-12


def test_fft_lengths_are_smooth_and_long_enough():
    for L in (1, 2, 7, 95, 542, 2110, 4097):
        N = bench._fft_len(L)
        assert N >= L
        k = N
        for f in (2, 3, 5):
            while k % f == 0:
                k //= f
        assert k == 1
        assert N < 2 * L or L == 1
