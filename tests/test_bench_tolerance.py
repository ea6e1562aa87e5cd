"""bench.py's meets_tol flag: FP32 is held to 1e-5 relative Frobenius error,
the split-precision forms to 1e-4 and 0.01 dB PSNR, and the single-product
BF16 / TF32 forms, which have no stated tolerance, report None (never True).
CPU only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fp32_tolerance():
    assert bench.meets_tol("fp32", 4.6e-7, -3e-7) is True
    assert bench.meets_tol("fp32", 2e-5, 0.0) is False


def test_split_forms_need_error_and_psnr():
    assert bench.meets_tol("bf16x3", 2.1e-5, -3.3e-4) is True
    assert bench.meets_tol("tf32x3", 1.9e-6, 0.02) is False      # PSNR off by more than 0.01 dB
    assert bench.meets_tol("bf16x3", 2e-4, 0.0) is False
    assert bench.meets_tol("bf16x3", 1e-5, None) is False


def test_single_product_forms_have_no_tolerance():
    # BF16 at 1.1e-2 and TF32 at 1.7e-3 are reported, not held: never True.
    assert bench.meets_tol("bf16", 1.1e-2, -3e-3) is None
    assert bench.meets_tol("tf32", 1.7e-3, -4e-4) is None
    assert bench.meets_tol("bf16", 1e-9, 0.0) is None
