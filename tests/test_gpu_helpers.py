"""The stage kernels' arithmetic helpers against the hardware's IEEE
operations (tests/cuda/helpers_check.cu, built here with nvcc):

* the FP64 reciprocal, reciprocal square root and square root (approximate
  seed + one third-order step): relative error at most 2^-50 (a few ulp) over
  exponents 2^-300..2^300, and the IEEE result on zero, subnormal, infinite
  and NaN inputs;
* the integer FP32<->FP64 conversions: bit-identical to the hardware
  conversions on every binary32 input and on 2^31 binary64 samples that
  include every rounding tie and exponent edge;
* the FP64 comparisons on the integer pipes (min, max, <, <=, sign tests,
  abs): identical to the IEEE ones on 2^28 random non-NaN pairs with zeros,
  subnormals, infinities and ties mixed in."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_arithmetic_helpers(tmp_path):
    exe = str(tmp_path / "helpers_check")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-I", os.path.join(ROOT, "paper_2606_12753_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                           "-o", exe, os.path.join(HERE, "cuda", "helpers_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["rcp_max_rel"] <= 2.0 ** -50, r
    assert r["rsqrt_max_rel"] <= 2.0 ** -50, r
    assert r["sqrt_max_rel"] <= 2.0 ** -50, r
    assert r["special_mismatch"] == 0, r
    assert r["widen_mismatch"] == 0, r
    assert r["narrow_mismatch"] == 0, r
    assert r["compare_mismatch"] == 0, r
