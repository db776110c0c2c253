"""Arithmetic helpers of the particle passes run as host code: the compensated FP32 polar
factors, and the fixed-point conversions of the deterministic grid sums.

`polar_refine2` / `polar_refine3` (csrc/mpm_common.cuh) are host-and-device functions; here
nvcc compiles them into a host program (tests/host/polar_refine_check.cu) that compares them
with an extended-precision (long double) polar decomposition on random F = R S (random and
small rotations, strains 1e-6 to 0.6).  Bars: R within 1e-13 (FP64-level; the FP32 forms reach
~6e-14), and F - R within 5e-7 relative to the case's largest |F - R| (one FP32 rounding, or
the R error at the smallest strains).  No GPU is needed.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_compensated_polar_factors_match_extended_precision(tmp_path):
    cc = _nvcc()
    if cc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "polar_refine_check")
    src = os.path.join(HERE, "host", "polar_refine_check.cu")
    subprocess.run([cc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-o", exe, src],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    res = {}
    for line in out.strip().splitlines():
        dim, n, fails, err_r, err_d = line.split()
        res[dim] = (int(n), int(fails), float(err_r), float(err_d))
    n3, f3, r3, d3 = res["3d"]
    assert f3 == 0 and r3 <= 1e-13 and d3 <= 5e-7, res
    n2, f2, r2, d2 = res["2d"]
    assert f2 == 0 and r2 <= 1e-13 and d2 <= 5e-7, res


def test_fixed_point_conversions_match_the_c_library(tmp_path):
    """fix_round (float -> nearest int64) and ll_to_float_rn (int64 -> nearest float) of the
    deterministic grid sums, built as host code, agree with llrintf and the C cast on random
    and halfway inputs (they replace conversions that issue on the GPU's FP64 pipe)."""
    cc = _nvcc()
    if cc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "fixed_point_check")
    src = os.path.join(HERE, "host", "fixed_point_check.cu")
    subprocess.run([cc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-o", exe, src],
                   check=True, capture_output=True, timeout=300)
    n, bad_round, bad_float = map(int, subprocess.run([exe], check=True, capture_output=True,
                                                      text=True, timeout=300).stdout.split())
    assert n > 0 and bad_round == 0 and bad_float == 0, (n, bad_round, bad_float)
