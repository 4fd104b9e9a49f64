"""Host check of the register FFT's 16-point butterflies: tests/host_dft16_check.cu
runs dft16 and the FMA-folded dft16_fma of csrc/fftreg.cuh on the CPU (the same
source the kernels compile) against the definition of the DFT, forward and
inverse, float and double. Bounds: a few units of rounding of the type (a
16-point DFT has two radix-4 stages and one twiddle multiplication per value)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_dft16_butterflies_match_the_dft(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "dft16_check")
    src = os.path.join(ROOT, "tests", "host_dft16_check.cu")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-O2", src, "-o", exe], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    err = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert len(err) == 8, out
    for k, e in err.items():
        bound = 4e-16 * 8 if "double" in k else 2.5e-7 * 8
        assert e < bound, (k, e)
    # the folded form is as accurate as the plain one
    for prec in ("double", "float"):
        for d in ("fwd", "inv"):
            assert err[f"dft16_fma_{prec}_{d}"] < 2 * err[f"dft16_{prec}_{d}"] + (1e-16 if prec == "double" else 1e-7)
