"""Host check of the register FFT's shared-memory index maps and twiddle indices
(tests/host_layout_check.cu compiles the layouts of csrc/fftreg.cuh for the CPU):
for every power-of-two length 16..4096 and every exchange of the forward and
inverse transforms, the base-plus-constant addresses equal the layouts'
definitions at the Stockham positions, are distinct within an exchange, and the
split twiddle index equals r (j mod NS) L/(NS RAD)."""
import os
import subprocess

import pytest

from test_fft_butterflies import ROOT, _nvcc


def test_layouts_and_twiddle_indices(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "layout_check")
    src = os.path.join(ROOT, "tests", "host_layout_check.cu")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-O2", src, "-o", exe], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    counts = {k: int(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert set(counts) == {"positions", "addresses", "unique", "twiddles", "disjoint"}, out
    assert all(v == 0 for v in counts.values()), counts
