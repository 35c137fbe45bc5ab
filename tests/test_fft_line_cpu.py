"""The line transforms of the CUDA path (csrc/fft_line.cuh) checked on the host: every grid
size the library instantiates, FP64 and FP32, inverse and forward, against the direct DFT sum
in long double; the pruned transform (known-zero inputs outside |m| <= N/4) against the full
one.  Bars: FP64 5e-16 and FP32 3e-7 relative (a few units of roundoff; the measured
worst cases are 1.9e-16 and 1.3e-7)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIZES = {12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48}


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_line_check")
    src = os.path.join(ROOT, "tests", "host", "fft_line_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-O2", src, "-o", exe], check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    rows = {}
    for line in out.splitlines():
        f = line.split()
        if f and f[0] == "N":
            rows[int(f[1])] = [float(v) for v in f[2:]]
    return rows


def test_every_instantiated_size_is_checked(results):
    assert set(results) == SIZES


def test_line_transforms_match_the_direct_sum(results):
    for n, r in results.items():
        assert max(r[0], r[1]) <= 5e-16, (n, r[:2])
        assert max(r[2], r[3]) <= 3e-7, (n, r[2:4])


def test_pruned_transforms_match_the_full_ones(results):
    for n, r in results.items():
        assert max(r[4], r[5]) <= 5e-16, (n, r[4:6])
        assert max(r[6], r[7]) <= 3e-7, (n, r[6:8])
