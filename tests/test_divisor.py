"""The device code's division by a small integer (Granlund-Montgomery
invariant-divisor method) against plain integer division, on the host."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_invariant_division_exhaustive_divisors(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "divisor_check"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-o", str(exe),
                           os.path.join(HERE, "native", "divisor_check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("OK")
