"""The exact 128-by-64-bit floor division behind every integer threshold.

Built for the host from the library's own header (no GPU needed) and run on
random and edge-case inputs against unsigned __int128 division.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_floor_div_sat_matches_int128(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "div_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2504_09311_gb300", "csrc"), "-o", exe,
                    os.path.join(ROOT, "tests", "div_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe, "2000000"], check=True, capture_output=True, text=True).stdout
    assert "0 mismatches" in out, out
