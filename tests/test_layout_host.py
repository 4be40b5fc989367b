"""The half-spectrum index maps of the two-stage FFT passes, checked on the host (no GPU): the
program includes the library's own header and runs on the CPU (host code only, no kernel launch)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1506_03737_gb300", "csrc")


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_half_spectrum_index_maps(tmp_path):
    exe = tmp_path / "layout_check"
    cc = nvcc()
    if not cc:
        pytest.skip("nvcc not available")
    subprocess.run([cc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(HERE, "host_layout_check.cu"), "-o", str(exe)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("one-to-one") == 4
