"""The two-stage FFT passes' index maps and register FFT, checked on the host (no GPU): the programs
include the library's own header and run on the CPU (host code only, no kernel launch)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1506_03737_gb300", "csrc")


def build_and_run(src, exe):
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    cc = cand if os.path.exists(cand) else shutil.which("nvcc")
    if not cc:
        pytest.skip("nvcc not available")
    subprocess.run([cc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(HERE, src), "-o", str(exe)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_half_spectrum_index_maps(tmp_path):
    out = build_and_run("host_layout_check.cu", tmp_path / "layout_check")
    assert out.count("one-to-one") == 4


def test_register_fft_against_fp64_dft(tmp_path):
    """Stage A for every task, then stage B for every task (what the block barrier between them
    guarantees), with the header's DFT, twiddle tables and exchange-buffer indexing."""
    out = build_and_run("host_fft_check.cu", tmp_path / "fft_check")
    assert sum(line.startswith("radix ") for line in out.splitlines()) == 8
    assert out.count("rms rel error") == 8 + 3 * 10


def test_paired_lane_transforms_against_fp64_dft(tmp_path):
    """The 1024-point force z pass with each radix-32 task split over two lanes: both exchange forms
    (decimation in time and in frequency) and the whole tile chain, with the header's own code."""
    out = build_and_run("host_pair_check.cu", tmp_path / "pair_check")
    assert out.count("rms rel error") == 6
