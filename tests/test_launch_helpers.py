"""The work-splitting helpers shared by the host planner and the kernels
(launch.cuh), compiled for the host and checked exhaustively over small
parameters (tests/launch_helpers_check.cpp): the tile order is a bijection,
digit pairs are numbered level by level, groups and segments partition the
pairs, and modular unit ranges cut the moduli at residue-pair boundaries."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_helpers(tmp_path):
    # nvcc compiles the header's device-only parts; only host code runs
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("needs nvcc")
    exe = str(tmp_path / "launch_helpers_check")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "launch_helpers_check.cpp"),
                    "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
