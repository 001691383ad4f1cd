"""The modular form's constant tables, checked on the host against exact
integer arithmetic (tests/modular_tables_check.cpp): split constants, the
epilogue's divisions by the moduli, the epilogue's group residues recombined
by the Chinese remainder theorem for every moduli count, the recombination's
quotient estimate and 128-bit reconstruction at the width rule's extremes,
and the split's FP32 residue arithmetic replayed with IEEE fmaf over the whole
fixed-point range."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_include():
    for base in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        inc = os.path.join(base, "include")
        if base and os.path.exists(os.path.join(inc, "vector_types.h")):
            return inc
    return None


def test_modular_tables_against_exact_arithmetic(tmp_path):
    gxx = shutil.which("g++")
    inc = cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "modular_tables_check")
    src = os.path.join(ROOT, "tests", "modular_tables_check.cpp")
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", inc, "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().startswith("ok")
