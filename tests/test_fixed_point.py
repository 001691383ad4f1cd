"""The split's fixed-point conversion (fixed_point.cuh, used on the device by
both emulation forms), compiled for the host: D = round-half-even(v 2^(width -
e)) against the oracle's or_fix on exact ties at every shift, subnormal
inputs, values just below 2^e, widths 1..62 and both signs; the exponent of a
maximum (frexp's exponent) against Python's; the non-finite flag; and the
digit form's balanced base-256 digits against the oracle's at every digit
count, up to the largest fixed-point values."""
import math
import os
import random
import shutil
import struct
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_include():
    for base in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        inc = os.path.join(base, "include")
        if base and os.path.exists(os.path.join(inc, "vector_types.h")):
            return inc
    return None


def bits_of(v: float) -> int:
    return struct.unpack("<q", struct.pack("<d", v))[0]


def e_of(v: float) -> int:
    # smallest e with |v| < 2^e (frexp's exponent); 0 for 0
    return 0 if v == 0 else math.frexp(abs(v))[1]


def cases():
    rnd = random.Random(9)
    vals = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072009e-308, 2.2250738585072014e-308, 1.0, -1.0,
            0.5, 0.75, 1 - 2 ** -53, -(1 - 2 ** -53), 3 * 2 ** -56, 2 ** -60, 1e300, -1e-300, 123.456]
    for k in range(1, 64):  # exact ties: odd multiples of 2^-k, and their neighbours
        t = (2 * rnd.getrandbits(10) + 1) * 2.0 ** -k
        vals += [t, -t, math.nextafter(t, 0), math.nextafter(t, math.inf)]
    vals += [rnd.uniform(-1, 1) * 2.0 ** rnd.randrange(-1074, 1000) for _ in range(3000)]
    vals += [struct.unpack("<d", struct.pack("<q", rnd.getrandbits(52)))[0] for _ in range(300)]  # subnormals
    out = []
    for v in vals:
        e = e_of(v)
        for width in (1, 7, 15, 23, 31, 47, 55, 62) if rnd.random() < 0.2 else (rnd.randrange(1, 63),):
            for de in (0, 1, 30):  # e may exceed v's own exponent (a row maximum elsewhere)
                out.append((v, e + de, width))
    return out


def test_fixed_point_matches_the_oracle(tmp_path):
    gxx, inc = shutil.which("g++"), cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "fixed_point_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", inc, os.path.join(ROOT, "tests", "fixed_point_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    cs = cases()
    special = [(math.inf, 1, 40), (-math.inf, 1, 40), (math.nan, 1, 40)]
    maxima = [abs(v) for v, _, _ in cs[:400]]
    lines = [f"F {bits_of(v)} {e} {w}" for v, e, w in cs + special] + [f"F {bits_of(m)} 0 0" for m in maxima]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120, check=True)
    got = [tuple(int(x) for x in line.split()) for line in r.stdout.strip().splitlines()]
    assert len(got) == len(lines)
    bad = [(v, e, w, g) for (v, e, w), g in zip(cs, got) if g != (oracle.fix(v, e, w), 0)]
    assert not bad, bad[:5]
    assert all(g == (0, 1) for g in got[len(cs):len(cs) + 3])  # Inf, NaN: D = 0, flagged
    assert [g[0] for g in got[len(cs) + 3:]] == [e_of(m) for m in maxima]


def test_digits_match_the_oracle(tmp_path):
    gxx, inc = shutil.which("g++"), cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "fixed_point_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", inc, os.path.join(ROOT, "tests", "fixed_point_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    rnd = random.Random(13)
    cases = []
    for s in range(1, 9):
        top = 1 << (8 * s - 1)  # |D| <= 2^(8s-1), as the split's fixed point gives
        if s == 8:
            top -= 1 << 10  # s = 8: |x| <= 1 - 2^-53 keeps |D| <= 2^63 - 2^10
        vals = [0, 1, -1, top, -top, top - 1, -(top - 1), 127, 128, -128, -129, 255, 256]
        vals += [rnd.randrange(-top, top + 1) for _ in range(2000)]
        cases += [(d, s) for d in vals if -top <= d <= top]
    lines = [f"G {d} {s}" for d, s in cases]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=60, check=True)
    got = [[int(x) for x in line.split()] for line in r.stdout.strip().splitlines()]
    assert len(got) == len(cases)
    bad = [(d, s, g) for (d, s), g in zip(cases, got) if g != oracle.emu_digits_of(d, s)]
    assert not bad, bad[:5]


def test_magnitude_and_sign_form_matches_the_oracle(tmp_path):
    # fixed_point_sm (the modular split's form: |D| with v's sign bit in bit
    # 63) on the same cases: |D| is |or_fix|, the sign bit is v's, widths up
    # to 62 leave bit 63 free; the non-finite flag as before.
    gxx, inc = shutil.which("g++"), cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "fixed_point_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", inc, os.path.join(ROOT, "tests", "fixed_point_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    cs = cases()
    lines = [f"S {bits_of(v)} {e} {w}" for v, e, w in cs] + [f"S {bits_of(v)} 1 40" for v in (math.inf, -math.nan)]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120, check=True)
    got = [tuple(int(x) for x in line.split()) for line in r.stdout.strip().splitlines()]
    assert len(got) == len(lines)
    bad = [(v, e, w, g) for (v, e, w), g in zip(cs, got)
           if g != (abs(oracle.fix(v, e, w)), 1 if math.copysign(1.0, v) < 0 else 0, 0)]
    assert not bad, bad[:5]
    assert all(g[0] < 2 ** 63 for g in got)
    assert got[-2] == (0, 0, 1) and got[-1][0] == 0 and got[-1][2] == 1
