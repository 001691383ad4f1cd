"""The recombinations' 128-bit helpers (recombine.cuh), compiled for the host.
The final rounding (round_i128_scaled):
one round-to-nearest-even of a two's-complement 128-bit integer to FP64, then
the power-of-two scaling, compiled for the host and compared bit for bit with
the oracle's model of the same step (or_int128_to_double, the C conversion of
a 128-bit integer, then ldexp) on ties, carries into the next binade, every
bit length, signs, and results that overflow, land in the subnormal range or
underflow to zero.  The digit form's level combination (i128_shift_add and
its 64-bit variant: T = T 2^shift + v, two's complement modulo 2^128) against
Python integers for random level sequences."""
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


def cases():
    rnd = random.Random(5)
    vals = [0, 1, -1, 2 ** 53, 2 ** 53 + 1, 2 ** 53 + 2, 2 ** 53 + 3, -(2 ** 53 + 1), 2 ** 54 + 2, 2 ** 54 + 6,
            2 ** 127 - 1, -(2 ** 127), 2 ** 64, 2 ** 64 - 1, 2 ** 63, 3 * 2 ** 70 + 2 ** 17]
    for b in range(1, 128):  # every bit length, with ties and near-ties below the 53rd bit
        top = 1 << (b - 1)
        vals += [top, top + rnd.getrandbits(b - 1), -(top + rnd.getrandbits(b - 1))]
        if b > 54:
            half = 1 << (b - 54)
            base = top | (rnd.getrandbits(53) << (b - 53)) & ((1 << (b - 1)) - 1)
            base &= ~((1 << (b - 53)) - 1)
            vals += [base + half, base + half + 1, base + half - 1, -(base + half),
                     (top | ((1 << (b - 1)) - (1 << (b - 54))))]  # rounds up into the next binade
    out = []
    for v in vals:
        for scale in (0, -60, -200, 900, -1000, -1070, -1100, -1130, -1180, 1000, 960, -1022 - 100):
            out.append((v, scale))
    for _ in range(3000):
        b = rnd.randrange(1, 127)
        v = rnd.getrandbits(b) * (1 if rnd.random() < 0.5 else -1)
        out.append((v, rnd.randrange(-1250, 1000)))
    return out


def test_round_i128_scaled_matches_the_oracle(tmp_path):
    gxx, inc = shutil.which("g++"), cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "round_i128_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", inc, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "round_i128_check.cpp"), "-o", exe], check=True, capture_output=True,
                   text=True)
    cs = cases()
    lines = []
    for v, scale in cs:
        u = v & ((1 << 128) - 1)
        hi = u >> 64
        hi = hi - (1 << 64) if hi >= 1 << 63 else hi
        lines.append(f"R {hi} {u & ((1 << 64) - 1)} {scale}")
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120, check=True)
    got = [int(x) for x in r.stdout.split()]
    assert len(got) == len(cs)
    bad = []
    for (v, scale), g in zip(cs, got):
        try:
            want = math.ldexp(oracle.int128_to_double(v), scale)
        except OverflowError:
            want = math.copysign(math.inf, v)
        wbits = struct.unpack("<q", struct.pack("<d", want))[0]
        if g != wbits:
            bad.append((v, scale, g, wbits))
    assert not bad, bad[:5]


def test_shift_add_matches_python_integers(tmp_path):
    gxx, inc = shutil.which("g++"), cuda_include()
    if not gxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "round_i128_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", inc, os.path.join(ROOT, "tests", "round_i128_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    rnd = random.Random(11)
    seqs = []
    for t in range(3000):
        wide = t % 2 == 1
        count = rnd.randrange(1, 9)
        seq = []
        for i in range(count):
            shift = 0 if i == 0 else 8 * rnd.randrange(0, 8)  # level gaps of 0..7 bytes
            bound = 1 << (62 if wide else 31)
            v = rnd.choice([rnd.randrange(-bound, bound), bound - 1, -bound, 0, -1])
            seq.append((shift, v))
        seqs.append(("B" if wide else "A", seq))
    lines = [f"{op} {len(seq)} " + " ".join(f"{sh} {v}" for sh, v in seq) for op, seq in seqs]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=60, check=True)
    got = [tuple(int(x) for x in line.split()) for line in r.stdout.strip().splitlines()]
    assert len(got) == len(seqs)
    for (op, seq), (hi, lo) in zip(seqs, got):
        T = 0
        for sh, v in seq:
            T = (T << sh) + v
        T &= (1 << 128) - 1
        assert ((hi & ((1 << 64) - 1)) << 64) | lo == T, (op, seq)
