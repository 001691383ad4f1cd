"""The digit shortcut used by the split kernel, checked against the oracle's definition.

The oracle defines the digits of D bottom-up (balanced residues mod 256).  The
kernel instead adds M = sum 128 * 256^k over the s-1 lower positions and reads
plain bytes; this test shows the two agree on edge cases and random values.
"""
import random

import oracle


def byte_digits(D, s):
    """The kernel's arithmetic, with its 64-bit wrap-around made explicit."""
    sh = 8 * (s - 1)
    M = sum(128 * 256 ** k for k in range(s - 1))
    u = D & (2 ** 64 - 1)                         # D as the kernel's uint64
    low = (u & (2 ** sh - 1)) + M                 # < 2^(sh+1): no overflow
    assert low < 2 ** 64
    out = [0] * s
    for t in range(s - 1, 0, -1):
        out[t] = ((low >> (8 * (s - 1 - t))) & 255) - 128
    top = D >> sh                                 # int64 arithmetic shift of D
    assert -2 ** 31 <= top < 2 ** 31
    out[0] = top + (low >> sh)
    return out


def test_byte_extraction_equals_balanced_digits():
    rng = random.Random(1)
    for s in range(1, 9):
        lim = min(2 ** (8 * s - 1), 2 ** 63 - 2 ** 10)
        cases = [0, 1, -1, 127, 128, -128, 255, -255, 256, lim, -lim, lim - 1]
        cases += [rng.randint(-lim, lim) for _ in range(2000)]
        for D in cases:
            if abs(D) > lim:
                continue
            assert byte_digits(D, s) == oracle.emu_digits_of(D, s), (s, D)
