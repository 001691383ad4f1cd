"""Pins of the oracle's INT8 slice model (oracle.c section 6), on the CPU.

The model splits each operand, scaled per row (A) or column (B), into s
balanced base-256 digits of the w = 8s - 2 bit fixed-point value, so that
every digit is a signed byte; keeps the digit pairs of level t + u <= s + 1;
sums them exactly and rounds once.  Pinned against:
  - the exact rounding of v 2^(8s-2-e) (Python fractions), ties included;
  - digit reconstruction and the signed-byte ranges;
  - the fixed-point model (oracle.fixed_gemm) at s = 1, where no pair is
    dropped: the same product by a different route, bit for bit;
  - a brute-force statement in Python integers on small cases (the full
    product of the rounded operands minus the dropped pairs), bit for bit;
  - exactness on small-integer inputs (entries in {-8..8}).
The error bound of the model is pinned in test_guard_rule.py."""
import math
import random
from fractions import Fraction as Fr

import numpy as np

import oracle
import workload


def rne(x: Fr) -> int:
    f = math.floor(x)
    r = x - f
    if r > Fr(1, 2) or (r == Fr(1, 2) and f % 2 == 1):
        return f + 1
    return f


def e_of(v: float) -> int:
    return 0 if v == 0 else math.frexp(abs(v))[1]


def test_fixed_point_is_the_exact_rounding():
    rnd = random.Random(1)
    for _ in range(3000):
        s = rnd.randrange(1, 9)
        v = rnd.uniform(-1, 1) * 2.0 ** rnd.randrange(-40, 40)
        e = e_of(v) + rnd.choice((0, 0, 1, 5))
        assert oracle.i8_fixed(v, e, s) == rne(Fr(v) * Fr(2) ** (8 * s - 2 - e))
    for s in range(1, 9):  # exact ties at the last kept bit
        w = 8 * s - 2
        for k in (1, 3, 5, 1001):
            v = (k + 0.5) * 2.0 ** -w
            assert oracle.i8_fixed(v, 0, s) == rne(Fr(v) * Fr(2) ** w)


def test_digits_are_signed_bytes_and_reconstruct():
    rnd = random.Random(2)
    for s in range(1, 9):
        top = 1 << (8 * s - 2)
        cases = [0, 1, -1, top, -top, top - 1, 127, 128, -129] + [rnd.randrange(-top, top + 1) for _ in range(500)]
        for D in (x for x in cases if abs(x) <= top):
            d = oracle.i8_digits_of(D, s)
            assert sum(dt * 256 ** (s - 1 - t) for t, dt in enumerate(d)) == D
            assert -64 <= d[0] <= 64
            assert all(-128 <= x <= 127 for x in d[1:])


def test_one_digit_equals_the_fixed_point_product():
    for n, dist in ((1, "uniform11"), (17, "uniform11"), (40, "loguniform20"), (33, "uniform01")):
        A, B = workload.pair(dist, 5 + n, n)
        np.testing.assert_array_equal(oracle.i8_gemm(A, B, 1).view(np.int64),
                                      oracle.fixed_gemm(A, B, 6).view(np.int64))


def brute(A, B, s):
    m, k = A.shape
    n = B.shape[1]
    w = 8 * s - 2
    e = [e_of(max(abs(x) for x in A[i])) for i in range(m)]
    f = [e_of(max(abs(B[j, l]) for j in range(k))) for l in range(n)]
    DA = [[rne(Fr(float(A[i, j])) * Fr(2) ** (w - e[i])) for j in range(k)] for i in range(m)]
    DB = [[rne(Fr(float(B[j, l])) * Fr(2) ** (w - f[l])) for l in range(n)] for j in range(k)]
    dA = [[oracle.i8_digits_of(x, s) for x in row] for row in DA]
    dB = [[oracle.i8_digits_of(x, s) for x in row] for row in DB]
    C = np.empty((m, n))
    for i in range(m):
        for l in range(n):
            full = sum(DA[i][j] * DB[j][l] for j in range(k))
            dropped = sum(dA[i][j][t] * dB[j][l][u] * 256 ** (2 * s - (t + 1) - (u + 1))
                          for j in range(k) for t in range(s) for u in range(s) if t + u + 2 >= s + 2)
            X = full - dropped  # the kept pairs: sum_L S_L 256^(2s - L)
            assert X % 256 ** (s - 1) == 0
            C[i, l] = math.ldexp(float(X // 256 ** (s - 1)), e[i] + f[l] - 8 * s - 4)
    return C


def test_model_equals_brute_force_on_small_cases():
    rnd = np.random.default_rng(3)
    for (m, n, k) in ((1, 1, 1), (2, 3, 4), (5, 2, 7), (4, 4, 9)):
        for s in (1, 2, 3, 5, 8):
            A = rnd.uniform(-1, 1, (m, k)) * np.exp2(rnd.integers(-30, 30, (m, k)))
            B = rnd.uniform(-1, 1, (k, n)) * np.exp2(rnd.integers(-30, 30, (k, n)))
            np.testing.assert_array_equal(oracle.i8_gemm(A, B, s).view(np.int64), brute(A, B, s).view(np.int64))


def test_exact_on_small_integers():
    for n in (1, 7, 64, 129):
        A, B = workload.pair("int8", 9, n)
        want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
        for s in (1, 2, 7):
            np.testing.assert_array_equal(oracle.i8_gemm(A, B, s), want)
