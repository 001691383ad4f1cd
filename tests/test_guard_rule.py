"""The accuracy certificate of the emulated forms, as mathematics, pinned
against exact rational arithmetic on the oracle's models of both forms.

The product is Alg. 1's c_ik = sum_j a_ij b_jk (Sec. 3.1).  For every element
of the modular model (oracle.fixed_gemm, width beta), of the digit model
(oracle.emu_gemm, s digits, width 8s - 1) and of the INT8 slice model
(oracle.i8_gemm, s digits, width 8s - 2) this checks
  (1) |c^ - c| <= 2^(e_i + f_k) (u (R + E') + E'),
      E' = 2^(-w-1) (SA_i + SB_k) + n 2^(-2w-2) + n kappa   (kappa = 0 for the modular form),
  (2) wherever (1 + u) E' <= (n - 1) u R, |c^ - c| <= n u (|A||B|)_ik,
with R = sum_j |a'||b'|, a' = a 2^-e_i, b' = b 2^-f_k, exactly, on random
inputs, on inputs spanning wide exponent ranges, and on inputs built so that
every rounding error and every dropped digit pair points the same way (where
(1) is nearly attained: a bound with a term missing, or half as large, fails).
The kernels evaluate the same rule with a lower bound of R (the magnitude
plane) and upper bounds of SA, SB; guard.cuh's arithmetic is checked in
test_guard.py."""
import math
import random
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

U = Fr(1, 2 ** 53)


def kappa(s: int, w: int) -> Fr:
    return sum((Fr(2 * s + 1 - L) * Fr(2) ** (14 + 16 * s - 8 * L - 2 * w) for L in range(s + 2, 2 * s + 1)), Fr(0))


def e_of(v: float) -> int:
    return 0 if v == 0 else math.frexp(abs(v))[1]


def check(A, B, w, kap, model):
    """Asserts (1) and (2) for every element; returns (max ratio of the error
    to the bound of (1), number of certified elements)."""
    n = A.shape[0]
    e = [e_of(max(abs(x) for x in A[i])) for i in range(n)]
    f = [e_of(max(abs(x) for x in B[:, k])) for k in range(n)]
    Ap = [[Fr(float(A[i, j])) / Fr(2) ** e[i] for j in range(n)] for i in range(n)]
    Bp = [[Fr(float(B[j, k])) / Fr(2) ** f[k] for k in range(n)] for j in range(n)]
    SA = [sum(abs(x) for x in row) for row in Ap]
    SB = [sum(abs(Bp[j][k]) for j in range(n)) for k in range(n)]
    worst, certified = Fr(0), 0
    for i in range(n):
        for k in range(n):
            c = sum(Ap[i][j] * Bp[j][k] for j in range(n))
            R = sum(abs(Ap[i][j] * Bp[j][k]) for j in range(n))
            Ep = Fr(1, 2 ** (w + 1)) * (SA[i] + SB[k]) + n * Fr(1, 2 ** (2 * w + 2)) + n * kap
            got = Fr(float(model[i, k])) / Fr(2) ** (e[i] + f[k])
            err = abs(got - c)
            bound1 = U * (R + Ep) + Ep
            assert err <= bound1, (i, k, float(err), float(bound1))
            if bound1 > 0:
                worst = max(worst, err / bound1)
            if (1 + U) * Ep <= (n - 1) * U * R:
                certified += 1
                assert err <= n * U * R, (i, k)
    return float(worst), certified


def random_pair(rnd, n, kind):
    if kind == "uniform":
        A = np.array([[rnd.uniform(-1, 1) for _ in range(n)] for _ in range(n)])
        B = np.array([[rnd.uniform(-1, 1) for _ in range(n)] for _ in range(n)])
    elif kind == "wide":  # magnitudes over 2^-60 .. 2^60 within every row and column
        A = np.array([[rnd.choice((-1, 1)) * 2.0 ** rnd.uniform(-60, 60) for _ in range(n)] for _ in range(n)])
        B = np.array([[rnd.choice((-1, 1)) * 2.0 ** rnd.uniform(-60, 60) for _ in range(n)] for _ in range(n)])
    else:  # one large entry per row of A meets small entries of B, and the mirror
        A = np.full((n, n), 2.0 ** -30)
        A[:, 0] = 1.0
        B = np.ones((n, n))
        B[0, :] = 2.0 ** -30
        A *= np.array([[rnd.uniform(0.5, 1) for _ in range(n)] for _ in range(n)])
        B *= np.array([[rnd.uniform(0.5, 1) for _ in range(n)] for _ in range(n)])
    return A, B


def coherent_pair(rnd, n, w, digits_s=0):
    """Entries x' = (D + 0.499...) 2^-w with D chosen so that every row and
    column maximum is just below a power of two (e = 0): every fixed-point
    rounding error is close to -1/2, and for a digit form every low digit is
    127, so the dropped pairs all add with the same sign."""
    top = (1 << w) - 2
    hi = 1 << (w - 8 * (digits_s - 1)) if digits_s else 0  # the leading digit is below this
    def entry():
        if digits_s:
            D = sum(127 << (8 * t) for t in range(digits_s - 1)) + (rnd.randrange(hi // 2, hi - 1) << (8 * (digits_s - 1)))
        else:
            D = rnd.randrange(top // 2, top)
        return (D + 0.499) / 2.0 ** w
    A = np.array([[entry() for _ in range(n)] for _ in range(n)])
    B = np.array([[entry() for _ in range(n)] for _ in range(n)])
    return A, B


@pytest.mark.parametrize("kind", ["uniform", "wide", "split_scales"])
def test_modular_model_obeys_the_bound(kind):
    rnd = random.Random(hash(kind) & 0xFFFF)
    for n in (1, 2, 5, 12):
        A, B = random_pair(rnd, n, kind)
        for w in (8, 20, 40, 52):
            model = oracle.fixed_gemm(A, B, w, nthreads=1)
            check(A, B, w, Fr(0), model)


@pytest.mark.parametrize("kind", ["uniform", "wide", "split_scales"])
def test_digit_model_obeys_the_bound(kind):
    rnd = random.Random(7 + (hash(kind) & 0xFFFF))
    for n in (1, 3, 9):
        A, B = random_pair(rnd, n, kind)
        for s in (1, 2, 4, 7):
            model = oracle.emu_gemm(A, B, s, nthreads=1)
            check(A, B, 8 * s - 1, kappa(s, 8 * s - 1), model)


@pytest.mark.parametrize("kind", ["uniform", "wide", "split_scales"])
def test_int8_slice_model_obeys_the_bound(kind):
    rnd = random.Random(17 + (hash(kind) & 0xFFFF))
    for n in (1, 3, 9):
        A, B = random_pair(rnd, n, kind)
        for s in (1, 2, 4, 7):
            check(A, B, 8 * s - 2, kappa(s, 8 * s - 2), oracle.i8_gemm(A, B, s, nthreads=1))


def test_bound_is_nearly_attained_by_coherent_rounding():
    rnd = random.Random(11)
    n, w = 8, 20
    A, B = coherent_pair(rnd, n, w)
    worst, _ = check(A, B, w, Fr(0), oracle.fixed_gemm(A, B, w, nthreads=1))
    assert worst > 0.9  # halving the rounding term would be violated
    s = 2
    A, B = coherent_pair(rnd, n, 8 * s - 1, digits_s=s)
    worst, _ = check(A, B, 8 * s - 1, kappa(s, 8 * s - 1), oracle.emu_gemm(A, B, s, nthreads=1))
    assert worst > 0.5  # the dropped pairs (kappa) carry most of it
    A, B = coherent_pair(rnd, n, 8 * s - 2, digits_s=s)
    worst, _ = check(A, B, 8 * s - 2, kappa(s, 8 * s - 2), oracle.i8_gemm(A, B, s, nthreads=1))
    assert worst > 0.5


def test_certificate_holds_for_typical_inputs_and_fails_for_split_scales():
    rnd = random.Random(5)
    n = 16
    A, B = random_pair(rnd, n, "uniform")
    _, cert = check(A, B, 52, Fr(0), oracle.fixed_gemm(A, B, 52, nthreads=1))
    assert cert == n * n
    A, B = random_pair(rnd, n, "split_scales")
    _, cert = check(A, B, 40, Fr(0), oracle.fixed_gemm(A, B, 40, nthreads=1))
    assert cert < n * n
