"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: the paper's printed tables, a
closed form, an exact rational computation, a textbook example or a
mathematical invariant.  A dropped term, a wrong index or a transposed
operand in oracle.c fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def exact_product(A, B):
    """Exact rational product of two float matrices (Python fractions)."""
    n = A.shape[0]
    FA = [[Fraction(float(x)) for x in row] for row in A]
    FB = [[Fraction(float(x)) for x in row] for row in B]
    return [[sum((FA[i][j] * FB[j][k] for j in range(n)), Fraction(0)) for k in range(n)]
            for i in range(n)]


# ---- the paper's metric (Sec. 3.1, Alg. 2, Tables 1-3) -----------------------

def test_flop_count_closed_form():
    # N^2 (2N - 1) operations (Sec. 3.1); e.g. N = 100 -> 1,990,000.
    assert workload.flops(100) == 1_990_000
    for n in (1, 2, 10, 2000):
        assert workload.flops(n) == n * n * (2 * n - 1)


def test_paper_tables_are_consistent_with_the_metric():
    g = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))
    Ns = g["N"]
    for prog in ("sequential", "openmp", "mpi"):
        for idx, n in enumerate(Ns):
            t = g["table1_runtime_s"][prog][idx]
            mflops = g["table2_mflops"][prog][idx]
            rate = workload.flops(n) / t / 1e6
            if n == 100 or (n == 2000 and prog in ("sequential", "openmp")):
                continue  # 1-2 significant digits, or the two inconsistent cells
            assert abs(rate - mflops) / mflops < 0.01, (prog, n, rate, mflops)
    # The two flagged cells really are inconsistent (8.91 vs about 66.4).
    assert workload.flops(2000) / 240.97 / 1e6 == pytest.approx(66.38, rel=1e-3)
    # Speedup = t_seq / t_par (Table 3).
    for prog in ("openmp", "mpi"):
        for idx, n in enumerate(Ns):
            sp = g["table1_runtime_s"]["sequential"][idx] / g["table1_runtime_s"][prog][idx]
            assert abs(sp - g["table3_speedup"][prog][idx]) < 0.051, (prog, n, sp)


# ---- the product (Alg. 1, 3, 4) -----------------------------------------------

def test_textbook_2x2():
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    B = np.array([[5.0, 6.0], [7.0, 8.0]])
    np.testing.assert_array_equal(oracle.gemm(A, B), [[19.0, 22.0], [43.0, 50.0]])
    np.testing.assert_array_equal(oracle.gemm_alg1(A, B), [[19.0, 22.0], [43.0, 50.0]])


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_tiny_sizes_by_brute_force_enumeration(n):
    # Entries that are small powers of two times small odd integers make every
    # partial sum exact, so the result must equal the exact rational product.
    rng = np.random.default_rng(100 + n)
    A = rng.integers(-9, 10, (n, n)) * 2.0 ** rng.integers(-3, 4, (n, n))
    B = rng.integers(-9, 10, (n, n)) * 2.0 ** rng.integers(-3, 4, (n, n))
    ex = exact_product(A, B)
    C = oracle.gemm(A, B)
    for i in range(n):
        for k in range(n):
            assert Fraction(float(C[i, k])) == ex[i][k]


def test_identity_and_permutation_are_exact():
    n = 37
    A, B = workload.pair("uniform01", 3, n)
    I = np.eye(n)
    np.testing.assert_array_equal(oracle.gemm(I, B), B)
    np.testing.assert_array_equal(oracle.gemm(A, I), A)
    perm = np.random.default_rng(1).permutation(n)
    P = np.eye(n)[perm]  # row i of P selects row perm[i]
    np.testing.assert_array_equal(oracle.gemm(P, B), B[perm])
    np.testing.assert_array_equal(oracle.gemm(A, P.T), A[:, perm])


@pytest.mark.parametrize("n", [1, 7, 64, 129])
def test_all_ones_gives_n(n):
    J = np.ones((n, n))
    np.testing.assert_array_equal(oracle.gemm(J, J), np.full((n, n), float(n)))


@pytest.mark.parametrize("n", [5, 33, 100])
def test_small_integers_are_exact(n):
    # Entries in {-8..8}: every partial sum is an integer below 2^53, so any
    # summation order gives the exact integer product (numpy int64 matmul).
    A, B = workload.pair("int8", 7, n)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(oracle.gemm(A, B), ref)
    np.testing.assert_array_equal(oracle.gemm_alg1(A, B), ref)
    # (AB)^T = B^T A^T exactly for integer inputs: catches a transposed operand.
    np.testing.assert_array_equal(oracle.gemm(B.T.copy(), A.T.copy()), ref.T)
    np.testing.assert_array_equal(oracle.absgemm(A, B),
                                  (np.abs(A).astype(np.int64) @ np.abs(B).astype(np.int64)))


def test_loop_order_and_thread_count_do_not_change_bits():
    n = 150
    A, B = workload.pair("uniform11", 11, n)
    ref = oracle.gemm_alg1(A, B)
    for t in (1, 2, 3, 8):
        np.testing.assert_array_equal(oracle.gemm(A, B, nthreads=t), ref)
    rows = [0, 5, 149, 77]
    np.testing.assert_array_equal(oracle.gemm_rows(A, B, rows), ref[rows])


@pytest.mark.parametrize("dist", ["uniform01", "uniform11", "loguniform20"])
def test_within_recursive_summation_bound_of_exact(dist):
    # Higham, Accuracy and Stability, Sec. 3.1: |fl(x.y) - x.y| <= gamma_n |x|.|y|.
    n = 9
    A, B = workload.pair(dist, 21, n)
    ex = exact_product(A, B)
    C = oracle.gemm(A, B)
    absAB = np.abs(A) @ np.abs(B)
    gamma = n * U / (1 - n * U)
    worst = 0.0
    for i in range(n):
        for k in range(n):
            err = abs(Fraction(float(C[i, k])) - ex[i][k])
            assert err <= Fraction(gamma) * Fraction(float(absAB[i, k])) * (1 + 1e-12)
            worst = max(worst, float(err))
    assert worst > 0.0  # rounding did occur, so the bound was exercised


def test_dot2_is_nearly_exact():
    # Ogita-Rump-Oishi: |res - x.y| <= u |x.y| + gamma_n^2 |x|.|y|.
    n = 12
    A, B = workload.pair("loguniform20", 5, n)
    ex = exact_product(A, B)
    D = oracle.gemm_dot2(A, B)
    absAB = np.abs(A) @ np.abs(B)
    gamma = n * U / (1 - n * U)
    for i in range(n):
        for k in range(n):
            bound = Fraction(U) * abs(ex[i][k]) + Fraction(gamma * gamma) * Fraction(float(absAB[i, k])) * 2
            assert abs(Fraction(float(D[i, k])) - ex[i][k]) <= bound


def test_freivalds_accepts_exact_and_rejects_planted_errors():
    n = 80
    A, B = workload.pair("uniform11", 2, n)
    C = oracle.gemm(A, B)
    rng = np.random.default_rng(0)
    for _ in range(4):
        x = rng.choice([-1.0, 1.0], n)
        bad, _, _ = oracle.freivalds(A, B, C, x)
        assert bad == 0
    # A single wrong entry far above the rounding level is caught by +-1 probes.
    Cw = C.copy()
    Cw[17, 33] += 1e-6
    caught = 0
    for _ in range(8):
        x = rng.choice([-1.0, 1.0], n)
        bad, _, _ = oracle.freivalds(A, B, Cw, x)
        caught += bad > 0
    assert caught == 8  # with +-1 probes a single-entry error is never cancelled
    # The transposed product is rejected.
    bad, _, _ = oracle.freivalds(A, B, oracle.gemm(B, A), rng.choice([-1.0, 1.0], n))
    assert bad > 0


# ---- model of the split-precision emulation -----------------------------------

def test_row_and_column_exponents_bracket_the_maximum():
    n = 50
    A = workload.matrix("loguniform20", 4, n)
    A[3] = 0.0
    e = oracle.emu_row_exponents(A)
    f = oracle.emu_col_exponents(A)
    for i in range(n):
        m = np.abs(A[i]).max()
        if m == 0:
            assert e[i] == 0
        else:
            assert m < 2.0 ** e[i] and m >= 2.0 ** (e[i] - 1)
    for k in range(n):
        m = np.abs(A[:, k]).max()
        assert m < 2.0 ** f[k] and m >= 2.0 ** (f[k] - 1)


def test_fixed_point_value_is_the_exact_rounding():
    rng = np.random.default_rng(9)
    vals = list(workload.values("loguniform20", 1, 200)) + [0.0, -0.0, 1 - 2 ** -53, -(1 - 2 ** -53),
                                                             0.5, 2 ** -60, 3 * 2 ** -56]
    for s in (1, 2, 5, 7, 8):
        for v in vals:
            e = 1 if abs(v) < 1 else math.frexp(abs(v))[1]
            if abs(v) >= 2.0 ** e:
                continue
            exact = Fraction(float(v)) * Fraction(2) ** (8 * s - 1 - e)
            assert oracle.emu_fixed(v, e, s) == round(exact)  # round() on Fraction: half to even
    # Ties go to even.
    assert oracle.emu_fixed(3 * 2.0 ** -8, 0, 1) == 2  # 1.5 -> 2
    assert oracle.emu_fixed(5 * 2.0 ** -8, 0, 1) == 2  # 2.5 -> 2
    assert oracle.emu_fixed(-5 * 2.0 ** -8, 0, 1) == -2
    _ = rng


def test_digits_reconstruct_and_respect_ranges():
    rng = np.random.default_rng(3)
    for s in range(1, 9):
        top = 2 ** (8 * s - 1)
        cases = [0, 1, -1, 127, 128, -128, 255, top, -top, top - 1, -(top - 1)]
        cases += [int(x) for x in rng.integers(-top if s < 8 else -(2 ** 62), top if s < 8 else 2 ** 62, 50)]
        for D in cases:
            if abs(D) > min(top, 2 ** 63 - 2 ** 10):
                continue  # |D| <= 2^(8s-1), and <= 2^63 - 2^10 at s = 8 since |x| <= 1 - 2^-53
            d = oracle.emu_digits_of(D, s)
            assert sum(dt * 256 ** (s - 1 - t) for t, dt in enumerate(d)) == D
            assert all(-128 <= x <= 127 for x in d[1:])
            assert -128 <= d[0] <= 128


@pytest.mark.parametrize("s", [1, 2, 3])
def test_level_sums_by_brute_force(s):
    n = 6
    A, B = workload.pair("uniform11", 8, n)
    e = oracle.emu_row_exponents(A)
    f = oracle.emu_col_exponents(B)
    dA = oracle.emu_digit_planes(A, e, s, False)
    dB = oracle.emu_digit_planes(B, f, s, True)
    # digits taken one value at a time agree with the planes
    for i in range(n):
        for j in range(n):
            assert list(dA[:, i, j]) == oracle.emu_digits_of(oracle.emu_fixed(A[i, j], e[i], s), s)
            assert list(dB[:, i, j]) == oracle.emu_digits_of(oracle.emu_fixed(B[i, j], f[j], s), s)
    S = oracle.emu_level_sums(dA, dB)
    for i in range(n):
        for k in range(n):
            for L in range(2, s + 2):
                want = sum(int(dA[t - 1, i, j]) * int(dB[L - t - 1, j, k])
                           for j in range(n) for t in range(1, s + 1) if 1 <= L - t <= s)
                assert S[L - 2, i, k] == want


def test_int128_rounding_matches_exact_conversion():
    rng = np.random.default_rng(12)
    cases = [0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 53 + 1), 2 ** 95 + 2 ** 42, 2 ** 95 + 2 ** 42 + 1,
             (2 ** 54 + 2) * 2 ** 30, (2 ** 54 + 6) * 2 ** 30, 2 ** 126 - 1]
    for _ in range(300):
        bits = int(rng.integers(1, 126))
        cases.append(int(rng.integers(0, 2 ** 62)) << max(0, bits - 62) | int(rng.integers(0, 2 ** 31)))
        cases.append(-cases[-1])
    for T in cases:
        assert oracle.int128_to_double(T) == float(T), T  # Python int -> float rounds half to even


def test_combine_is_the_rounded_exact_sum():
    rng = np.random.default_rng(5)
    for s in (1, 4, 8):
        for _ in range(50):
            lv = [int(x) for x in rng.integers(-2 ** 31, 2 ** 31, s)]
            e, f = int(rng.integers(-20, 21)), int(rng.integers(-20, 21))
            T = sum(S * 256 ** (s + 1 - L) for L, S in zip(range(2, s + 2), lv))
            want = float(Fraction(T) * Fraction(2) ** (e + f - 8 * s - 6))
            # float(Fraction) is correctly rounded; here T fits the exponent range,
            # so one rounding of T then exact scaling equals rounding the scaled value.
            assert oracle.emu_combine(lv, s, e, f) == want


@pytest.mark.parametrize("s", [1, 3, 7])
def test_emulation_is_exact_on_small_integers(s):
    n = 40
    A, B = workload.pair("int8", 13, n)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(oracle.emu_gemm(A, B, s), ref)


def test_emulation_of_identity_is_exact():
    n = 24
    B = 0.5 + 0.5 * workload.matrix("uniform01", 6, n)  # one binade: 54 bits suffice
    I = np.eye(n)
    np.testing.assert_array_equal(oracle.emu_gemm(I, B, 7), B)
    np.testing.assert_array_equal(oracle.emu_gemm(B, I, 7), B)


def test_emulation_error_shrinks_with_slices_and_meets_bound():
    n = 32
    A, B = workload.pair("uniform11", 17, n)
    ex = np.array([[float(x) for x in row] for row in exact_product(A, B)])  # exact to 1/2 ulp
    absAB = np.abs(A) @ np.abs(B)
    errs = []
    for s in range(2, 9):
        C = oracle.emu_gemm(A, B, s)
        errs.append(np.max(np.abs(C - ex) / absAB))
    assert all(b <= a * 1.0001 or b < 1e-17 for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 2 * n * U  # two slices are far from FP64 accuracy
    assert errs[-2] <= 2 * n * U  # seven slices meet the componentwise bound
    assert errs[-1] <= 2 * n * U


def test_emulated_rows_match_full_model():
    n = 70
    A, B = workload.pair("loguniform20", 23, n)
    C = oracle.emu_gemm(A, B, 5)
    rows = [0, 69, 31]
    np.testing.assert_array_equal(oracle.emu_gemm_rows(A, B, 5, rows), C[rows])


# ---- the modular form's definition: exact product of fixed-point operands ----

def _py_exponent(vals):
    m = max(abs(float(v)) for v in vals)
    return 0 if m == 0 else math.frexp(m)[1]  # m = f 2^e, f in [0.5, 1)


def _py_fixed_product(A, B, beta):
    """Every step with Python integers and fractions, independent of oracle.c."""
    n = A.shape[0]
    e = [_py_exponent(A[i, :]) for i in range(n)]
    f = [_py_exponent(B[:, k]) for k in range(n)]
    Ai = [[round(Fraction(float(A[i, j])) * Fraction(2) ** (beta - e[i])) for j in range(n)] for i in range(n)]
    Bi = [[round(Fraction(float(B[j, k])) * Fraction(2) ** (beta - f[k])) for k in range(n)] for j in range(n)]
    C = np.empty((n, n))
    for i in range(n):
        for k in range(n):
            X = sum(Ai[i][j] * Bi[j][k] for j in range(n))
            C[i, k] = float(Fraction(X) * Fraction(2) ** (e[i] + f[k] - 2 * beta))  # correctly rounded
    return C


def test_fix_is_the_exact_rounding():
    vals = list(workload.values("loguniform20", 4, 200)) + [0.0, -0.0, 1 - 2 ** -53, -(1 - 2 ** -53), 0.5,
                                                             2 ** -60, 3 * 2 ** -56]
    for beta in (1, 7, 30, 47, 55, 62):
        for v in vals:
            e = 1 if abs(v) < 1 else math.frexp(abs(v))[1]
            assert oracle.fix(v, e, beta) == round(Fraction(float(v)) * Fraction(2) ** (beta - e))
    assert oracle.fix(3 * 2.0 ** -3, 0, 2) == 2   # 1.5 -> 2 (ties to even)
    assert oracle.fix(5 * 2.0 ** -3, 0, 2) == 2   # 2.5 -> 2
    assert oracle.fix(-5 * 2.0 ** -3, 0, 2) == -2


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("dist", ["uniform11", "loguniform20"])
def test_fixed_product_by_exact_integers(n, dist):
    A, B = workload.pair(dist, 30 + n, n)
    A[0, :] *= 2.0 ** 30  # rows and columns on different scales
    B[:, -1] *= 2.0 ** -25
    for beta in (3, 21, 40, 55, 60):
        np.testing.assert_array_equal(oracle.fixed_gemm(A, B, beta), _py_fixed_product(A, B, beta))


def test_fixed_product_with_zero_rows_and_columns():
    n = 6
    A, B = workload.pair("uniform11", 41, n)
    A[2, :] = 0.0
    B[:, 4] = -0.0
    C = oracle.fixed_gemm(A, B, 50)
    np.testing.assert_array_equal(C, _py_fixed_product(A, B, 50))
    assert np.all(C[2, :] == 0) and np.all(C[:, 4] == 0)


@pytest.mark.parametrize("beta", [4, 20, 55])
def test_fixed_product_is_exact_on_small_integers(beta):
    n = 40  # entries in {-8..8}: a 2^(beta - e) is an integer once beta >= 4
    A, B = workload.pair("int8", 13, n)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(oracle.fixed_gemm(A, B, beta), ref)


@pytest.mark.parametrize("dist", ["uniform11", "loguniform20"])
def test_fixed_product_error_bound(dist):
    # a_ij 2^(beta - e_i) moves by at most 1/2 when rounded, so
    # |X 2^(e+f-2beta) - (AB)_ik| <= 2^(-beta-1) (2^e_i sum_j |b_jk| + 2^f_k sum_j |a_ij|)
    #                                 + n 2^(e_i + f_k - 2 beta - 2),
    # and the final rounding adds at most 2^-53 of the result.
    n = 32
    A, B = workload.pair(dist, 17, n)
    ex = exact_product(A, B)
    e = np.array([_py_exponent(A[i, :]) for i in range(n)], dtype=np.float64)
    f = np.array([_py_exponent(B[:, k]) for k in range(n)], dtype=np.float64)
    rowsum = np.abs(A).sum(axis=1)
    colsum = np.abs(B).sum(axis=0)
    errs = []
    for beta in (16, 30, 45, 55):
        C = oracle.fixed_gemm(A, B, beta)
        worst = 0.0
        for i in range(n):
            for k in range(n):
                fix_err = (2.0 ** (e[i] - beta - 1) * colsum[k] + 2.0 ** (f[k] - beta - 1) * rowsum[i]
                           + n * 2.0 ** (e[i] + f[k] - 2 * beta - 2))
                bound = Fraction(fix_err) + Fraction(U) * (abs(ex[i][k]) + Fraction(fix_err))
                err = abs(Fraction(float(C[i, k])) - ex[i][k])
                assert err <= bound * Fraction(1001, 1000), (beta, i, k)
                worst = max(worst, float(err / max(Fraction(float((np.abs(A) @ np.abs(B))[i, k])), Fraction(1, 2**1000))))
        errs.append(worst)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    if dist == "uniform11":
        assert errs[0] > 2 * n * U >= errs[-1], errs  # 16 bits are not FP64, 55 bits meet the bound
    # (wide-range entries: the width is relative to the row and column maxima,
    # so at n = 32 a dot product of small entries keeps a larger relative error)


def test_fixed_rows_match_full_product():
    n = 70
    A, B = workload.pair("loguniform20", 23, n)
    C = oracle.fixed_gemm(A, B, 48)
    rows = [0, 69, 31]
    np.testing.assert_array_equal(oracle.fixed_gemm_rows(A, B, 48, rows), C[rows])


def test_modular_width_rule():
    M = oracle.MODULI
    assert len(M) == 16 and list(M) == sorted(M, reverse=True) and max(M) <= 256
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(M) for b in M[i + 1:])
    assert math.prod(M) < 2 ** 126  # recovered integers fit a signed 128-bit word
    for k in range(2, 17):
        Mk = math.prod(M[:k])
        for n in (1, 100, 500, 2000, 4095, 8192, 16384, 32767):
            beta = oracle.modular_beta(k, n)
            if beta == 0:
                assert 514 * n * 4 > 256 * Mk
                continue
            # |X| <= n 2^(2 beta) is below M_k / 2 with a margin of M_k / 514
            assert 2 * n * 2 ** (2 * beta) + Fraction(Mk, 257) <= Mk
            assert beta == oracle.MAX_FIXED_BITS or 514 * n * 2 ** (2 * beta + 2) > 256 * Mk
    assert oracle.modular_beta(16, 100) == 58 and oracle.modular_beta(16, 500) == 57
    assert oracle.modular_beta(16, 2000) == 56 and oracle.modular_beta(16, 16384) == 55
    assert oracle.modular_beta(14, 8192) == 48 and oracle.modular_beta(14, 2000) == 49
    assert oracle.modular_beta(15, 2000) == 52


# ---------------------------------------------------------------------------
# Rectangular products (oracle section 5): C (m x n) = A (m x k) . B (k x n)
# ---------------------------------------------------------------------------
RECT_SHAPES = [(1, 1, 1), (1, 5, 3), (4, 1, 6), (3, 7, 1), (5, 3, 9), (9, 4, 2), (6, 6, 6)]


def _py_left_to_right(A, B):
    m, k = A.shape
    n = B.shape[1]
    C = np.empty((m, n))
    for i in range(m):
        for l in range(n):
            c = 0.0
            for j in range(k):
                c = c + float(A[i, j]) * float(B[j, l])  # Python floats: rounded product, rounded sum
            C[i, l] = c
    return C


def _py_fixed_product_mnk(A, B, beta):
    """Every step with Python integers and fractions, for any m x k times k x n."""
    m, k = A.shape
    n = B.shape[1]
    e = [_py_exponent(A[i, :]) for i in range(m)]
    f = [_py_exponent(B[:, l]) for l in range(n)]
    Ai = [[round(Fraction(float(A[i, j])) * Fraction(2) ** (beta - e[i])) for j in range(k)] for i in range(m)]
    Bi = [[round(Fraction(float(B[j, l])) * Fraction(2) ** (beta - f[l])) for l in range(n)] for j in range(k)]
    C = np.empty((m, n))
    for i in range(m):
        for l in range(n):
            X = sum(Ai[i][j] * Bi[j][l] for j in range(k))
            C[i, l] = float(Fraction(X) * Fraction(2) ** (e[i] + f[l] - 2 * beta))
    return C


@pytest.mark.parametrize("m,n,k", RECT_SHAPES)
def test_rect_product_is_the_left_to_right_sum(m, n, k):
    A, B = workload.rect_pair("uniform11", 7 * m + n + k, m, n, k)
    want = _py_left_to_right(A, B)
    np.testing.assert_array_equal(oracle.gemm_mnk(A, B), want)
    np.testing.assert_array_equal(oracle.gemm_mnk(A, B, rows=[m - 1, 0]), want[[m - 1, 0]])
    np.testing.assert_array_equal(oracle.absgemm_mnk(A, B), _py_left_to_right(np.abs(A), np.abs(B)))


def test_rect_functions_reduce_to_the_square_ones():
    n = 23
    A, B = workload.pair("loguniform20", 5, n)
    A2, B2 = workload.rect_pair("loguniform20", 5, n, n, n)
    np.testing.assert_array_equal(A, A2)
    np.testing.assert_array_equal(B, B2)
    np.testing.assert_array_equal(oracle.gemm_mnk(A, B), oracle.gemm(A, B))
    np.testing.assert_array_equal(oracle.fixed_gemm_mnk(A, B, 45), oracle.fixed_gemm(A, B, 45))
    np.testing.assert_array_equal(oracle.emu_gemm_mnk(A, B, 7), oracle.emu_gemm(A, B, 7))


@pytest.mark.parametrize("m,n,k", [(5, 3, 40), (2, 9, 17), (12, 1, 33)])
def test_rect_integer_products_are_exact(m, n, k):
    A, B = workload.rect_pair("int8", 3 + k, m, n, k)
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(oracle.gemm_mnk(A, B), want)
    np.testing.assert_array_equal(oracle.fixed_gemm_mnk(A, B, 20), want)
    np.testing.assert_array_equal(oracle.emu_gemm_mnk(A, B, 2), want)


@pytest.mark.parametrize("m,n,k", RECT_SHAPES)
@pytest.mark.parametrize("beta", [5, 33, 60])
def test_rect_fixed_product_against_exact_integers(m, n, k, beta):
    A, B = workload.rect_pair("loguniform20", 11 * m + k, m, n, k)
    A[0, 0] = 0.0
    np.testing.assert_array_equal(oracle.fixed_gemm_mnk(A, B, beta), _py_fixed_product_mnk(A, B, beta))


@pytest.mark.parametrize("m,n,k", [(5, 3, 9), (9, 4, 2), (1, 7, 30), (13, 2, 5)])
def test_rect_emulation_models_commute_with_transposition(m, n, k):
    # (A B)^T = B^T A^T: a row exponent of A becomes a column exponent of
    # A^T, the digit pairs (t, u) become (u, t) -- the kept set t + u <= s + 1
    # is symmetric -- and every integer sum is the same, so both models give
    # the transposed result bit for bit.  A swapped exponent, a row/column
    # mix-up or an asymmetric pair set breaks it.
    A, B = workload.rect_pair("loguniform20", 17 + m, m, n, k)
    for s in (3, 7):
        np.testing.assert_array_equal(oracle.emu_gemm_mnk(A, B, s), oracle.emu_gemm_mnk(B.T, A.T, s).T)
    for beta in (21, 58):
        np.testing.assert_array_equal(oracle.fixed_gemm_mnk(A, B, beta), oracle.fixed_gemm_mnk(B.T, A.T, beta).T)


def test_rect_emulation_model_error_bound():
    # With enough digits the digit model is within 2 k u |A||B| of the exact product.
    m, n, k = 7, 5, 300
    A, B = workload.rect_pair("uniform11", 2, m, n, k)
    exact = np.array([[float(sum(Fraction(float(A[i, j])) * Fraction(float(B[j, l])) for j in range(k)))
                       for l in range(n)] for i in range(m)])
    absab = oracle.absgemm_mnk(A, B)
    for C in (oracle.emu_gemm_mnk(A, B, 7), oracle.fixed_gemm_mnk(A, B, 55), oracle.gemm_mnk(A, B)):
        assert np.all(np.abs(C - exact) <= 2 * k * 2.0 ** -53 * absab)
