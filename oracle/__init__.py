"""CPU oracle for the dense N x N FP64 product C = A.B (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports, links or runs it, and it shares no code with
that path.

The arithmetic lives in ``oracle.c`` (plain C, FP64, no FMA contraction);
this module compiles it with gcc on first use and binds it with ctypes.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  gemm / gemm_alg1 / gemm_rows -- identity, permutation, all-ones, small
      integers (exact), hand-expanded 1x1..4x4, textbook 2x2, loop-order
      and thread-count invariance, exact rational product within gamma_n.
  absgemm -- exact integer case, bound against the exact rational value.
  gemm_dot2 -- exact rational product (Python fractions) on small cases.
  freivalds -- accepts exact products, rejects planted errors.
  fixed_gemm / fixed_gemm_rows / fix -- the exact product of the rounded
      fixed-point operands, against Python integers and fractions on small
      random cases (every step: exponents, rounding, exact sum, one final
      rounding), exact on small-integer inputs, within the fixed-point error
      bound of the exact product on random ones.
  modular_beta -- the fixed-point width rule, against Python big integers.
  i8_* -- the INT8 slice model: D equals the exact rounding of
      a 2^(8s-2-e) (Python fractions); its digits are signed bytes and
      reconstruct D; the whole product equals a brute-force restatement in
      Python integers on small cases, is exact on small-integer inputs, and
      obeys the certificate's error bound (test_guard_rule.py).
  emu_* -- digits reconstruct D exactly; D equals the exact rounding of
      a 2^(8s-1-e) (Python fractions); level sums equal brute force with
      Python integers; RN of 128-bit integers equals Python's correctly
      rounded int -> float; the full model is exact on small-integer inputs
      and within the error bound of the exact product on random ones.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]

_lock = threading.Lock()
_lib = None

MAX_SLICES = 8


def build(force: bool = False) -> str:
    """Compiles oracle.c into oracle/_build/liboracle.so; returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if force or not fresh:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_I16 = ctypes.POINTER(ctypes.c_int16)
_I64 = ctypes.POINTER(ctypes.c_int64)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            c_int, c_double = ctypes.c_int, ctypes.c_double
            L.or_gemm_alg1.argtypes = [c_int, _D, _D, _D]
            L.or_gemm.argtypes = [c_int, _D, _D, _D, c_int]
            L.or_gemm_rows.argtypes = [c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_absgemm.argtypes = [c_int, _D, _D, _D, c_int]
            L.or_gemm_dot2.argtypes = [c_int, _D, _D, _D, c_int]
            L.or_freivalds.argtypes = [c_int, _D, _D, _D, _D, c_double, _D, _D]
            L.or_freivalds.restype = c_int
            L.or_emu_row_exponents.argtypes = [c_int, _D, _I]
            L.or_emu_col_exponents.argtypes = [c_int, _D, _I]
            L.or_emu_fixed.argtypes = [c_double, c_int, c_int]
            L.or_emu_fixed.restype = ctypes.c_int64
            L.or_emu_digits_of.argtypes = [ctypes.c_int64, c_int, _I]
            L.or_emu_digit_planes.argtypes = [c_int, c_int, _D, _I, c_int, _I16]
            L.or_emu_level_sums.argtypes = [c_int, c_int, _I16, _I16, _I64, c_int]
            L.or_emu_combine.argtypes = [_I64, c_int, c_int, c_int]
            L.or_emu_combine.restype = c_double
            L.or_emu_gemm.argtypes = [c_int, c_int, _D, _D, _D, c_int]
            L.or_emu_gemm.restype = c_int
            L.or_emu_gemm_rows.argtypes = [c_int, c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_emu_gemm_rows.restype = c_int
            L.or_max_threads.restype = c_int
            L.or_int128_to_double.argtypes = [ctypes.c_int64, ctypes.c_uint64]
            L.or_int128_to_double.restype = c_double
            L.or_fix.argtypes = [c_double, c_int, c_int]
            L.or_fix.restype = ctypes.c_int64
            L.or_fixed_gemm.argtypes = [c_int, c_int, _D, _D, _D, c_int]
            L.or_fixed_gemm.restype = c_int
            L.or_fixed_gemm_rows.argtypes = [c_int, c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_fixed_gemm_rows.restype = c_int
            L.or_gemm_mnk.argtypes = [c_int, c_int, c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_absgemm_mnk.argtypes = [c_int, c_int, c_int, _D, _D, _D, c_int]
            L.or_fixed_gemm_mnk.argtypes = [c_int, c_int, c_int, c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_fixed_gemm_mnk.restype = c_int
            L.or_emu_gemm_mnk.argtypes = [c_int, c_int, c_int, c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_emu_gemm_mnk.restype = c_int
            L.or_i8_fixed.argtypes = [c_double, c_int, c_int]
            L.or_i8_fixed.restype = ctypes.c_int64
            L.or_i8_digits_of.argtypes = [ctypes.c_int64, c_int, _I]
            L.or_i8_combine.argtypes = [_I64, c_int, c_int, c_int]
            L.or_i8_combine.restype = c_double
            L.or_i8_gemm_mnk.argtypes = [c_int, c_int, c_int, c_int, _D, _D, _I, c_int, _D, c_int]
            L.or_i8_gemm_mnk.restype = c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _square(A, B):
    A, B = _f64(A), _f64(B)
    n = A.shape[0]
    if A.shape != (n, n) or B.shape != (n, n):
        raise ValueError("oracle: A and B must be square and of the same size")
    return A, B, n


def threads(nthreads: int | None) -> int:
    return lib().or_max_threads() if nthreads is None else int(nthreads)


def gemm(A, B, nthreads: int | None = None) -> np.ndarray:
    """C = A.B with the paper's arithmetic (Alg. 1 / Alg. 4)."""
    A, B, n = _square(A, B)
    C = np.empty((n, n), np.float64)
    lib().or_gemm(n, _dp(A), _dp(B), _dp(C), threads(nthreads))
    return C


def gemm_alg1(A, B) -> np.ndarray:
    """C = A.B by the literal i, k, j loop of Alg. 1 (single thread)."""
    A, B, n = _square(A, B)
    C = np.empty((n, n), np.float64)
    lib().or_gemm_alg1(n, _dp(A), _dp(B), _dp(C))
    return C


def gemm_rows(A, B, rows, nthreads: int | None = None) -> np.ndarray:
    """Rows ``rows`` of A.B (same arithmetic as :func:`gemm`)."""
    A, B, n = _square(A, B)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty((len(r), n), np.float64)
    lib().or_gemm_rows(n, _dp(A), _dp(B), r.ctypes.data_as(_I), len(r), _dp(out), threads(nthreads))
    return out


def absgemm(A, B, nthreads: int | None = None) -> np.ndarray:
    """|A||B|, the denominator of the componentwise error."""
    A, B, n = _square(A, B)
    C = np.empty((n, n), np.float64)
    lib().or_absgemm(n, _dp(A), _dp(B), _dp(C), threads(nthreads))
    return C


def gemm_dot2(A, B, nthreads: int | None = None) -> np.ndarray:
    """A.B with compensated (Dot2) dot products: nearly the exact product."""
    A, B, n = _square(A, B)
    C = np.empty((n, n), np.float64)
    lib().or_gemm_dot2(n, _dp(A), _dp(B), _dp(C), threads(nthreads))
    return C


def freivalds(A, B, C, x, slack: float = 4.0):
    """Freivalds' check with probe x; returns (bad_rows, y, tol)."""
    A, B, n = _square(A, B)
    C, x = _f64(C), _f64(x)
    y = np.empty(n, np.float64)
    tol = np.empty(n, np.float64)
    bad = lib().or_freivalds(n, _dp(A), _dp(B), _dp(C), _dp(x), float(slack), _dp(y), _dp(tol))
    if bad < 0:
        raise MemoryError("oracle: freivalds allocation failed")
    return bad, y, tol


# ---- model of the split-precision emulation ---------------------------------

def emu_row_exponents(A) -> np.ndarray:
    A = _f64(A)
    n = A.shape[0]
    e = np.empty(n, np.int32)
    lib().or_emu_row_exponents(n, _dp(A), e.ctypes.data_as(_I))
    return e


def emu_col_exponents(B) -> np.ndarray:
    B = _f64(B)
    n = B.shape[0]
    f = np.empty(n, np.int32)
    lib().or_emu_col_exponents(n, _dp(B), f.ctypes.data_as(_I))
    return f


def emu_fixed(v: float, e: int, s: int) -> int:
    return int(lib().or_emu_fixed(float(v), int(e), int(s)))


def emu_digits_of(D: int, s: int) -> list[int]:
    d = (ctypes.c_int * s)()
    lib().or_emu_digits_of(int(D), int(s), d)
    return list(d)


def emu_digit_planes(M, ex, s: int, col_major: bool) -> np.ndarray:
    """Digit planes [s][n][n] (int16) of an operand; see oracle.c."""
    M = _f64(M)
    n = M.shape[0]
    ex = np.ascontiguousarray(ex, dtype=np.int32)
    out = np.empty((s, n, n), np.int16)
    lib().or_emu_digit_planes(n, s, _dp(M), ex.ctypes.data_as(_I), int(col_major),
                              out.ctypes.data_as(_I16))
    return out


def emu_level_sums(dA, dB, nthreads: int | None = None) -> np.ndarray:
    """Exact level sums S_L, L = 2..s+1, as int64 [s][n][n]."""
    dA = np.ascontiguousarray(dA, dtype=np.int16)
    dB = np.ascontiguousarray(dB, dtype=np.int16)
    s, n, _ = dA.shape
    S = np.empty((s, n, n), np.int64)
    lib().or_emu_level_sums(n, s, dA.ctypes.data_as(_I16), dB.ctypes.data_as(_I16),
                            S.ctypes.data_as(_I64), threads(nthreads))
    return S


def emu_combine(levels, s: int, e: int, f: int) -> float:
    lv = np.ascontiguousarray(levels, dtype=np.int64)
    return float(lib().or_emu_combine(lv.ctypes.data_as(_I64), int(s), int(e), int(f)))


def emu_gemm(A, B, s: int, nthreads: int | None = None) -> np.ndarray:
    """The emulated product with s slices, from the model's definitions."""
    A, B, n = _square(A, B)
    C = np.empty((n, n), np.float64)
    rc = lib().or_emu_gemm(n, int(s), _dp(A), _dp(B), _dp(C), threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: emu_gemm failed ({rc})")
    return C


def emu_gemm_rows(A, B, s: int, rows, nthreads: int | None = None) -> np.ndarray:
    A, B, n = _square(A, B)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty((len(r), n), np.float64)
    rc = lib().or_emu_gemm_rows(n, int(s), _dp(A), _dp(B), r.ctypes.data_as(_I), len(r), _dp(out),
                                threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: emu_gemm_rows failed ({rc})")
    return out


def int128_to_double(T: int) -> float:
    hi = T >> 64
    lo = T & ((1 << 64) - 1)
    return float(lib().or_int128_to_double(hi, lo))


def max_threads() -> int:
    return int(lib().or_max_threads())


# ---- 4. the modular form: exact product of fixed-point operands -------------

# The moduli of the modular emulation form, in the order the library uses
# them: pairwise coprime, each at most 256 so that every symmetric residue
# (|r| <= 128) is an exact bf16 value.  The first k are used with k moduli.
MODULI = (256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193)
MAX_FIXED_BITS = 62


def modular_beta(k: int, n: int) -> int:
    """Fixed-point width used with the first k moduli at size n.

    The largest beta <= 62 with 514 n 2^(2 beta) <= 256 M_k (M_k the product
    of the first k moduli): the exact product X of two beta-bit operands has
    |X| <= n 2^(2 beta) <= (256/514) M_k / 2 < M_k / 2, so X is the unique
    integer of its residue class within half the modulus of zero, and stays
    a margin of M_k / 514 away from the ends of that range.  0 means k is too
    small for n.
    """
    M = 1
    for m in MODULI[:k]:
        M *= m
    for beta in range(MAX_FIXED_BITS, 0, -1):
        if 514 * n * (1 << (2 * beta)) <= 256 * M:
            return beta
    return 0


def fix(v: float, e: int, beta: int) -> int:
    """round-half-even(v 2^(beta - e))."""
    return int(lib().or_fix(float(v), int(e), int(beta)))


def fixed_gemm(A, B, beta: int, nthreads: int | None = None) -> np.ndarray:
    """RN(sum_j A_int B_int) 2^(e_i + f_k - 2 beta): the modular form's result."""
    A, B, n = _square(A, B)
    C = np.empty((n, n), np.float64)
    rc = lib().or_fixed_gemm(n, int(beta), _dp(A), _dp(B), _dp(C), threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: fixed_gemm failed ({rc})")
    return C


def fixed_gemm_rows(A, B, beta: int, rows, nthreads: int | None = None) -> np.ndarray:
    A, B, n = _square(A, B)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty((len(r), n), np.float64)
    rc = lib().or_fixed_gemm_rows(n, int(beta), _dp(A), _dp(B), r.ctypes.data_as(_I), len(r), _dp(out),
                                  threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: fixed_gemm_rows failed ({rc})")
    return out


# ---------------------------------------------------------------------------
# Rectangular products: C (m x n) = A (m x k) . B (k x n), section 5 of
# oracle.c (the paper's NRA x NCA times NCA x NCB, Alg. 2).
# ---------------------------------------------------------------------------
def _rect(A, B):
    A = _f64(A)
    B = _f64(B)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError(f"oracle: shapes {A.shape} and {B.shape} do not chain")
    return A, B, A.shape[0], B.shape[1], A.shape[1]


def _rows_arg(rows, m):
    if rows is None:
        return None, m
    r = np.ascontiguousarray(rows, dtype=np.int32)
    return r, len(r)


def gemm_mnk(A, B, rows=None, nthreads: int | None = None) -> np.ndarray:
    """Alg. 1's sum for rectangular operands (j increasing from 0.0)."""
    A, B, m, n, k = _rect(A, B)
    r, nr = _rows_arg(rows, m)
    C = np.empty((nr, n), np.float64)
    lib().or_gemm_mnk(m, n, k, _dp(A), _dp(B), r.ctypes.data_as(_I) if r is not None else None, nr, _dp(C),
                      threads(nthreads))
    return C


def absgemm_mnk(A, B, nthreads: int | None = None) -> np.ndarray:
    A, B, m, n, k = _rect(A, B)
    C = np.empty((m, n), np.float64)
    lib().or_absgemm_mnk(m, n, k, _dp(A), _dp(B), _dp(C), threads(nthreads))
    return C


def fixed_gemm_mnk(A, B, beta: int, rows=None, nthreads: int | None = None) -> np.ndarray:
    """The modular form's result for rectangular operands (exponents over the k entries)."""
    A, B, m, n, k = _rect(A, B)
    r, nr = _rows_arg(rows, m)
    C = np.empty((nr, n), np.float64)
    rc = lib().or_fixed_gemm_mnk(m, n, k, int(beta), _dp(A), _dp(B), r.ctypes.data_as(_I) if r is not None else None,
                                 nr, _dp(C), threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: fixed_gemm_mnk failed ({rc})")
    return C


def emu_gemm_mnk(A, B, s: int, rows=None, nthreads: int | None = None) -> np.ndarray:
    """The digit form's result for rectangular operands."""
    A, B, m, n, k = _rect(A, B)
    r, nr = _rows_arg(rows, m)
    C = np.empty((nr, n), np.float64)
    rc = lib().or_emu_gemm_mnk(m, n, k, int(s), _dp(A), _dp(B), r.ctypes.data_as(_I) if r is not None else None,
                               nr, _dp(C), threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: emu_gemm_mnk failed ({rc})")
    return C


# ---- section 6: the INT8 slice form -------------------------------------------

def i8_fixed(v: float, e: int, s: int) -> int:
    """round-half-even(v 2^(8s - 2 - e))."""
    return int(lib().or_i8_fixed(float(v), int(e), int(s)))


def i8_digits_of(D: int, s: int) -> list[int]:
    """Digits d_1..d_s of D, |D| <= 2^(8s-2): d_2..d_s in [-128, 127], d_1 in [-64, 64]."""
    d = (ctypes.c_int * s)()
    lib().or_i8_digits_of(int(D), int(s), d)
    return list(d)


def i8_combine(levels, s: int, e: int, f: int) -> float:
    """RN(sum_L S_L 2^(8(s+1-L))) 2^(e + f - 8s - 4) for levels S_2..S_{s+1}."""
    lv = (ctypes.c_int64 * s)(*[int(x) for x in levels])
    return float(lib().or_i8_combine(lv, int(s), int(e), int(f)))


def i8_gemm(A, B, s: int, rows=None, nthreads: int | None = None) -> np.ndarray:
    """The INT8 slice form's result (square or rectangular operands; the
    listed rows of A only, if `rows` is given)."""
    A, B, m, n, k = _rect(A, B)
    r, nr = _rows_arg(rows, m)
    C = np.empty((nr, n), np.float64)
    rc = lib().or_i8_gemm_mnk(m, n, k, int(s), _dp(A), _dp(B), r.ctypes.data_as(_I) if r is not None else None,
                              nr, _dp(C), threads(nthreads))
    if rc != 0:
        raise ValueError(f"oracle: i8_gemm failed ({rc})")
    return C
