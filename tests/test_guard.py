"""The accuracy certificate's arithmetic (guard.cuh, used on the device by the
split and the slice-product kernel), compiled for the host and checked
against exact rational arithmetic: the magnitude digit is the floor of the
lowest |v'| 2^7 a fixed-point value D can stand for, and the row/column sum
term bounds the highest |v'| 2^24 from above by less than one; the FP32 constants bound the exact K1 from
above and K2 (1 - 2^-20) from below; and every FP32 test that passes implies
the exact inequality (SA + SB) + K1 <= K2 S."""
import math
import os
import random
import shutil
import subprocess
from fractions import Fraction as Fr

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U = Fr(1, 2 ** 53)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("needs g++")
    exe = str(tmp_path_factory.mktemp("guard") / "guard_check")
    subprocess.run([gxx, "-std=c++17", "-O2", os.path.join(ROOT, "tests", "guard_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120,
                           check=True)
        out = r.stdout.strip().splitlines()
        assert len(out) == len(lines)
        return out
    return run


def kappa(s: int, w: int) -> Fr:
    """Digit pairs (t, u), 1 <= t, u <= s, t + u = L >= s + 2, each at most
    2^14 in magnitude, weigh 2^(8(2s - L)) 2^-2w after scaling by 2^-2w."""
    return sum((Fr(2 * s + 1 - L) * Fr(2) ** (14 + 16 * s - 8 * L - 2 * w) for L in range(s + 2, 2 * s + 1)), Fr(0))


def d_cases(rnd):
    out = []
    for w in list(range(1, 63)):
        top = 1 << w
        ds = [0, 1, -1, 2, top, -top, top - 1, 1 << max(w - 7, 0), (1 << max(w - 7, 0)) + 1]
        ds += [rnd.randrange(-top, top + 1) for _ in range(40)]
        out += [(d, w) for d in ds]
    return out


def test_magnitude_digit_is_the_floor_of_its_lower_bound(harness):
    cs = d_cases(random.Random(1))
    got = [int(x) for x in harness([f"M {d} {w}" for d, w in cs])]
    for (d, w), m in zip(cs, got):
        want = 0 if d == 0 else math.floor((Fr(abs(d)) - Fr(1, 2)) * Fr(2) ** (7 - w))
        assert m == want, (d, w, m, want)
        assert 0 <= m <= 127


def test_sum_term_bounds_the_magnitude_from_above_within_one(harness):
    cs = d_cases(random.Random(2))
    lines = [f"U {d} {w} 1" for d, w in cs] + [f"U 0 {w} 0" for w in range(1, 63)]
    got = [int(x) for x in harness(lines)]
    for (d, w), t in zip(cs, got):
        bound = (Fr(abs(d)) + Fr(1, 2)) * Fr(2) ** (24 - w)  # the largest |v'| 2^24 with this D
        assert bound <= t < bound + 1, (d, w, t)
        if w < 24:
            assert t == bound  # exact below width 24
    assert all(t == 0 for t in got[len(cs):])  # a zero entry adds nothing


def exact_constants(n, w, s):
    K1 = n * Fr(2) ** (23 - w) + n * (kappa(s, w) if s else 0) * Fr(2) ** (w + 25)
    K2 = Fr(n - 1) * Fr(2) ** (w - 42) / (1 + U)
    return K1, K2


CONST_CASES = [(n, w, 0) for n in (1, 2, 3, 300, 2000, 65535) for w in (1, 30, 45, 49, 56, 62)] + \
              [(n, 8 * s - d, s) for n in (2, 500, 131071) for s in range(1, 9) for d in (1, 2)]


def test_constants_bound_the_exact_ones(harness):
    got = harness([f"K {n} {w} {s}" for n, w, s in CONST_CASES])
    for (n, w, s), line in zip(CONST_CASES, got):
        k1, k2 = (Fr(float.fromhex(x)) for x in line.split())
        K1, K2 = exact_constants(n, w, s)
        assert k1 >= K1
        assert k1 <= K1 * (1 + Fr(1, 2 ** 20)) + Fr(1, 2 ** 120)  # not needlessly loose
        assert k2 <= K2 * (1 - Fr(1, 2 ** 20))
        assert k2 >= K2 * (1 - Fr(1, 2 ** 19))


def test_fp32_test_implies_the_exact_inequality(harness):
    rnd = random.Random(3)
    consts = harness([f"K {n} {w} {s}" for n, w, s in CONST_CASES])
    lines, meta = [], []
    for (n, w, s), line in zip(CONST_CASES, consts):
        k1s, k2s = line.split()
        K1, K2 = exact_constants(n, w, s)
        k2 = float.fromhex(k2s)
        for _ in range(60):
            S = rnd.randrange(0, min(n * 2 ** 14, 2 ** 31))
            # sums near the threshold, where rounding decides
            room = max(float(K2) * S - float(K1), 2.0)
            tot = max(1, int(room * rnd.choice((0.5, 0.999999, 1.0, 1.000001, 2.0))))
            tot = min(tot, 2 * n * (2 ** 24 + 1))  # each sum is at most n (2^24 + 1)
            sa = rnd.randrange(1, tot + 1) if tot > 1 else 1
            sb = max(tot - sa, 1)
            lines.append(f"C {sa} {sb} {S} {k1s} {k2s}")
            meta.append((sa, sb, S, K1, K2, k2))
        lines.append(f"C 0 5 0 {k1s} {k2s}")  # zero row: exempt
        meta.append(None)
    got = [int(x) for x in harness(lines)]
    passed = 0
    for m, g in zip(meta, got):
        if m is None:
            assert g == 1
            continue
        sa, sb, S, K1, K2, k2 = m
        if g:
            passed += 1
            assert Fr(sa + sb) + K1 <= K2 * S, m
    assert passed > len(meta) // 4  # the test is not vacuous


def test_magnitude_forms_from_the_absolute_value_match(harness):
    # mag7_of_abs / sum24_of_abs (the modular split's 32-bit forms for widths
    # >= 39, the 64-bit ones below) give mag7_of(D, w) and sum24_of(D, w, true)
    # for a = |D| at every width, including |D| = 0, 1, 2^w and values at the
    # word boundary of the shifts.
    rnd = random.Random(29)
    cases = []
    for w in range(1, 63):
        top = 1 << w
        vals = [0, 1, 2, top, top - 1, top // 2, (1 << 32) - 1, 1 << 32, (1 << 32) + 1]
        vals += [rnd.randrange(0, top + 1) for _ in range(300)]
        cases += [(a, w) for a in vals if a <= top]
    got = harness([f"A {a} {w}" for a, w in cases])
    want_m = harness([f"M {a} {w}" for a, w in cases])
    want_u = harness([f"U {a} {w} 1" for a, w in cases])
    assert len(got) == len(cases)
    bad = [(a, w, g, m, u) for (a, w), g, m, u in zip(cases, got, want_m, want_u) if g.split() != [m.strip(), u.strip()]]
    assert not bad, bad[:5]
