"""Parity of the INT8 slice form (MM_EMU_INT8: signed-byte digits, int32
accumulation on the mma.sync s8 path) with the oracle.

The form's result has a model in the oracle (section 6: the (8s - 2)-bit
fixed point, balanced base-256 digits, digit pairs of level <= s + 1, one
rounding), pinned on the CPU in test_i8_model.py; every comparison with it
here is bit for bit, through the C ABI, with the accuracy certificate off
(MM_FLAG_NO_GUARD) so that nothing is replaced by native FP64.  With the
certificate on (the default) results are checked against the plain product
at the bound 2 N 2^-53 |A||B|.
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import U, assert_within_bound, dev, host

pytestmark = pytest.mark.gpu


def handle(s=7, flags=None, tune_path=None):
    import paper_1012_2273_gb300 as mm
    return mm.Handle("int8", slices=s, flags=mm.FLAG_NO_GUARD if flags is None else flags, tune_path=tune_path)


def bits(C):
    return np.asarray(C).view(np.int64)


@pytest.mark.parametrize("dist", ["uniform11", "loguniform20"])
@pytest.mark.parametrize("n", [1, 7, 63, 64, 65, 127, 128, 129, 200, 255, 256, 257, 300, 511, 640])
def test_int8_bit_exact_vs_model(n, dist):
    A, B = workload.pair(dist, 700 + n, n)
    with handle(7) as h:
        assert h.plan(n) == (3, 7)
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(bits(C), bits(oracle.i8_gemm(A, B, 7)))


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6, 8])
def test_int8_every_slice_count(s):
    n = 300
    A, B = workload.pair("uniform11", 80 + s, n)
    with handle(s) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(bits(C), bits(oracle.i8_gemm(A, B, s)))


def test_int8_exact_on_small_integers_and_zero_rows():
    n = 333
    A, B = workload.pair("int8", 4, n)
    A[7, :] = 0.0
    B[:, 9] = 0.0
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for s in (1, 7):
        with handle(s, flags=0) as h:  # certificate on: integers are exact anyway
            C = host(h.gemm(dev(A), dev(B)))
            h.check()
        np.testing.assert_array_equal(C, want)


@pytest.mark.parametrize("groups", [1, 2, 5, 28])
def test_int8_forced_pair_groups_are_bit_exact(tmp_path, groups):
    tune = tmp_path / "tune.txt"
    tune.write_text(f"100000 3 7 128 {groups}\n")
    n = 520
    A, B = workload.pair("loguniform20", 21, n)
    with handle(7, tune_path=str(tune)) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(bits(C), bits(oracle.i8_gemm(A, B, 7)))


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(1, 300, 77), (300, 7, 45), (129, 257, 513), (257, 129, 3)])
def test_int8_rectangular_and_transposed(m, n, k, ta, tb):
    A, B = workload.rect_pair("uniform11", 30 + m, m, n, k)
    dA = dev(A.T.copy()).T if ta else dev(A)
    dB = dev(B.T.copy()).T if tb else dev(B)
    with handle(6) as h:
        C = host(h.gemm(dA, dB))
        h.check()
    np.testing.assert_array_equal(bits(C), bits(oracle.i8_gemm(A, B, 6)))


@pytest.mark.parametrize("use_graph", [True, False])
def test_grouped_call_with_int8_modular_and_native_problems(tmp_path, use_graph):
    import paper_1012_2273_gb300 as mm
    tune = tmp_path / "tune.txt"
    tune.write_text("60 0 7 256 0\n400 3 7 128 0\n100000 2 15 256 0\n")
    sizes = [700, 40, 250, 1, 129, 300, 64, 401]
    pairs = [workload.pair("uniform11", 170 + i, n) for i, n in enumerate(sizes)]
    flags = mm.FLAG_NO_GUARD | (0 if use_graph else mm.FLAG_NO_GRAPH)
    with mm.Handle("auto", flags=flags, tune_path=str(tune)) as h:
        plans = {n: h.plan(n) for n in sizes}
        for _ in range(2):
            Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
            h.check()
            for (A, B), C, n in zip(pairs, Cs, sizes):
                form, k = plans[n]
                C = host(C)
                if form == 0:
                    assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)
                elif form == 3:
                    np.testing.assert_array_equal(bits(C), bits(oracle.i8_gemm(A, B, k)))
                else:
                    np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm(A, B, oracle.modular_beta(k, n))))
    assert {f for f, _ in plans.values()} == {0, 2, 3}


@pytest.mark.parametrize("dist,s", [("uniform11", 7), ("loguniform20", 8)])
def test_int8_n2000_within_the_bound_with_the_certificate(dist, s):
    n = 2000
    A, B = workload.pair(dist, 9, n)
    with handle(s, flags=0) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
        replaced, _ = h.guard_read()
    rows = [0, 1, 777, n - 1]
    ref = oracle.gemm_rows(A, B, rows)
    assert_within_bound(C[rows], ref, np.abs(A[rows]) @ np.abs(B), n)
    bad, _, _ = oracle.freivalds(A, B, C, np.random.default_rng(5).choice([-1.0, 1.0], n))
    assert bad == 0
    if replaced == 0:
        np.testing.assert_array_equal(bits(C[rows[:2]]), bits(oracle.i8_gemm(A, B, s, rows=rows[:2])))


def test_int8_structured_inputs_stay_within_the_bound():
    n = 300
    for kind in workload.STRUCTURES:
        A, B = workload.structured_pair(kind, 55, n)
        with handle(7, flags=0) as h:
            C = host(h.gemm(dev(A), dev(B)))
            h.check()
        assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)


def test_int8_probe_reports_a_positive_rate():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("auto") as h:
        tops = h.probe_int8_peak()
    assert tops > 1.0
