"""Failure detection without a GPU fault: bounded device waits and the status word."""
import time

import numpy as np
import pytest

import oracle
import workload
from helpers import assert_within_bound, dev, host

pytestmark = pytest.mark.gpu


def test_wait_on_a_barrier_nothing_arrives_on_times_out_and_is_reported():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("auto") as h:
        t0 = time.perf_counter()
        h.selftest_wait(200)
        with pytest.raises(mm.MMError) as ei:
            h.check()
        waited = time.perf_counter() - t0
        assert ei.value.code == 5  # MM_ERR_TIMEOUT
        assert 0.15 < waited < 10.0
        # The context is still usable and the status word was cleared.
        n = 300
        A, B = workload.pair("uniform11", 1, n)
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
        assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)


def test_status_word_reports_the_first_error_only():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("emulated", slices=7) as h:
        A, B = workload.pair("uniform01", 2, 64)
        A[0, 0] = np.nan
        h.gemm(dev(A), dev(B))       # MM_ERR_NONFINITE first
        h.selftest_wait(50)          # then a timeout
        with pytest.raises(mm.MMError) as ei:
            h.check()
        assert ei.value.code == 6
        h.check()


def test_selftest_argument_checks():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("auto") as h:
        L = mm.lib()
        assert L.mm_selftest_wait(h._h, 0, None) == 1
        assert L.mm_selftest_wait(h._h, 60001, None) == 1


@pytest.mark.parametrize("pair", ["1", "0"])
def test_pipeline_waits_that_run_out_wind_down_and_later_calls_are_exact(monkeypatch, pair):
    # A limit of 100 ns on every wait of the slice-product pipeline (TMA
    # stages, accumulators, the unit ring): a normal N = 2000 product's waits
    # run out, the kernel records MM_ERR_TIMEOUT, lets its copies and MMAs
    # finish (the waits for MMAs keep their own 2 s limit; CTA pairs hold
    # both CTAs until every copy has landed), frees its tensor memory and
    # returns.  Later calls on fresh handles with the default limit run (a
    # leaked TMEM allocation would stall them) and are exact.  Both residue-
    # product kernels: CTA pairs and single CTAs (with the certificate's
    # single-CTA launch beside them).
    import paper_1012_2273_gb300 as mm
    monkeypatch.setenv("MM_PAIR_MMA", pair)
    n, k = 2000, 14
    A, B = workload.pair("uniform11", 14, n)
    dA, dB = dev(A), dev(B)
    monkeypatch.setenv("MM_TIMEOUT_MS", "0.0001")
    with mm.Handle("modular", slices=k) as h:
        h.gemm(dA, dB)
        with pytest.raises(mm.MMError) as ei:
            h.check()
        assert ei.value.code == 5  # MM_ERR_TIMEOUT
    monkeypatch.delenv("MM_TIMEOUT_MS")
    rows = [0, 999, n - 1]
    want = oracle.fixed_gemm_rows(A, B, oracle.modular_beta(k, n), rows)
    for _ in range(2):
        with mm.Handle("modular", slices=k, flags=mm.FLAG_NO_GUARD) as h:
            C = host(h.gemm(dA, dB))
            h.check()
        np.testing.assert_array_equal(C[rows].view(np.int64), want.view(np.int64))
