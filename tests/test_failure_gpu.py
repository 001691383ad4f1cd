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
