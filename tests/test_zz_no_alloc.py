"""mm_split_noalloc: the scale-and-split step for callers that cannot allocate.

Checks the allocation-free entry point against mm_split (the entry point that
uses the handle's workspace) on two calls in a row.  The second call has far
smaller values than the first, so maxima left over in the shared static
scratch from the first call would change its exponents; both calls must
match mm_split bit for bit (exponents and digits are integers).  Collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import workload
from helpers import dev

pytestmark = pytest.mark.gpu


def reference_split(M, by_columns, s):
    import paper_1012_2273_gb300 as mm
    with mm.Handle("emulated") as h:
        e, d = h.split(dev(M), by_columns, s)
        h.check()
    return e.cpu().numpy(), d.cpu().numpy()


def noalloc_split(M, by_columns, s):
    import torch
    import paper_1012_2273_gb300 as mm
    n = M.shape[0]
    rows, ld = -(-n // 128) * 128, -(-n // 64) * 64
    exps = torch.full((n,), -12345, dtype=torch.int32, device="cuda")
    digits = torch.full((s, rows, ld), 0x7FC0, dtype=torch.int16, device="cuda")  # NaN patterns
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = mm.split_noalloc(dev(M), by_columns, s, exps, digits, status)
    assert rc == 0
    torch.cuda.synchronize()
    return exps.cpu().numpy(), digits.cpu().numpy(), int(status.item())


def test_noalloc_split_matches_mm_split_on_two_calls_in_a_row():
    s = 7
    A = workload.matrix("loguniform20", 31, 300)                 # maxima up to 2^20
    B = workload.matrix("uniform01", 32, 200) * 2.0 ** -30       # maxima below 2^-30
    for M, by_columns in ((A, False), (B, True)):
        e, d, st = noalloc_split(M, by_columns, s)
        e_ref, d_ref = reference_split(M, by_columns, s)
        assert st == 0
        np.testing.assert_array_equal(e, e_ref)
        np.testing.assert_array_equal(d, d_ref)


def test_noalloc_split_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_1012_2273_gb300 as mm
    L = mm.lib()
    n = mm.SPLIT_NOALLOC_MAX_N + 1
    small = torch.zeros(256, dtype=torch.float64, device="cuda")
    buf = torch.zeros(256, dtype=torch.int32, device="cuda")
    rows, ld = -(-n // 128) * 128, -(-n // 64) * 64
    # Refused before any device work: nothing is read or written.
    rc = L.mm_split_noalloc(n, small.data_ptr(), 0, 7, buf.data_ptr(), buf.data_ptr(), rows, ld, None, None)
    assert rc == 4  # MM_ERR_UNSUPPORTED
    rc = L.mm_split_noalloc(10, small.data_ptr(), 0, 7, buf.data_ptr(), buf.data_ptr(), 100, 64, None, None)
    assert rc == 1  # rows not a multiple of 128: MM_ERR_INVALID
    _ = ctypes


def test_noalloc_split_reports_nonfinite_input():
    M = workload.matrix("uniform01", 33, 64)
    M[5, 7] = np.inf
    _, _, st = noalloc_split(M, False, 3)
    assert st == 6  # MM_ERR_NONFINITE
