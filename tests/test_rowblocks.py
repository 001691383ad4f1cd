"""The paper's row-block decomposition (Alg. 2-4) on one GPU: the split of
the rows (CPU) and the bitwise equality of the decomposed product with the
single call in every form (GPU)."""
import numpy as np
import pytest

import workload
from helpers import dev, host


@pytest.mark.parametrize("n,w", [(10, 3), (2000, 8), (7, 7), (5, 8), (1, 1), (1000, 6)])
def test_row_ranges_follow_the_remainder_rule(n, w):
    # n // w rows per worker, one more for each of the first n % w workers,
    # contiguous and in order (Sec. 3.1.1)
    from paper_1012_2273_gb300.rowblocks import row_ranges
    r = row_ranges(n, w)
    assert len(r) == w and r[0][0] == 0 and r[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [b - a for a, b in r]
    assert sizes == [n // w + (1 if i < n % w else 0) for i in range(w)]
    assert row_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]


@pytest.mark.gpu
@pytest.mark.parametrize("mode,slices", [("native", 0), ("modular", 15), ("emulated", 7), ("auto", 0)])
def test_row_blocks_equal_the_single_call(mode, slices):
    import paper_1012_2273_gb300 as mm
    from paper_1012_2273_gb300.rowblocks import RowBlockGemm
    n = 777
    A, B = workload.pair("uniform11", 13, n)
    dA, dB = dev(A), dev(B)
    with mm.Handle(mode, slices=slices) as h:
        ref = host(h.gemm(dA, dB))
        h.check()
    for w in (1, 2, 3, 8):
        rb = RowBlockGemm(w, mode, slices)
        C = host(rb(dA, dB))
        rb.check()
        rb.close()
        assert np.array_equal(C.view(np.int64), ref.view(np.int64)), w
