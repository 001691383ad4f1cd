"""The host-to-host entry points (mm_gemm_host, mm_gemm_grouped_host).

The grouped host call cuts the problems into chunks whose copies overlap the
neighbouring chunks' products; its results must equal the device-side grouped
call bit for bit (same plans, same kernels), for pageable and pinned host
memory, with empty problems, and on repeated calls (the chunks' graphs are
replayed).
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import assert_within_bound, dev, host

pytestmark = pytest.mark.gpu


SIZES = [10, 0, 100, 500, 1000, 1500, 2000, 1, 257]


@pytest.fixture(scope="module")
def pairs():
    return [workload.pair("uniform01", 60 + i, n) for i, n in enumerate(SIZES)]


def test_grouped_host_equals_grouped_device(pairs):
    import paper_1012_2273_gb300 as mm
    with mm.Handle("auto") as h:
        want = [host(c) for c in h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])]
        h.check()
        for _ in range(2):
            got = h.gemm_grouped_host([a for a, _ in pairs], [b for _, b in pairs])
            h.check()
            for n, g, w in zip(SIZES, got, want):
                np.testing.assert_array_equal(g.view(np.int64), w.view(np.int64), err_msg=f"N={n}")


def test_grouped_host_pinned_tensors_and_accuracy(pairs):
    import torch
    import paper_1012_2273_gb300 as mm
    As = [torch.from_numpy(a).pin_memory() for a, _ in pairs]
    Bs = [torch.from_numpy(b).pin_memory() for _, b in pairs]
    Cs = [torch.empty_like(a).pin_memory() for a in As]
    with mm.Handle("auto") as h:
        h.gemm_grouped_host(As, Bs, Cs)
        h.check()
    for (A, B), C, n in zip(pairs, Cs, SIZES):
        if 0 < n <= 500:
            assert_within_bound(C.numpy(), oracle.gemm(A, B), oracle.absgemm(A, B), n)
        elif n > 500:
            r = [0, n // 2, n - 1]
            assert_within_bound(C.numpy()[r], oracle.gemm_rows(A, B, r), np.abs(A[r]) @ np.abs(B), n)


def test_grouped_host_rejects_bad_input():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("auto") as h:
        with pytest.raises(ValueError):
            h.gemm_grouped_host([np.zeros((3, 4))], [np.zeros((3, 4))])
        with pytest.raises(TypeError):
            h.gemm_grouped_host([dev(np.zeros((4, 4)))], [dev(np.zeros((4, 4)))])


def test_grouped_host_many_similar_problems_fill_every_chunk():
    # 48 problems of similar size: the leading chunks close at a quarter of
    # the work each (three of them) and the last takes the rest, so every
    # chunk boundary falls inside a run of near-equal sizes; the results are
    # the device-side grouped call's bits, on two calls in a row.
    import paper_1012_2273_gb300 as mm
    sizes = [int(x) for x in np.random.default_rng(7).integers(180, 260, size=48)]
    pairs = [workload.pair("uniform11", 300 + i, n) for i, n in enumerate(sizes)]
    with mm.Handle("auto") as h:
        want = [host(c) for c in h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])]
        h.check()
        for _ in range(2):
            got = h.gemm_grouped_host([a for a, _ in pairs], [b for _, b in pairs])
            h.check()
            for n, g, w in zip(sizes, got, want):
                np.testing.assert_array_equal(g.view(np.int64), w.view(np.int64), err_msg=f"N={n}")
    A, B = pairs[0]
    assert_within_bound(got[0], oracle.gemm(A, B), oracle.absgemm(A, B), sizes[0])
