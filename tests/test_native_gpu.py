"""Parity of the native FP64 path (mma.sync f64) with the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import workload
from helpers import assert_within_bound, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("native") as handle:
        yield handle


def test_config_n500_uniform_seed0(h):
    # Smallest benchmark configuration: N = 500, uniform [0, 1), seed 0.
    A, B = workload.pair("uniform01", 0, 500)
    C = host(h.gemm(dev(A), dev(B)))
    h.check()
    assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), 500)
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.absgemm(A, B), 500, factor=1.0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 17, 31, 33, 63, 64, 65, 100, 127, 129, 200, 257])
def test_ragged_sizes(h, n):
    A, B = workload.pair("uniform11", 1000 + n, n)
    C = host(h.gemm(dev(A), dev(B)))
    assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)


@pytest.mark.parametrize("n", [10, 100, 500, 1000])
def test_sweep_sizes(h, n):
    A, B = workload.pair("uniform01", n, n)
    C = host(h.gemm(dev(A), dev(B)))
    assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)


@pytest.mark.parametrize("n", [10, 100, 500, 1000, 1500, 2000])
def test_integer_inputs_bit_exact(h, n):
    # Entries in {-8..8}: every partial sum is an exact integer, so any order is exact.
    A, B = workload.pair("int8", 7, n)
    C = host(h.gemm(dev(A), dev(B)))
    np.testing.assert_array_equal(C, oracle.gemm(A, B))


def test_loguniform_inputs(h):
    n = 300
    A, B = workload.pair("loguniform20", 3, n)
    C = host(h.gemm(dev(A), dev(B)))
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.absgemm(A, B), n)


def test_identity_permutation_ones(h):
    n = 130
    A, B = workload.pair("uniform01", 5, n)
    I = np.eye(n)
    np.testing.assert_array_equal(host(h.gemm(dev(I), dev(B))), B)
    P = np.eye(n)[np.random.default_rng(2).permutation(n)]
    np.testing.assert_array_equal(host(h.gemm(dev(P), dev(B))), P @ B)
    J = np.ones((n, n))
    np.testing.assert_array_equal(host(h.gemm(dev(J), dev(J))), np.full((n, n), float(n)))


def test_zero_size_and_bad_arguments(h):
    import torch
    import paper_1012_2273_gb300 as mm
    e = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    assert h.gemm(e, e).shape == (0, 0)
    L = mm.lib()
    assert L.mm_gemm(h._h, -1, None, None, None, None) == 1
    A = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    # misaligned pointer
    assert L.mm_gemm(h._h, 4, A.data_ptr() + 8, A.data_ptr(), A.data_ptr() + 256, None) == 1
    # C overlapping A
    assert L.mm_gemm(h._h, 4, A.data_ptr(), A.data_ptr() + 256, A.data_ptr(), None) == 1


def test_grouped_uneven_native(h):
    sizes = [10, 1, 64, 65, 200, 33, 0, 129]
    pairs = [workload.pair("uniform11", 50 + i, n) for i, n in enumerate(sizes)]
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    for rep in range(2):  # second call replays the captured graph
        Cs = h.gemm_grouped(As, Bs)
        h.check()
        for (A, B), C, n in zip(pairs, Cs, sizes):
            if n == 0:
                continue
            assert_within_bound(host(C), oracle.gemm(A, B), oracle.absgemm(A, B), n)


def test_host_entry_point(h):
    n = 257
    A, B = workload.pair("int8", 9, n)
    C = h.gemm_host(A, B)
    np.testing.assert_array_equal(C, oracle.gemm(A, B))


def test_native_bitwise_reproducible_across_runs_tile_shapes_and_calls():
    # Each output of the native form is summed in one fixed order in both
    # kernels (16 x 8 tiles with the k chunks shared over four warps below 512
    # rows, columns and depth; 64 x 64 tiles above): chains of mma.sync over
    # 32-deep chunks of k, the chunks' sums added left to right; no atomics.
    # So the result is bitwise reproducible: across runs, between the two
    # kernels (a 500 x 500 product against the first 500 rows of a 600 x 500
    # one with the same rows of A) and between single and grouped calls.
    import torch
    import paper_1012_2273_gb300 as mm
    n = 500
    A, B = workload.pair("loguniform20", 19, n)
    A2 = np.vstack([A, workload.matrix("uniform11", 20, n)[:100]])
    with mm.Handle("native") as h:
        C1 = host(h.gemm(dev(A), dev(B)))
        C2 = host(h.gemm(dev(A), dev(B)))
        big = host(h.gemm(dev(A2), dev(B)))            # 600 x 500: the 64 x 64 kernel
        G = h.gemm_grouped([dev(A), dev(A2)], [dev(B), dev(B)])
        h.check()
    assert np.array_equal(C1.view(np.int64), C2.view(np.int64))
    assert np.array_equal(C1.view(np.int64), big[:n].view(np.int64))
    assert np.array_equal(host(G[0]).view(np.int64), C1.view(np.int64))
    assert np.array_equal(host(G[1]).view(np.int64), big.view(np.int64))


def test_many_small_problems_one_warp_per_tile_same_bits():
    # A grouped call of many small native problems runs one warp per 16 x 8
    # tile (its chunks in order); single calls of the same problems run the
    # latency kernel (a tile's chunks over four warps).  Both add the chunk
    # sums in the canonical order, so the bits agree, and every result is
    # within the bound of the oracle's.
    import paper_1012_2273_gb300 as mm
    sizes = workload.loguniform_sizes(300, 10, 250, seed=4)
    pairs = [workload.pair("uniform11", 500 + i, n) for i, n in enumerate(sizes)]
    with mm.Handle("native") as h:
        Cs = [host(c) for c in h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])]
        h.check()
        for i in range(0, len(sizes), 7):
            A, B = pairs[i]
            C1 = host(h.gemm(dev(A), dev(B)))
            h.check()
            np.testing.assert_array_equal(C1.view(np.int64), Cs[i].view(np.int64))
    for i in range(0, len(sizes), 5):
        A, B = pairs[i]
        assert_within_bound(Cs[i], oracle.gemm(A, B), oracle.absgemm(A, B), sizes[i])
