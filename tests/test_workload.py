"""The seeded input generators (shared by both sides; no product arithmetic)."""
import numpy as np
import pytest

import workload


def test_splitmix64_reference_vector():
    # First outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014 reference code).
    z = workload.splitmix64(0, 3)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    assert int(z[2]) == 0x06C45D188009454F


def test_counter_based_streams_are_reproducible():
    a = workload.splitmix64(42, 100)
    b = workload.splitmix64(42, 50, start=50)
    np.testing.assert_array_equal(a[50:], b)


def test_ranges():
    n = 20000
    u = workload.values("uniform01", 1, n)
    assert u.min() >= 0 and u.max() < 1
    v = workload.values("uniform11", 1, n)
    assert v.min() >= -1 and v.max() < 1 and v.min() < -0.99
    w = workload.values("loguniform20", 1, n)
    a = np.abs(w)
    assert a.min() >= 2.0 ** -20 and a.max() <= 2.0 ** 20
    assert 0.45 < (w < 0).mean() < 0.55
    # log-uniform: log2 magnitudes are uniform over [-20, 20]
    assert abs(np.log2(a).mean()) < 0.5
    k = workload.values("int8", 1, n)
    assert set(np.unique(k)) == set(range(-8, 9))


def test_pair_streams_differ_and_repeat():
    A, B = workload.pair("uniform01", 0, 16)
    A2, B2 = workload.pair("uniform01", 0, 16)
    np.testing.assert_array_equal(A, A2)
    np.testing.assert_array_equal(B, B2)
    assert not np.array_equal(A, B)


def test_loguniform_sizes():
    sizes = workload.loguniform_sizes(1024, 10, 2000, seed=1)
    assert len(sizes) == 1024 and min(sizes) >= 10 and max(sizes) <= 2000
    # about half of the problems are at most ~140 (median of log-uniform [10, 2001])
    med = float(np.median(sizes))
    assert 100 < med < 200


def test_device_generator_matches_the_host_draws():
    # bench.py generates its largest inputs with PyTorch (here on the CPU):
    # uniform draws bit for bit, log-uniform magnitudes within the last bit of exp2
    torch = pytest.importorskip("torch")
    for seed in (0, 3, 5 * 1000003 + 9, workload.B_STREAM_OFFSET):
        np.testing.assert_array_equal(workload.values_torch("uniform01", seed, 4096, "cpu").numpy(),
                                      workload.values("uniform01", seed, 4096))
        h = workload.values("loguniform20", seed, 4096)
        d = workload.values_torch("loguniform20", seed, 4096, "cpu").numpy()
        assert np.array_equal(np.sign(h), np.sign(d))
        assert np.max(np.abs(d - h) / np.abs(h)) <= 2.0 ** -51
    A, B = workload.pair_torch("uniform01", 7, 33, "cpu")
    hA, hB = workload.pair("uniform01", 7, 33)
    np.testing.assert_array_equal(A.numpy(), hA)
    np.testing.assert_array_equal(B.numpy(), hB)
    _ = torch
