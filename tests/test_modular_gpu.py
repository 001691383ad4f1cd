"""Parity of the modular emulation form (residue products on the tcgen05 tensor
cores, Chinese-remainder recombination) with the oracle.

What the form computes has a plain definition -- one rounding of the exact
product of the operands rounded to beta-bit fixed point -- and the oracle
computes exactly that with 128-bit integers, so every comparison here is bit
for bit (plus the FP64 tolerance against the plain product where the width
allows it).  beta comes from the library's width rule, which the CPU tests
pin against the oracle's own statement of it.

The emulated handles here run without the accuracy certificate
(MM_FLAG_NO_GUARD): it may send elements to native FP64, which the models do
not describe.  test_guard_gpu.py covers the guarded path.
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import U, assert_within_bound, dev, host

pytestmark = pytest.mark.gpu


def handle(k=16, flags=0, tune_path=None):
    import paper_1012_2273_gb300 as mm
    return mm.Handle("modular", slices=k, flags=flags | mm.FLAG_NO_GUARD, tune_path=tune_path)


def beta_of(k, n):
    b = oracle.modular_beta(k, n)
    assert b > 0
    return b


def assert_bits(C, want):
    np.testing.assert_array_equal(np.asarray(C).view(np.int64), np.asarray(want).view(np.int64))


@pytest.mark.parametrize("dist", ["uniform11", "loguniform20"])
@pytest.mark.parametrize("n", [1, 7, 63, 64, 65, 127, 128, 129, 200, 255, 256, 257, 300, 511, 640])
def test_modular_bit_exact_vs_fixed_point_product(n, dist):
    A, B = workload.pair(dist, 500 + n, n)
    with handle(16) as h:
        assert h.plan(n) == (2, 16)
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    assert_bits(C, oracle.fixed_gemm(A, B, beta_of(16, n)))


@pytest.mark.parametrize("k", [2, 3, 5, 8, 11, 13, 14, 15])
def test_modular_every_moduli_count(k):
    n = 300
    A, B = workload.pair("uniform11", 70 + k, n)
    with handle(k) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    assert_bits(C, oracle.fixed_gemm(A, B, beta_of(k, n)))


def test_modular_zero_rows_columns_and_matrices():
    n = 200
    A, B = workload.pair("uniform11", 9, n)
    A[5, :] = 0.0
    A[:, 17] = 0.0
    B[:, 33] = -0.0
    B[150, :] = 0.0
    with handle(16) as h:
        C = host(h.gemm(dev(A), dev(B)))
        Z = host(h.gemm(dev(np.zeros((n, n))), dev(B)))
        h.check()
    assert_bits(C, oracle.fixed_gemm(A, B, beta_of(16, n)))
    assert np.all(C[5, :] == 0) and np.all(C[:, 33] == 0)
    assert np.all(Z == 0) and not np.signbit(Z).any()


@pytest.mark.parametrize("n", [40, 333, 1000])
def test_modular_integer_inputs_are_exact(n):
    A, B = workload.pair("int8", 21, n)
    with handle(16) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("n", [1000, 2000])
@pytest.mark.parametrize("dist", ["uniform11", "uniform01"])
def test_modular_within_fp64_tolerance(n, dist):
    A, B = workload.pair(dist, 31, n)
    with handle(16) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    if n <= 1000:
        assert_bits(C, oracle.fixed_gemm(A, B, beta_of(16, n)))
        assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)
    else:
        rows = [0, 1, n // 2, n - 1]
        assert_bits(C[rows], oracle.fixed_gemm_rows(A, B, beta_of(16, n), rows))
        assert_within_bound(C[rows], oracle.gemm_rows(A, B, rows), np.abs(A[rows]) @ np.abs(B), n)


@pytest.mark.parametrize("bn", [128, 256])
@pytest.mark.parametrize("groups", [1, 3, 16])
def test_modular_tile_widths_and_forced_groups(tmp_path, bn, groups):
    # Units = (tile, group of moduli); every split gives the same bits.
    tune = tmp_path / "tune.txt"
    tune.write_text(f"100000 2 16 {bn} {groups}\n")
    n = 520
    A, B = workload.pair("loguniform20", 8, n)
    with handle(16, tune_path=str(tune)) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    assert_bits(C, oracle.fixed_gemm(A, B, beta_of(16, n)))


@pytest.mark.parametrize("use_graph", [True, False])
def test_modular_grouped_uneven_sizes_and_moduli(tmp_path, use_graph):
    # One launch holds problems with different moduli counts (per-size rows of
    # the tune table) and some native ones.
    import paper_1012_2273_gb300 as mm
    tune = tmp_path / "tune.txt"
    tune.write_text("40 0 7 256 0\n200 2 14 256 0\n400 2 15 256 0\n100000 2 16 256 0\n")
    sizes = [130, 1, 64, 0, 300, 17, 257, 129, 700, 33]
    pairs = [workload.pair("uniform11", 90 + i, n) for i, n in enumerate(sizes)]
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    flags = 0 if use_graph else mm.FLAG_NO_GRAPH
    with mm.Handle("auto", flags=flags | mm.FLAG_NO_GUARD, tune_path=str(tune)) as h:
        plans = {n: h.plan(n) for n in sizes if n}
        for _ in range(2):
            Cs = h.gemm_grouped(As, Bs)
            h.check()
            for (A, B), C, n in zip(pairs, Cs, sizes):
                if n == 0:
                    continue
                form, k = plans[n]
                if form == 0:
                    assert_within_bound(host(C), oracle.gemm(A, B), oracle.absgemm(A, B), n)
                else:
                    assert form == 2
                    assert_bits(host(C), oracle.fixed_gemm(A, B, beta_of(k, n)))
    assert plans[300] == (2, 15) and plans[130] == (2, 14) and plans[700] == (2, 16)


def test_modular_grouped_batch_matches_single_calls():
    sizes = workload.loguniform_sizes(48, 10, 700, seed=4)
    pairs = workload.batch("uniform01", 4, sizes)
    with handle(16) as h:
        Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
        h.check()
    for (A, B), C, n in zip(pairs, Cs, sizes):
        assert_bits(host(C), oracle.fixed_gemm(A, B, beta_of(16, n)))


@pytest.mark.parametrize("n", [4096])
def test_modular_large_sampled_rows_and_freivalds(n):
    A, B = workload.pair("loguniform20", 12, n)
    with handle(16) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    rows = [0, 1, n // 3, n // 2 + 1, n - 2, n - 1]
    assert_bits(C[rows], oracle.fixed_gemm_rows(A, B, beta_of(16, n), rows))
    rng = np.random.default_rng(1)
    for _ in range(3):
        bad, _, _ = oracle.freivalds(A, B, C, rng.choice([-1.0, 1.0], n))
        assert bad == 0


def test_modular_precision_grows_with_moduli():
    # More moduli allow a wider fixed point: the error against the plain
    # product shrinks until it meets the FP64 bound (uniform entries).
    n = 1000
    A, B = workload.pair("uniform11", 3, n)
    rows = [0, 500, 999]
    ref = oracle.gemm_rows(A, B, rows)
    absab = np.abs(A[rows]) @ np.abs(B)
    errs = []
    for k in (8, 10, 12, 14, 16):
        with handle(k) as h:
            C = host(h.gemm(dev(A), dev(B)))
            h.check()
        errs.append(float(np.max(np.abs(C[rows] - ref) / absab)))
    assert all(b < a for a, b in zip(errs, errs[1:]) if a > 4 * n * U), errs
    assert errs[0] > 2 * n * U >= errs[-1], errs


def test_modular_nonfinite_input_is_reported():
    import paper_1012_2273_gb300 as mm
    n = 64
    A, B = workload.pair("uniform01", 1, n)
    B[3, 4] = np.inf
    with handle(16) as h:
        h.gemm(dev(A), dev(B))
        with pytest.raises(mm.MMError) as ei:
            h.check()
        assert ei.value.code == 6
        h.check()


def test_modular_rejects_too_few_moduli_and_bad_counts():
    import paper_1012_2273_gb300 as mm
    with pytest.raises(mm.MMError):
        mm.Handle("modular", slices=17)
    with pytest.raises(mm.MMError):
        mm.Handle("modular", slices=1)
    import torch
    n = 8129  # the smallest size at which two moduli leave no fixed-point width
    assert oracle.modular_beta(2, n) == 0 and oracle.modular_beta(2, n - 1) == 1
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    with handle(2) as h:
        with pytest.raises(mm.MMError) as ei:
            h.gemm(A, A)
        assert ei.value.code == 4


@pytest.mark.parametrize("use_graph", [True, False])
def test_grouped_call_mixing_native_digit_and_modular_forms(tmp_path, use_graph):
    # Three forms in one grouped call: native FP64, the digit form (its own
    # launch group) and the modular form (another), one after another on the
    # call's stream, each problem bit-exact against its form's model.
    import paper_1012_2273_gb300 as mm
    tune = tmp_path / "tune.txt"
    tune.write_text("60 0 7 256 0\n300 1 7 256 0\n100000 2 15 256 0\n")
    sizes = [700, 40, 250, 1, 129, 513, 300, 64]
    pairs = [workload.pair("uniform11", 150 + i, n) for i, n in enumerate(sizes)]
    flags = 0 if use_graph else mm.FLAG_NO_GRAPH
    with mm.Handle("auto", flags=flags | mm.FLAG_NO_GUARD, tune_path=str(tune)) as h:
        plans = {n: h.plan(n) for n in sizes}
        for _ in range(2):
            Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
            h.check()
            for (A, B), C, n in zip(pairs, Cs, sizes):
                form, k = plans[n]
                C = host(C)
                if form == 0:
                    assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)
                elif form == 1:
                    assert_bits(C, oracle.emu_gemm(A, B, k))
                else:
                    assert_bits(C, oracle.fixed_gemm(A, B, beta_of(k, n)))
    assert {f for f, _ in plans.values()} == {0, 1, 2}


@pytest.mark.parametrize("pair", ["1", "0"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_modular_cta_pair_kernel_bit_exact(tmp_path, monkeypatch, use_graph, pair):
    # The paired kernel (two CTAs per 256 x 256 tile, the default at tile
    # width 256) and the single-CTA kernel (MM_PAIR_MMA=0) compute the same
    # residue products: single problems (rows padded to 256 for pairs) and a
    # grouped call with uneven sizes and moduli counts, bit for bit.
    import paper_1012_2273_gb300 as mm
    monkeypatch.setenv("MM_PAIR_MMA", pair)
    tune = tmp_path / "tune.txt"
    tune.write_text("300 2 14 256 0\n700 2 15 256 0\n100000 2 16 256 0\n")
    flags = 0 if use_graph else mm.FLAG_NO_GRAPH
    sizes = [1, 129, 257, 300, 385, 640, 1000]
    pairs = [workload.pair("loguniform20", 60 + i, n) for i, n in enumerate(sizes)]
    with mm.Handle("auto", flags=flags | mm.FLAG_NO_GUARD, tune_path=str(tune)) as h:
        plans = {n: h.plan(n) for n in sizes}
        for (A, B), n in zip(pairs[:3], sizes[:3]):
            C = host(h.gemm(dev(A), dev(B)))
            h.check()
            form, k = plans[n]
            if form == 2:
                assert_bits(C, oracle.fixed_gemm(A, B, beta_of(k, n)))
        Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
        h.check()
    for (A, B), C, n in zip(pairs, Cs, sizes):
        form, k = plans[n]
        C = host(C)
        if form == 2:
            assert_bits(C, oracle.fixed_gemm(A, B, beta_of(k, n)))
        else:
            assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)
    assert plans[1000] == (2, 16) and plans[300] == (2, 14)


@pytest.mark.parametrize("pair", ["1", "0"])
def test_modular_cta_pairs_beside_the_certificate(tmp_path, monkeypatch, pair):
    # With the accuracy certificate on, the residue products (CTA pairs or
    # single CTAs) run beside the certificate's own launch, which keeps
    # single-CTA tiles with tensor maps of its own.  Uniform inputs pass the
    # certificate everywhere, so the results are the model's bits and nothing
    # is recomputed; grouped (graph and no graph) and single calls.
    import paper_1012_2273_gb300 as mm
    monkeypatch.setenv("MM_PAIR_MMA", pair)
    tune = tmp_path / "tune.txt"
    tune.write_text("300 2 15 256 0\n100000 2 16 256 0\n")
    sizes = [129, 300, 385, 640, 1000, 1500]
    pairs = [workload.pair("uniform11", 80 + i, n) for i, n in enumerate(sizes)]
    for flags in (0, mm.FLAG_NO_GRAPH):
        with mm.Handle("auto", flags=flags, tune_path=str(tune)) as h:
            plans = {n: h.plan(n) for n in sizes}
            A, B = pairs[3]
            C1 = host(h.gemm(dev(A), dev(B)))
            Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
            h.check()
            assert h.guard_read() == (0, 0)
        k = plans[640][1]
        assert_bits(C1, oracle.fixed_gemm(A, B, beta_of(k, 640)))
        for (A, B), C, n in zip(pairs, Cs, sizes):
            form, k = plans[n]
            assert form == 2
            assert_bits(host(C), oracle.fixed_gemm(A, B, beta_of(k, n)))
