"""Parity of the split-precision emulation (tcgen05 bf16 digit products) with the oracle.

Every step is compared through the C ABI with the oracle's model of the same
step: exponents and digits (a3/a4) and level sums (a5) bit for bit, the
recombination (a6) bit for bit, and the whole product bit for bit against
the model and within 2 N 2^-53 |A||B| of the plain FP64 product.

The emulated handles here run without the accuracy certificate
(MM_FLAG_NO_GUARD): it may send elements to native FP64, which the models do
not describe.  test_guard_gpu.py covers the guarded path.
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import U, assert_within_bound, componentwise_error, dev, host

pytestmark = pytest.mark.gpu


def handle(slices=7, mode="emulated", flags=0):
    import paper_1012_2273_gb300 as mm
    return mm.Handle(mode, slices=slices, flags=flags | mm.FLAG_NO_GUARD)


def bf16_planes_to_int(t):
    import torch
    torch.cuda.synchronize()
    return t.view(torch.bfloat16).float().cpu().numpy().astype(np.int64)


# ---- a3/a4: scale and split ----------------------------------------------------

@pytest.mark.parametrize("dist", ["uniform01", "loguniform20", "int8"])
@pytest.mark.parametrize("n,s", [(1, 1), (5, 3), (64, 7), (100, 8), (130, 2), (300, 7)])
def test_split_matches_model(dist, n, s):
    A, B = workload.pair(dist, 40 + n, n)
    A[n // 2] = 0.0  # a zero row
    with handle(s) as h:
        ea, da = h.split(dev(A), False, s)
        eb, db = h.split(dev(B), True, s)
        h.check()
    ea, eb = ea.cpu().numpy(), eb.cpu().numpy()
    np.testing.assert_array_equal(ea, oracle.emu_row_exponents(A))
    np.testing.assert_array_equal(eb, oracle.emu_col_exponents(B))
    da, db = bf16_planes_to_int(da), bf16_planes_to_int(db)
    want_a = oracle.emu_digit_planes(A, ea, s, False)
    want_b = oracle.emu_digit_planes(B, eb, s, True)  # [u][j][k]
    np.testing.assert_array_equal(da[:, :n, :n], want_a)
    np.testing.assert_array_equal(db[:, :n, :n], np.transpose(want_b, (0, 2, 1)))  # B^T planes: [u][k][j]
    assert not da[:, n:, :].any() and not da[:, :, n:].any()  # padding is zero
    assert not db[:, n:, :].any() and not db[:, :, n:].any()


# ---- a5: exact level sums on the tensor cores ----------------------------------

@pytest.mark.parametrize("n,s", [(64, 1), (100, 2), (129, 3), (257, 4), (300, 7), (520, 8)])
def test_level_sums_match_model(n, s):
    A, B = workload.pair("uniform11", 60 + n, n)
    with handle(s) as h:
        ea, da = h.split(dev(A), False, s)
        eb, db = h.split(dev(B), True, s, rows=-(-n // 256) * 256)
        S = h.level_sums(n, s, da, db)
        h.check()
    S = S.cpu().numpy().astype(np.int64)
    dA = oracle.emu_digit_planes(A, oracle.emu_row_exponents(A), s, False)
    dB = oracle.emu_digit_planes(B, oracle.emu_col_exponents(B), s, True)
    want = oracle.emu_level_sums(dA, dB)
    if not np.array_equal(S, want):
        bad = np.argwhere(S != want)
        L, i, k = bad[0]
        raise AssertionError(f"{len(bad)} level sums differ; first L={L + 2} ({i},{k}): got {S[L, i, k]} "
                             f"want {want[L, i, k]}; rows hit {np.unique(bad[:, 1])[:10]}, "
                             f"cols hit {np.unique(bad[:, 2])[:10]}")


def test_tensor_core_accumulation_is_exact_at_the_chunk_bound():
    # One 1024-deep chunk (n = 1024): top digits of magnitude up to 128 with
    # aligned signs drive its FP32 sums towards 2^24, the largest magnitude at
    # which every integer is an FP32 value; any rounding inside the tensor core
    # shows up here.  Row/column pairs 0-3 reach the bound exactly: 1024
    # products of 128 * 128 (+2^24 and -2^24), and 127 * 127 (every partial
    # sum after an odd number of products is odd and above 2^23).
    n, s = 1024, 1
    rng = np.random.default_rng(77)
    da = rng.integers(120, 129, (n, n)) * np.where(rng.random((n, n)) < 0.9, 1, -1)
    db = rng.integers(120, 129, (n, n)) * np.where(rng.random((n, n)) < 0.9, 1, -1)
    da[0, :], db[:, 0] = 128, 128
    da[1, :], db[:, 1] = -128, 128
    da[2, :], db[:, 2] = 127, 127
    da[3, :], db[:, 3] = -127, 127
    # x = d/128 (1 - 2^-40): every row and column maximum is below 1, so e = f = 0
    # and the single digit of x is d itself.
    A = da / 128.0 * (1 - 2.0 ** -40)
    B = db / 128.0 * (1 - 2.0 ** -40)
    with handle(s) as h:
        ea, dA = h.split(dev(A), False, s)
        eb, dB = h.split(dev(B), True, s)
        S = h.level_sums(n, s, dA, dB)
        h.check()
    want = oracle.emu_level_sums(oracle.emu_digit_planes(A, oracle.emu_row_exponents(A), s, False),
                                 oracle.emu_digit_planes(B, oracle.emu_col_exponents(B), s, True))
    got = S.cpu().numpy().astype(np.int64)
    assert want[0, 0, 0] == 2 ** 24 and want[0, 1, 1] == -2 ** 24 and want[0, 2, 2] == 1024 * 127 * 127
    assert np.abs(want).max() == 2 ** 24
    assert (np.abs(want) > 2 ** 23).mean() > 0.5  # most sums near the bound
    np.testing.assert_array_equal(got, want)


# ---- a6: recombination ------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 4, 7, 8])
def test_recombine_matches_model(s):
    import torch
    n = 70
    rng = np.random.default_rng(s)
    lv = rng.integers(-2 ** 31, 2 ** 31, (s, n, n)).astype(np.int32)
    lv[:, 0, :] = 0  # exact zeros
    e = rng.integers(-25, 26, n).astype(np.int32)
    f = rng.integers(-25, 26, n).astype(np.int32)
    e[5] = -1060  # subnormal results
    f[7] = -1100  # results that round to zero
    f[6] = 1000   # overflow to infinity for large entries
    with handle(s) as h:
        C = h.recombine(n, s, torch.from_numpy(lv).cuda(), torch.from_numpy(e).cuda(), torch.from_numpy(f).cuda())
        h.check()
    C = host(C)
    want = np.empty((n, n))
    for i in range(n):
        for k in range(n):
            want[i, k] = oracle.emu_combine(lv[:, i, k].astype(np.int64), s, int(e[i]), int(f[k]))
    np.testing.assert_array_equal(C.view(np.int64), want.view(np.int64))  # bit patterns, incl. signed zeros


# ---- whole emulated product -----------------------------------------------------

@pytest.mark.parametrize("n,s,dist", [(1, 7, "uniform01"), (7, 7, "uniform11"), (64, 7, "uniform01"),
                                      (100, 8, "loguniform20"), (129, 6, "uniform11"), (257, 7, "uniform01"),
                                      (300, 3, "uniform11"), (500, 7, "uniform01")])
def test_emulated_gemm_bit_exact_vs_model(n, s, dist):
    A, B = workload.pair(dist, 80 + n, n)
    with handle(s) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    want = oracle.emu_gemm(A, B, s)
    np.testing.assert_array_equal(C.view(np.int64), want.view(np.int64))


@pytest.mark.parametrize("n", [100, 500, 1000])
@pytest.mark.parametrize("dist", ["uniform01", "uniform11"])
def test_emulated_within_fp64_tolerance(n, dist):
    A, B = workload.pair(dist, 0, n)
    with handle(7) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    absAB = oracle.absgemm(A, B)
    assert_within_bound(C, oracle.gemm(A, B), absAB, n)
    assert componentwise_error(C, oracle.gemm_dot2(A, B), absAB) <= 2 * n * U


def test_emulated_loguniform_within_tolerance_with_eight_slices():
    n = 512
    A, B = workload.pair("loguniform20", 4, n)
    with handle(8) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    assert_within_bound(C, oracle.gemm_dot2(A, B), oracle.absgemm(A, B), n)


@pytest.mark.parametrize("n", [10, 100, 500, 1000, 1500, 2000])
def test_emulated_integer_inputs_bit_exact(n):
    A, B = workload.pair("int8", 7, n)
    with handle(1) as h:  # one slice holds every {-8..8} entry exactly
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(C, oracle.gemm(A, B))


@pytest.mark.parametrize("use_graph", [True, False])
def test_grouped_emulated_uneven_sizes(use_graph):
    import paper_1012_2273_gb300 as mm
    sizes = [130, 1, 64, 0, 300, 17, 257, 129]
    pairs = [workload.pair("uniform11", 90 + i, n) for i, n in enumerate(sizes)]
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    with handle(7, flags=0 if use_graph else mm.FLAG_NO_GRAPH) as h:
        for _ in range(2):
            Cs = h.gemm_grouped(As, Bs)
            h.check()
            for (A, B), C, n in zip(pairs, Cs, sizes):
                if n == 0:
                    continue
                want = oracle.emu_gemm(A, B, 7)
                np.testing.assert_array_equal(host(C).view(np.int64), want.view(np.int64))


@pytest.mark.parametrize("n", [2000, 4096])
def test_large_sizes_sampled_rows_and_freivalds(n):
    A, B = workload.pair("uniform11", 3, n)
    with handle(7) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    rows = [0, 1, n // 3, n // 2 + 1, n - 2, n - 1]
    want = oracle.emu_gemm_rows(A, B, 7, rows)
    np.testing.assert_array_equal(C[rows].view(np.int64), want.view(np.int64))
    ref_rows = oracle.gemm_rows(A, B, rows)
    absab = np.abs(A[rows]) @ np.abs(B)
    assert_within_bound(C[rows], ref_rows, absab, n)
    rng = np.random.default_rng(1)
    for _ in range(3):
        bad, _, _ = oracle.freivalds(A, B, C, rng.choice([-1.0, 1.0], n))
        assert bad == 0


def test_nonfinite_input_is_reported():
    import paper_1012_2273_gb300 as mm
    n = 64
    A, B = workload.pair("uniform01", 1, n)
    A[3, 4] = np.nan
    with handle(7) as h:
        h.gemm(dev(A), dev(B))
        with pytest.raises(mm.MMError) as ei:
            h.check()
        assert ei.value.code == 6
        h.check()  # the status word was cleared


def test_auto_plan_picks_native_small_digits_middle_modular_large():
    import paper_1012_2273_gb300 as mm
    with mm.Handle("auto") as h:
        assert h.plan(10)[0] == 0
        assert h.plan(600)[0] == 2
        assert h.plan(4096)[0] == 2  # modular form above


@pytest.mark.parametrize("groups", [1, 2, 5, 13, 28])
def test_forced_pair_groups_are_bit_exact(tmp_path, groups):
    # Units = (tile, pair group); any split of the 28 digit pairs (s = 7) must
    # give the same bits: the partial sums are integers, added exactly.
    import paper_1012_2273_gb300 as mm
    tune = tmp_path / "tune.txt"
    tune.write_text(f"# max_n form slices bn groups\n100000 1 7 256 {groups}\n")
    n = 300
    A, B = workload.pair("uniform11", 7, n)
    with mm.Handle("emulated", slices=7, flags=mm.FLAG_NO_GUARD, tune_path=str(tune)) as h:
        C = host(h.gemm(dev(A), dev(B)))
        sizes = [300, 64, 513]
        pairs = [workload.pair("uniform01", 20 + i, m) for i, m in enumerate(sizes)]
        Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
        h.check()
    want = oracle.emu_gemm(A, B, 7)
    np.testing.assert_array_equal(C.view(np.int64), want.view(np.int64))
    for (a, b), c in zip(pairs, Cs):
        np.testing.assert_array_equal(host(c).view(np.int64), oracle.emu_gemm(a, b, 7).view(np.int64))


def test_prepared_calls_give_the_same_bits():
    # Handle.grouped_call / gemm_call validate and marshal once and then call
    # the C ABI directly; repeated calls give the bits of the plain calls
    # (mixed native and emulated problems, a strided view for the single one).
    import torch
    import paper_1012_2273_gb300 as mm
    sizes = [10, 100, 300, 700]
    pairs = [workload.pair("uniform11", 40 + i, n) for i, n in enumerate(sizes)]
    with mm.Handle("auto") as h:
        want = [host(c) for c in h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])]
        As, Bs = [dev(a) for a, _ in pairs], [dev(b) for _, b in pairs]
        Cs = [torch.empty_like(a) for a in As]
        call = h.grouped_call(As, Bs, Cs)
        for _ in range(2):
            call()
            h.check()
            for w, c in zip(want, Cs):
                np.testing.assert_array_equal(host(c).view(np.int64), w.view(np.int64))
        big = torch.zeros((310, 305), dtype=torch.float64, device="cuda")
        A = big[5:, :300]  # a 305 x 300 view with leading dimension 305
        A.copy_(dev(pairs[2][0][:305, :300] if pairs[2][0].shape[0] >= 305 else np.vstack([pairs[2][0], pairs[2][0][:5]])))
        B = dev(pairs[2][1])
        C = torch.empty((305, 300), dtype=torch.float64, device="cuda")
        single = h.gemm_call(A, B, C)
        for _ in range(2):
            single()
            h.check()
            np.testing.assert_array_equal(host(C).view(np.int64), host(h.gemm(A, B)).view(np.int64))
