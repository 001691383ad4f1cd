"""Rectangular products C (m x n) = A (m x k) . B (k x n) through mm_gemm_ex and
mm_gemm_grouped_ex, against the oracle's rectangular functions: the native
form within 2 k u |A||B| of the left-to-right sum, the modular and digit
forms bit for bit against their models, with leading dimensions (views into
larger arrays, whose other elements must stay untouched), K = 0, empty
shapes and argument checks.

The emulated handles here run without the accuracy certificate
(MM_FLAG_NO_GUARD): it may send elements to native FP64, which the models do
not describe.  test_guard_gpu.py covers the guarded path.
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import assert_within_bound, dev, host

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (1, 300, 77), (300, 1, 77), (7, 300, 45), (300, 7, 45), (129, 257, 513), (640, 64, 1000),
          (1000, 520, 37), (64, 700, 640), (257, 129, 3)]


def handle(mode="auto", slices=0, flags=0, **kw):
    import paper_1012_2273_gb300 as mm
    return mm.Handle(mode, slices=slices, flags=flags | mm.FLAG_NO_GUARD, **kw)


def bits(C):
    return np.asarray(C).view(np.int64)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_native_rect_within_bound(m, n, k):
    A, B = workload.rect_pair("uniform11", 3 * m + n, m, n, k)
    with handle("native") as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    assert C.shape == (m, n)
    assert_within_bound(C, oracle.gemm_mnk(A, B), oracle.absgemm_mnk(A, B), k)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_modular_rect_bit_exact(m, n, k):
    A, B = workload.rect_pair("loguniform20", 5 * m + k, m, n, k)
    with handle("modular", 16) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    beta = oracle.modular_beta(16, k)
    np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm_mnk(A, B, beta)))


@pytest.mark.parametrize("m,n,k", SHAPES[:7])
def test_digit_rect_bit_exact(m, n, k):
    A, B = workload.rect_pair("uniform11", 11 * n + k, m, n, k)
    with handle("emulated", 7) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(bits(C), bits(oracle.emu_gemm_mnk(A, B, 7)))


@pytest.mark.parametrize("mode,slices", [("native", 0), ("modular", 14), ("emulated", 3)])
def test_rect_integer_inputs_exact_in_every_form(mode, slices):
    m, n, k = 333, 129, 700
    A, B = workload.rect_pair("int8", 9, m, n, k)
    with handle(mode, slices) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("mode,slices", [("native", 0), ("modular", 16), ("emulated", 7), ("auto", 0)])
def test_rect_views_with_leading_dimensions(mode, slices):
    # A, B, C are windows of larger arrays (row strides > row lengths, odd
    # offsets: 8- but not 16-byte aligned); everything outside C's window
    # must keep its sentinel value.
    import torch
    m, n, k = 201, 150, 333
    A, B = workload.rect_pair("uniform11", 4, m, n, k)
    bigA = torch.full((m + 5, k + 7), 7.0, dtype=torch.float64, device="cuda")
    bigB = torch.full((k + 3, n + 9), -3.0, dtype=torch.float64, device="cuda")
    bigC = torch.full((m + 4, n + 11), 123.0, dtype=torch.float64, device="cuda")
    vA = bigA[2:2 + m, 3:3 + k]
    vB = bigB[1:1 + k, 5:5 + n]
    vC = bigC[3:3 + m, 1:1 + n]
    vA.copy_(torch.from_numpy(A))
    vB.copy_(torch.from_numpy(B))
    with handle(mode, slices) as h:
        h.gemm(vA, vB, vC)
        h.check()
    got = host(bigC)
    C = got[3:3 + m, 1:1 + n]
    outside = np.ones(got.shape, bool)
    outside[3:3 + m, 1:1 + n] = False
    assert np.all(got[outside] == 123.0)
    if mode == "modular":
        np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm_mnk(A, B, oracle.modular_beta(16, k))))
    elif mode == "emulated":
        np.testing.assert_array_equal(bits(C), bits(oracle.emu_gemm_mnk(A, B, 7)))
    else:
        assert_within_bound(C, oracle.gemm_mnk(A, B), oracle.absgemm_mnk(A, B), k)


@pytest.mark.parametrize("mode,slices", [("native", 0), ("modular", 16), ("emulated", 7)])
def test_rect_zero_inner_dimension_and_empty_shapes(mode, slices):
    import torch
    with handle(mode, slices) as h:
        A = torch.empty((50, 0), dtype=torch.float64, device="cuda")
        B = torch.empty((0, 70), dtype=torch.float64, device="cuda")
        C = torch.full((50, 70), 5.0, dtype=torch.float64, device="cuda")
        h.gemm(A, B, C)
        h.check()
        assert torch.all(C == 0) and not torch.signbit(C).any()
        E = h.gemm(torch.empty((0, 9), dtype=torch.float64, device="cuda"),
                   torch.ones((9, 4), dtype=torch.float64, device="cuda"))
        h.check()
        assert tuple(E.shape) == (0, 4)


@pytest.mark.parametrize("use_graph", [True, False])
def test_grouped_rect_mixed_shapes_forms_and_views(tmp_path, use_graph):
    import torch
    import paper_1012_2273_gb300 as mm
    tune = tmp_path / "tune.txt"
    tune.write_text("60 0 7 256 0\n300 1 7 256 0\n100000 2 15 256 0\n")
    shapes = [(700, 300, 513), (40, 500, 20), (250, 250, 250), (1, 1000, 64), (129, 5, 900), (512, 640, 300),
              (60, 61, 59), (30, 20, 50), (0, 10, 10), (10, 10, 0)]
    pairs = [workload.rect_pair("uniform11", 40 + i, m, n, k) for i, (m, n, k) in enumerate(shapes)]
    As, Bs, Cs = [], [], []
    for i, ((A, B), (m, n, k)) in enumerate(zip(pairs, shapes)):
        if i % 2:  # every other problem as a strided view
            bA = torch.zeros((m + 1, k + 3), dtype=torch.float64, device="cuda")
            bA[1:, 3:].copy_(torch.from_numpy(A))
            As.append(bA[1:, 3:])
        else:
            As.append(dev(A))
        Bs.append(dev(B))
        Cs.append(torch.full((m, n), 9.0, dtype=torch.float64, device="cuda"))
    flags = 0 if use_graph else mm.FLAG_NO_GRAPH
    with mm.Handle("auto", flags=flags | mm.FLAG_NO_GUARD, tune_path=str(tune)) as h:
        plans = {s: h.plan(max(s)) for s in shapes if min(s[:2]) > 0}
        for _ in range(2):
            h.gemm_grouped(As, Bs, Cs)
            h.check()
            for (A, B), C, s in zip(pairs, Cs, shapes):
                m, n, k = s
                C = host(C)
                if m == 0 or n == 0:
                    continue
                if k == 0:
                    assert np.all(C == 0)
                    continue
                form, sl = plans[s]
                if form == 0:
                    assert_within_bound(C, oracle.gemm_mnk(A, B), oracle.absgemm_mnk(A, B), k)
                elif form == 1:
                    np.testing.assert_array_equal(bits(C), bits(oracle.emu_gemm_mnk(A, B, sl)))
                else:
                    np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm_mnk(A, B, oracle.modular_beta(sl, k))))
    assert {f for f, _ in plans.values()} == {0, 1, 2}


def test_rect_argument_checks():
    import torch
    import paper_1012_2273_gb300 as mm
    L = mm.lib()
    A = torch.zeros((8, 6), dtype=torch.float64, device="cuda")
    B = torch.zeros((6, 5), dtype=torch.float64, device="cuda")
    C = torch.zeros((8, 5), dtype=torch.float64, device="cuda")
    with handle("native") as h:
        hp = h._h
        a, b, c = A.data_ptr(), B.data_ptr(), C.data_ptr()
        assert L.mm_gemm_ex(hp, 0, 0, 8, 5, 6, a, 5, b, 5, c, 5, None) == 1  # lda < K
        assert L.mm_gemm_ex(hp, 0, 0, 8, 5, 6, a, 6, b, 4, c, 5, None) == 1  # ldb < N
        assert L.mm_gemm_ex(hp, 0, 0, 8, 5, 6, a, 6, b, 5, c, 4, None) == 1  # ldc < N
        assert L.mm_gemm_ex(hp, 0, 0, -1, 5, 6, a, 6, b, 5, c, 5, None) == 1
        assert L.mm_gemm_ex(hp, 0, 0, 8, 5, 6, a + 4, 6, b, 5, c, 5, None) == 1  # misaligned
        assert L.mm_gemm_ex(hp, 0, 0, 8, 5, 6, a, 6, b, 5, a, 5, None) == 1  # C overlaps A
        assert L.mm_gemm_ex(hp, 0, 0, 0, 5, 6, None, 6, None, 5, None, 5, None) == 0  # M = 0: no-op
        with pytest.raises(ValueError):
            h.gemm(A, torch.zeros((5, 5), dtype=torch.float64, device="cuda"))
        h.check()


def test_rect_large_sampled_rows(tmp_path):
    # auto plan at size max(m, n, k) = 3000: modular; rows checked against the model
    m, n, k = 3000, 1800, 1300
    A, B = workload.rect_pair("loguniform20", 77, m, n, k)
    with handle("auto") as h:
        form, sl = h.plan(max(m, n, k))
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    assert form == 2
    rows = [0, 1, m // 2, m - 1]
    np.testing.assert_array_equal(bits(C[rows]), bits(oracle.fixed_gemm_mnk(A, B, oracle.modular_beta(sl, k), rows=rows)))
    rng = np.random.default_rng(3)
    x = rng.choice([-1.0, 1.0], n)
    y = A @ (B @ x) - C @ x
    tol = 4 * k * 2.0 ** -53 * (np.abs(A) @ (np.abs(B) @ np.abs(x)) + np.abs(C) @ np.abs(x))
    assert np.all(np.abs(y) <= tol)


@pytest.mark.parametrize("pair", ["1", "0"])
def test_rect_cta_pair_kernel(monkeypatch, pair):
    monkeypatch.setenv("MM_PAIR_MMA", pair)
    m, n, k = 700, 513, 900  # m padded to 768 rows (three 256-row pair tiles)
    A, B = workload.rect_pair("uniform11", 31, m, n, k)
    with handle("modular", 15) as h:
        C = host(h.gemm(dev(A), dev(B)))
        h.check()
    np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm_mnk(A, B, oracle.modular_beta(15, k))))


def stored(X, transposed, pad_rows=0, pad_cols=0):
    """Device operand for op() = X: X itself, or the transpose of a stored X^T
    (passed as a .T view), optionally as a window of a larger array."""
    import torch
    S = np.ascontiguousarray(X.T) if transposed else X
    big = torch.full((S.shape[0] + pad_rows, S.shape[1] + pad_cols), 11.0, dtype=torch.float64, device="cuda")
    win = big[pad_rows:, pad_cols:]
    win.copy_(torch.from_numpy(S))
    return win.T if transposed else win


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("mode,slices", [("native", 0), ("modular", 16), ("emulated", 7)])
def test_rect_transposed_operands(mode, slices, ta, tb):
    m, n, k = 300, 129, 257
    A, B = workload.rect_pair("loguniform20" if mode == "modular" else "uniform11", 50 + 2 * ta + tb, m, n, k)
    dA = stored(A, ta, pad_rows=1, pad_cols=3)
    dB = stored(B, tb, pad_rows=2, pad_cols=1)
    assert (dA.stride(0) == 1) == bool(ta) and (dB.stride(0) == 1) == bool(tb)
    with handle(mode, slices) as h:
        C = host(h.gemm(dA, dB))
        h.check()
    if mode == "modular":
        np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm_mnk(A, B, oracle.modular_beta(16, k))))
    elif mode == "emulated":
        np.testing.assert_array_equal(bits(C), bits(oracle.emu_gemm_mnk(A, B, 7)))
    else:
        assert_within_bound(C, oracle.gemm_mnk(A, B), oracle.absgemm_mnk(A, B), k)


def test_native_transposes_give_the_same_bits():
    # the native kernel sums each output in the same k order whatever the storage
    m, n, k = 517, 300, 200
    A, B = workload.rect_pair("uniform11", 8, m, n, k)
    with handle("native") as h:
        ref = host(h.gemm(dev(A), dev(B)))
        for ta in (0, 1):
            for tb in (0, 1):
                C = host(h.gemm(stored(A, ta), stored(B, tb)))
                np.testing.assert_array_equal(bits(C), bits(ref))
        h.check()


def test_grouped_with_transposed_operands(tmp_path):
    tune = tmp_path / "tune.txt"
    tune.write_text("60 0 7 256 0\n300 1 7 256 0\n100000 2 15 256 0\n")
    import paper_1012_2273_gb300 as mm
    shapes = [(700, 300, 513), (250, 250, 250), (30, 20, 50), (129, 257, 640), (64, 64, 1)]
    pairs = [workload.rect_pair("uniform11", 70 + i, *s[:2], s[2]) for i, s in enumerate(shapes)]
    As = [stored(A, i % 2) for i, (A, _) in enumerate(pairs)]
    Bs = [stored(B, (i // 2) % 2) for i, (_, B) in enumerate(pairs)]
    with mm.Handle("auto", flags=mm.FLAG_NO_GUARD, tune_path=str(tune)) as h:
        plans = {s: h.plan(max(s)) for s in shapes}
        Cs = h.gemm_grouped(As, Bs)
        h.check()
    for (A, B), C, s in zip(pairs, Cs, shapes):
        form, sl = plans[s]
        C = host(C)
        k = s[2]
        if form == 0:
            assert_within_bound(C, oracle.gemm_mnk(A, B), oracle.absgemm_mnk(A, B), k)
        elif form == 1:
            np.testing.assert_array_equal(bits(C), bits(oracle.emu_gemm_mnk(A, B, sl)))
        else:
            np.testing.assert_array_equal(bits(C), bits(oracle.fixed_gemm_mnk(A, B, oracle.modular_beta(sl, k))))


def test_transposed_argument_checks():
    import torch
    import paper_1012_2273_gb300 as mm
    L = mm.lib()
    A = torch.zeros((6, 8), dtype=torch.float64, device="cuda")  # stored K x M for op(A) = A^T, M = 8, K = 6
    B = torch.zeros((5, 6), dtype=torch.float64, device="cuda")  # stored N x K for op(B) = B^T
    C = torch.zeros((8, 5), dtype=torch.float64, device="cuda")
    with handle("native") as h:
        hp = h._h
        a, b, c = A.data_ptr(), B.data_ptr(), C.data_ptr()
        assert L.mm_gemm_ex(hp, 1, 1, 8, 5, 6, a, 8, b, 6, c, 5, None) == 0
        h.check()
        assert L.mm_gemm_ex(hp, 2, 0, 8, 5, 6, a, 8, b, 6, c, 5, None) == 1  # flag not 0/1
        assert L.mm_gemm_ex(hp, 1, 1, 8, 5, 6, a, 7, b, 6, c, 5, None) == 1  # lda < M for a stored K x M
        assert L.mm_gemm_ex(hp, 1, 1, 8, 5, 6, a, 8, b, 5, c, 5, None) == 1  # ldb < K for a stored N x K
        with pytest.raises(ValueError):
            h.gemm(A.T, B.T, C[:, :4])
        h.check()
