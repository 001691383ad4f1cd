"""Parity at the benchmark configurations (paper sweep, precision study, grouped batch).

Full products are compared with the oracle where the oracle finishes in
seconds; larger ones are checked on rows the oracle computes one by one and
with Freivalds' test on the whole result.  Errors are componentwise,
|C - C_ref| / (|A||B|), against the bound 2 N 2^-53.  The precision study
reports each slice or moduli count twice: the raw emulation
(MM_FLAG_NO_GUARD) and the library's default, where the accuracy certificate
sends what it cannot vouch for to native FP64 (with the share it sent).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workload
from helpers import U, assert_within_bound, dev, host

pytestmark = pytest.mark.gpu

REPORT_DIR = os.environ.get("MM_REPORT_DIR")


def report(name, payload):
    if REPORT_DIR:
        os.makedirs(REPORT_DIR, exist_ok=True)
        with open(os.path.join(REPORT_DIR, name), "w") as f:
            json.dump(payload, f, indent=1)


def rows_of(n, k=6):
    return sorted({0, 1, n // 3, n // 2, n - 2, n - 1} | set(range(0, n, max(1, n // k))))[: k + 6]


def check_rows(C, A, B, n, factor=2.0):
    r = rows_of(n)
    ref = oracle.gemm_rows(A, B, r)
    absab = np.abs(A[r]) @ np.abs(B)
    assert_within_bound(C[r], ref, absab, n, factor)
    return r


# ---- paper sweep: N = 10 .. 2000, uniform [0, 1) and integers {-8..8} ---------

@pytest.mark.parametrize("form", ["native", "emulated", "modular", "auto"])
def test_paper_sweep_both_forms(form):
    import paper_1012_2273_gb300 as mm
    with mm.Handle(form) as h:
        for n in workload.SWEEP_SIZES:
            A, B = workload.pair("uniform01", 0, n)
            C = host(h.gemm(dev(A), dev(B)))
            h.check()
            if n <= 1000:
                assert_within_bound(C, oracle.gemm(A, B), oracle.absgemm(A, B), n)
            else:
                check_rows(C, A, B, n)
                bad, _, _ = oracle.freivalds(A, B, C, np.random.default_rng(n).choice([-1.0, 1.0], n))
                assert bad == 0
            Ai, Bi = workload.pair("int8", 0, n)
            Ci = host(h.gemm(dev(Ai), dev(Bi)))
            want = (Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64)
            np.testing.assert_array_equal(Ci, want)


# ---- precision study: error per slice count ---------------------------------------

def test_precision_per_slice_count_n2000():
    import paper_1012_2273_gb300 as mm
    n = 2000
    out = {"N": n, "bound_2Nu": 2 * n * U, "rows": {}}
    for dist in ("uniform11", "loguniform20"):
        A, B = workload.pair(dist, 3, n)
        r = rows_of(n, 10)
        ref = oracle.gemm_rows(A, B, r)
        absab = np.abs(A[r]) @ np.abs(B)
        errs = {}
        with mm.Handle("native") as h:
            C = host(h.gemm(dev(A), dev(B)))
        errs["native"] = float(np.max(np.abs(C[r] - ref) / absab))
        guarded = {}
        for s in range(2, 9):
            with mm.Handle("emulated", slices=s, flags=mm.FLAG_NO_GUARD) as h:
                C = host(h.gemm(dev(A), dev(B)))
                h.check()
            errs[f"s={s}"] = float(np.max(np.abs(C[r] - ref) / absab))
            with mm.Handle("emulated", slices=s) as h:
                C = host(h.gemm(dev(A), dev(B)))
                h.check()
                replaced, _ = h.guard_read()
            e = float(np.max(np.abs(C[r] - ref) / absab))
            guarded[f"s={s}"] = {"error": e, "replaced_fraction": replaced / (n * n)}
            assert e <= 2 * n * U  # the certificate holds whatever s is
        out["rows"][dist] = errs
        out.setdefault("guarded", {})[dist] = guarded
        # More slices never make the result worse by more than rounding.
        seq = [errs[f"s={s}"] for s in range(2, 9)]
        assert all(b <= a * 1.01 + 2 * n * U for a, b in zip(seq, seq[1:])), seq
        assert errs["native"] <= 2 * n * U
        if dist == "uniform11":
            assert errs["s=7"] <= 2 * n * U
            assert errs["s=3"] > 2 * n * U  # three bf16 slices: about FP32 accuracy, not FP64
        else:
            assert errs["s=8"] <= 2 * n * U
    report("precision_n2000.json", out)


def test_precision_per_moduli_count_n2000():
    # The modular form: error against the plain product per moduli count k
    # (fixed-point width beta from the width rule).
    import paper_1012_2273_gb300 as mm
    n = 2000
    out = {"N": n, "bound_2Nu": 2 * n * U, "rows": {}}
    for dist in ("uniform11", "loguniform20"):
        A, B = workload.pair(dist, 3, n)
        r = rows_of(n, 10)
        ref = oracle.gemm_rows(A, B, r)
        absab = np.abs(A[r]) @ np.abs(B)
        errs, guarded = {}, {}
        for k in range(8, 17):
            with mm.Handle("modular", slices=k) as h:
                Cg = host(h.gemm(dev(A), dev(B)))
                h.check()
                replaced, _ = h.guard_read()
            e = float(np.max(np.abs(Cg[r] - ref) / absab))
            guarded[f"k={k}"] = {"error": e, "replaced_fraction": replaced / (n * n)}
            assert e <= 2 * n * U
            with mm.Handle("modular", slices=k, flags=mm.FLAG_NO_GUARD) as h:
                C = host(h.gemm(dev(A), dev(B)))
                h.check()
            errs[f"k={k} beta={oracle.modular_beta(k, n)}"] = float(np.max(np.abs(C[r] - ref) / absab))
            if k == 16:
                np.testing.assert_array_equal(C[r[:2]].view(np.int64),
                                              oracle.fixed_gemm_rows(A, B, oracle.modular_beta(k, n), r[:2]).view(np.int64))
        out["rows"][dist] = errs
        out.setdefault("guarded", {})[dist] = guarded
        seq = list(errs.values())
        assert all(b <= a * 1.01 + 2 * n * U for a, b in zip(seq, seq[1:])), seq
        assert seq[-2] <= 2 * n * U and seq[-1] <= 2 * n * U  # 15 and 16 moduli
        assert seq[0] > 2 * n * U  # 8 moduli: about 25 bits
    report("precision_modular_n2000.json", out)


def test_precision_per_int8_slice_count_n2000():
    # The INT8 slice form (signed-byte digits of the (8s - 2)-bit value,
    # int32 accumulation): error against the plain product per digit count,
    # raw and with the certificate (and the share it sent to native FP64).
    import paper_1012_2273_gb300 as mm
    n = 2000
    out = {"N": n, "bound_2Nu": 2 * n * U, "rows": {}, "guarded": {}}
    for dist in ("uniform11", "loguniform20"):
        A, B = workload.pair(dist, 3, n)
        r = rows_of(n, 10)
        ref = oracle.gemm_rows(A, B, r)
        absab = np.abs(A[r]) @ np.abs(B)
        errs, guarded = {}, {}
        for s in range(2, 9):
            with mm.Handle("int8", slices=s, flags=mm.FLAG_NO_GUARD) as h:
                C = host(h.gemm(dev(A), dev(B)))
                h.check()
            errs[f"s={s}"] = float(np.max(np.abs(C[r] - ref) / absab))
            if s == 8:
                np.testing.assert_array_equal(C[r[:2]].view(np.int64), oracle.i8_gemm(A, B, s, rows=r[:2]).view(np.int64))
            with mm.Handle("int8", slices=s) as h:
                Cg = host(h.gemm(dev(A), dev(B)))
                h.check()
                replaced, _ = h.guard_read()
            e = float(np.max(np.abs(Cg[r] - ref) / absab))
            guarded[f"s={s}"] = {"error": e, "replaced_fraction": replaced / (n * n)}
            assert e <= 2 * n * U
        out["rows"][dist] = errs
        out["guarded"][dist] = guarded
        seq = [errs[f"s={s}"] for s in range(2, 9)]
        assert all(b <= a * 1.01 + 2 * n * U for a, b in zip(seq, seq[1:])), seq
        assert errs["s=8"] <= 2 * n * U
    report("precision_int8_n2000.json", out)


@pytest.mark.parametrize("n", [4096, 8192])
def test_precision_large_sizes_rows(n):
    import paper_1012_2273_gb300 as mm
    out = {"N": n, "bound_2Nu": 2 * n * U, "rows": {}}
    for dist, s in (("uniform11", 7), ("loguniform20", 8)):
        A, B = workload.pair(dist, 5, n)
        with mm.Handle("emulated", slices=s, flags=mm.FLAG_NO_GUARD) as h:
            C = host(h.gemm(dev(A), dev(B)))
            h.check()
        r = rows_of(n, 4)
        ref = oracle.gemm_rows(A, B, r)
        absab = np.abs(A[r]) @ np.abs(B)
        err = float(np.max(np.abs(C[r] - ref) / absab))
        out["rows"][f"{dist} s={s}"] = err
        assert err <= 2 * n * U
        want = oracle.emu_gemm_rows(A, B, s, r[:3])
        np.testing.assert_array_equal(C[r[:3]].view(np.int64), want.view(np.int64))
        bad, _, _ = oracle.freivalds(A, B, C, np.random.default_rng(7).choice([-1.0, 1.0], n))
        assert bad == 0
    report(f"precision_n{n}.json", out)


# ---- grouped batch: 1024 problems, N log-uniform over [10, 2000] ---------------

@pytest.fixture(scope="module")
def batch_1024():
    sizes = workload.loguniform_sizes(1024, 10, 2000, seed=1)
    pairs = workload.batch("uniform01", 1, sizes)
    return sizes, pairs


@pytest.mark.parametrize("form", ["native", "emulated", "modular", "auto"])
def test_grouped_batch_1024(batch_1024, form):
    import torch
    import paper_1012_2273_gb300 as mm
    sizes, pairs = batch_1024
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    with mm.Handle(form) as h:
        Cs = h.gemm_grouped(As, Bs)
        Cs = h.gemm_grouped(As, Bs, Cs)  # graph replay
        h.check()
        replaced, _ = h.guard_read()
        plans = {n: h.plan(n) for n in set(sizes)}
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    worst = 0.0
    for p, ((A, B), C, n) in enumerate(zip(pairs, Cs, sizes)):
        C = C.cpu().numpy()
        bad, _, _ = oracle.freivalds(A, B, C, rng.choice([-1.0, 1.0], n))
        assert bad == 0, (p, n)
        if n <= 200:
            ref = oracle.gemm(A, B)
            absab = oracle.absgemm(A, B)
            assert_within_bound(C, ref, absab, n)
            worst = max(worst, float(np.max(np.abs(C - ref) / absab)) / (2 * n * U))
        elif p % 16 == 0:
            check_rows(C, A, B, n)
        if plans[n][0] != 0 and p % 64 == 1 and replaced == 0:  # the models describe unreplaced results
            r = rows_of(n, 2)[:3]
            if plans[n][0] == 1:
                want = oracle.emu_gemm_rows(A, B, plans[n][1], r)
            else:
                want = oracle.fixed_gemm_rows(A, B, oracle.modular_beta(plans[n][1], n), r)
            np.testing.assert_array_equal(C[r].view(np.int64), want.view(np.int64))
    report(f"grouped_1024_{form}.json", {"worst_error_over_bound_small_problems": worst,
                                          "elements_replaced_by_the_certificate_two_calls": replaced})
    if form in ("modular", "auto"):
        assert replaced == 0  # uniform inputs: the certificate vouches for every element


def test_grouped_workspace_waves(monkeypatch):
    # A workspace limit far below the batch's need forces several waves.
    import paper_1012_2273_gb300 as mm
    monkeypatch.setenv("MM_WORKSPACE_LIMIT_MB", "96")
    sizes = [700, 300, 1000, 64, 513, 1300]
    pairs = [workload.pair("uniform11", 40 + i, n) for i, n in enumerate(sizes)]
    with mm.Handle("emulated", slices=7, flags=mm.FLAG_NO_GUARD) as h:
        Cs = h.gemm_grouped([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs])
        h.check()
    for (A, B), C, n in zip(pairs, Cs, sizes):
        C = host(C)
        if n <= 700:
            np.testing.assert_array_equal(C.view(np.int64), oracle.emu_gemm(A, B, 7).view(np.int64))
        else:
            r = rows_of(n, 2)[:4]
            np.testing.assert_array_equal(C[r].view(np.int64), oracle.emu_gemm_rows(A, B, 7, r).view(np.int64))
