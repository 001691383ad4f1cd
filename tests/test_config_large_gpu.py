"""The large configuration: 64 grouped problems with N log-uniform over [1000, 16384]
and a single N = 16384 product, log-uniform-magnitude entries, emulated form.

About 73 GB of operands on the device; the oracle cannot form these products
in full, so every result is checked with Freivalds' test (the oracle's, on
the host) and on rows the oracle computes one by one, and a few rows are
compared bit for bit with the oracle's model of the emulation.
"""
import numpy as np
import pytest

import oracle
import workload
from helpers import U

pytestmark = pytest.mark.gpu


def verify(A, B, C, plan, rng, exact_rows=0):
    n = A.shape[0]
    bad, _, _ = oracle.freivalds(A, B, C, rng.choice([-1.0, 1.0], n))
    assert bad == 0, n
    rows = [0, int(rng.integers(1, n - 1)), n - 1]
    ref = oracle.gemm_rows(A, B, rows)
    absab = np.abs(A[rows]) @ np.abs(B)
    err = float(np.max(np.abs(C[rows] - ref) / absab))
    assert err <= 2 * n * U, (n, err)
    if exact_rows:
        if plan[0] == 2:  # modular form: the exact product of the fixed-point operands
            want = oracle.fixed_gemm_rows(A, B, oracle.modular_beta(plan[1], n), rows[:exact_rows])
        else:
            want = oracle.emu_gemm_rows(A, B, plan[1], rows[:exact_rows])
        np.testing.assert_array_equal(C[rows[:exact_rows]].view(np.int64), want.view(np.int64))
    return err


def test_grouped_64_loguniform_1000_to_16384_and_single_16384():
    import torch
    import paper_1012_2273_gb300 as mm
    free, _ = torch.cuda.mem_get_info()
    sizes = workload.loguniform_sizes(64, 1000, 16384, seed=5)
    need = sum(24 * n * n for n in sizes) + 24 * 16384 ** 2
    if free < need * 1.6:
        pytest.skip(f"needs about {need * 1.6 / 2**30:.0f} GiB free on the device, {free / 2**30:.0f} available")
    rng = np.random.default_rng(3)
    worst = 0.0
    with mm.Handle("auto") as h:
        # grouped batch: generate, copy, compute, verify problem by problem on the host
        host = []
        As, Bs = [], []
        for p, n in enumerate(sizes):
            A, B = workload.pair("loguniform20", 5 * 1000003 + p, n)
            host.append((A, B))
            As.append(torch.from_numpy(A).cuda())
            Bs.append(torch.from_numpy(B).cuda())
        Cs = h.gemm_grouped(As, Bs)
        h.check()
        replaced, _ = h.guard_read()  # the models describe the result only where nothing was replaced
        plans = {n: h.plan(n) for n in set(sizes)}
        order = sorted(range(len(sizes)), key=lambda i: -sizes[i])
        for rank, p in enumerate(order):
            C = Cs[p].cpu().numpy()
            A, B = host[p]
            worst = max(worst, verify(A, B, C, plans[sizes[p]], rng, exact_rows=1 if rank < 2 and not replaced else 0)
                        / (2 * sizes[p] * U))
        del As, Bs, Cs, host
        torch.cuda.empty_cache()
        # the single N = 16384 product
        n = 16384
        A, B = workload.pair("loguniform20", 16384, n)
        C = h.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
        h.check()
        replaced, _ = h.guard_read()
        worst = max(worst, verify(A, B, C.cpu().numpy(), h.plan(n), rng, exact_rows=0 if replaced else 1)
                    / (2 * n * U))
    assert worst <= 1.0
