"""The paper's row-block decomposition on one GPU.

The paper parallelises C = A.B by giving each of W workers a block of rows of
A (and all of B); each worker computes its rows of C and the master gathers
them (Alg. 2-4).  The rows are split evenly and the first N mod W workers get
one row more (the remainder rule of Sec. 3.1.1).  Here a worker is a CUDA
stream with its own handle (a handle's workspace must not be shared by
concurrent calls): worker w computes C[r0:r1] = A[r0:r1] . B through
mm_gemm_ex on row-block views.  Every form computes each row of C from that
row of A and all of B alone, with the same plan for every block of a square
product, so the decomposition returns the single call's result bit for bit.

On a GPU the single call already spreads its tiles over every SM, so the
decomposition measures what the paper's scheme adds on top of that (nothing
is expected): ``python -m paper_1012_2273_gb300.rowblocks --n 2000`` prints
one JSON line per worker count.
"""
from __future__ import annotations

import argparse
import json


def row_ranges(n_rows: int, workers: int) -> list[tuple[int, int]]:
    """Row blocks [r0, r1) of the paper's split (shard.rows_of_worker): n // W
    rows each, one more for each of the first n % W workers."""
    from paper_1012_2273_gb300.shard import rows_of_worker
    if workers < 1:
        raise ValueError("workers must be >= 1")
    return [(o, o + c) for o, c in (rows_of_worker(n_rows, workers, w) for w in range(workers))]


class RowBlockGemm:
    """W workers (stream + handle each) computing row blocks of C = A.B."""

    def __init__(self, workers: int, mode: str = "auto", slices: int = 0, **handle_kw):
        import torch
        import paper_1012_2273_gb300 as mm
        self.workers = workers
        self.handles = [mm.Handle(mode, slices=slices, **handle_kw) for _ in range(workers)]
        self.streams = [torch.cuda.Stream() for _ in range(workers)]

    def __call__(self, A, B, C=None):
        import torch
        if C is None:
            C = torch.empty((A.shape[0], B.shape[1]), dtype=torch.float64, device=A.device)
        main = torch.cuda.current_stream()
        for h, s, (r0, r1) in zip(self.handles, self.streams, row_ranges(A.shape[0], self.workers)):
            s.wait_stream(main)  # inputs ready; the "distribution" of Alg. 2 is a view, no copy
            if r1 > r0:
                h.gemm(A[r0:r1], B, C[r0:r1], stream=s)
        for s in self.streams:  # the "gather": the master waits for every worker
            main.wait_stream(s)
        return C

    def check(self):
        for h in self.handles:
            h.check()

    def close(self):
        for h in self.handles:
            h.close()


def main() -> None:
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--workers", type=int, nargs="+", default=[1, 2, 4, 8])
    ap.add_argument("--mode", default="auto")
    ap.add_argument("--reps", type=int, default=20)
    args = ap.parse_args()
    n = args.n
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.rand((n, n), dtype=torch.float64, device="cuda", generator=g)
    B = torch.rand((n, n), dtype=torch.float64, device="cuda", generator=g)
    flops = n * n * (2 * n - 1)
    base_ms = None
    ref = None
    for W in args.workers:
        rb = RowBlockGemm(W, args.mode)
        C = rb(A, B)
        torch.cuda.synchronize()
        rb.check()
        if ref is None:
            ref = C.clone()
        same = bool(torch.equal(C.view(torch.int64), ref.view(torch.int64)))
        for _ in range(3):
            rb(A, B, C)
        times = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            rb(A, B, C)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        rb.check()
        rb.close()
        ms = sorted(times)[len(times) // 2]
        base_ms = ms if base_ms is None else base_ms
        print(json.dumps({"n": n, "workers": W, "mode": args.mode, "ms_median": round(ms, 4),
                          "tflops": round(flops / ms / 1e9, 3), "speedup_vs_first": round(base_ms / ms, 3),
                          "bit_identical_to_first": same}), flush=True)


if __name__ == "__main__":
    main()
