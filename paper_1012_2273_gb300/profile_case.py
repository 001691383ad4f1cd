"""One small, self-contained product for kernel profiling (e.g. under ncu).

    python -m paper_1012_2273_gb300.profile_case --n 2048 --form emulated --reps 3
    python -m paper_1012_2273_gb300.profile_case --n 2048 --form modular --slices 16 --reps 3
    python -m paper_1012_2273_gb300.profile_case --sweep --reps 2
    python -m paper_1012_2273_gb300.profile_case --batch-native --reps 2

--sweep runs the benchmark's step instead: one grouped call over the paper's
size sweep (N = 10, 100, 500, 1000, 1500, 2000, automatic plan), the exact
launches bench.py times.  --profile creates the handle with MM_FLAG_PROFILE,
as bench.py's per-kernel timing pass does: kernels one after another, each
on every SM.  --batch-native runs the native bucket of the benchmark's
batch configuration (its problems with N < 256: N log-uniform over [10, 2000],
seed 1, entries uniform [0, 1)) as one grouped native call.

Generates seeded inputs (uniform [0, 1), seed 0), runs the product `reps`
times through the C ABI and exits 0 if every call succeeded.  The operands of
N = 2048 plus the emulation workspace exceed the 129 MB L2, so DRAM counters
stay meaningful, while the device footprint stays well under a gigabyte.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--form", choices=("native", "emulated", "modular", "auto"), default="emulated")
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--dist", default="uniform01")
    ap.add_argument("--sweep", action="store_true", help="run the benchmark's grouped sweep step")
    ap.add_argument("--profile", action="store_true", help="MM_FLAG_PROFILE: the bench's per-kernel timing pass")
    ap.add_argument("--batch-native", action="store_true", help="the batch configuration's native bucket, one call")
    args = ap.parse_args()

    import torch

    import paper_1012_2273_gb300 as mm
    import workload

    if args.batch_native:
        sizes = [n for n in workload.loguniform_sizes(1024, 10, 2000, seed=1) if n < 256]
        dev = torch.device("cuda")
        pairs = [workload.pair_torch("uniform01", 1 * 1000003 + p, n, dev)
                 for p, n in enumerate(workload.loguniform_sizes(1024, 10, 2000, seed=1)) if n < 256]
        with mm.Handle("native", flags=mm.FLAG_NO_GRAPH) as h:
            for _ in range(args.reps):
                h.gemm_grouped([a for a, _ in pairs], [b for _, b in pairs])
            h.check()
        torch.cuda.synchronize()
        print(f"profile_case: batch native bucket, {len(sizes)} problems, reps={args.reps} ok")
        return 0
    if args.sweep:
        pairs = [workload.pair("uniform01", 0, n) for n in workload.SWEEP_SIZES]
        As = [torch.from_numpy(a).cuda() for a, _ in pairs]
        Bs = [torch.from_numpy(b).cuda() for _, b in pairs]
        with mm.Handle("auto", flags=mm.FLAG_PROFILE if args.profile else 0) as h:
            for _ in range(args.reps):
                h.gemm_grouped(As, Bs)
            h.check()
        torch.cuda.synchronize()
        print(f"profile_case: sweep {list(workload.SWEEP_SIZES)} reps={args.reps} ok")
        return 0
    A, B = workload.pair(args.dist, 0, args.n)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.empty_like(dA)
    with mm.Handle(args.form, slices=args.slices) as h:
        for _ in range(args.reps):
            h.gemm(dA, dB, dC)
        h.check()
    torch.cuda.synchronize()
    print(f"profile_case: N={args.n} form={args.form} reps={args.reps} ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
