"""Autotuner: per size bucket, the fastest plan that keeps FP64 accuracy.

    python -m paper_1012_2273_gb300.autotune --out tune/gb300.tune

For each bucket of N it times the native FP64 form, the digit emulation for
every slice count s in 6..8 and the modular emulation for every moduli count
k in 13..16, each at tile widths 128 and 256 (pair groups chosen
automatically), at one representative size, and keeps the fastest plan whose
result stays close to native FP64 -- at the representative size and at the
bucket's smallest size -- on two input classes: uniform [-1, 1) and log-uniform
magnitudes 2^U(-20,20).  The handles run with the accuracy certificate on (the
library's default), so a plan's time is the mean over its two input classes,
native recomputation of the elements its certificate cannot vouch for
included: a plan too narrow for log-uniform inputs pays for it there.  "Close"
means
max |C_plan - C_native| / (|A||B|) <= N 2^-53 / 2; the native result is itself
within gamma_N |A||B| of the exact product, so an accepted plan is within
(N/2 + N + small) 2^-53 |A||B| < 2 N 2^-53 |A||B|, the library's accuracy
contract.  |A||B| is computed by the native form on |A| and |B|.

Among accurate plans the modular form is preferred unless another is more
than 5% faster: it serves every size above this range, and problems of
different forms in one grouped call run as separate launch groups, one after
another.

The modular form's fixed-point width shrinks by half a bit per doubling of N
while the allowance doubles, so within a bucket its worst case is the
smallest size, which is checked.

The output is a tune file ("max_n form slices bn groups" per line) that
mm_create accepts as mm_config.tune_path; the library's built-in table is
the result of running this on a GB300.
"""
from __future__ import annotations

import argparse
import os
import statistics
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

# (largest N of the bucket, size timed) -- accuracy is checked at the timed
# size and at the bucket's smallest size, where the bound is tightest.
BUCKETS = ((31, 24), (63, 48), (127, 96), (255, 192), (511, 384), (767, 640), (1023, 896), (1535, 1280),
           (1999, 1792), (2047, 2000), (3071, 2560), (4095, 3584), (6143, 5120), (65535, 8192))
# Above the modular form's limit (N <= 65535) the table falls back to this plan.
FALLBACK = (1 << 30, ("emulated", 6, 256, 0.0))
FORM_CODE = {"native": 0, "emulated": 1, "modular": 2}
U = 2.0 ** -53
MODULAR_PREFERENCE = 0.95  # a modular plan's time is compared after this factor


def _time_ms(fn, flush, reps):
    import torch
    stream = torch.cuda.current_stream()
    fn()
    ts = []
    for r in range(reps):
        flush.fill_(float(r))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune(buckets=BUCKETS, slices=(6, 7, 8), moduli=(13, 14, 15, 16), widths=(128, 256), reps=5, log=print):
    import torch

    import paper_1012_2273_gb300 as mm
    import workload

    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
    tmp = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"mm_autotune_{os.getpid()}.tune")
    rows = []
    native = mm.Handle("native")
    lo = 1
    for max_n, n in buckets:
        classes = []  # (A, B, native C, |A||B|, size)
        for size in sorted({n, max(lo, 8)}, reverse=True):
            for dist in ("uniform11", "loguniform20"):
                A, B = workload.pair(dist, 0, size)
                dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
                ref = native.gemm(dA, dB)
                absab = native.gemm(dA.abs(), dB.abs())
                classes.append((dA, dB, ref, absab, size))
        lo = max_n + 1
        native.check()
        best = ("native", 0, 256, _time_ms(lambda: native.gemm(classes[0][0], classes[0][1]), flush, reps))
        log(f"N={n:5d} native {best[3]:.3f} ms")
        candidates = [("emulated", s, bn) for s in slices for bn in widths]
        candidates += [("modular", k, bn) for k in moduli for bn in widths]
        for form, s, bn in candidates:
            if form == "modular" and min(mm.modular_params(s, size)[0] for *_, size in classes) < 1:
                continue
            with open(tmp, "w") as f:
                f.write(f"{1 << 30} {FORM_CODE[form]} {s} {bn} 0\n")
            h = mm.Handle(form, slices=s, tune_path=tmp)
            worst = 0.0  # deviation relative to each size's allowance N u / 2
            for dA, dB, ref, absab, size in classes:
                C = h.gemm(dA, dB)
                d = ((C - ref).abs() / absab.clamp_min(1e-300)).max().item()
                worst = max(worst, d / (size * U / 2))
            h.check()
            ok = worst <= 1.0
            # both input classes at the representative size (classes[0:2])
            ms = statistics.mean(_time_ms(lambda c=c: h.gemm(c[0], c[1]), flush, reps) for c in classes[:2])
            h.guard_read()
            h.close()
            log(f"N={n:5d} {form} {'k' if form == 'modular' else 's'}={s} bn={bn} {ms:.3f} ms  "
                f"max dev / allowance {worst:.3g} ({'ok' if ok else 'too far'})")
            score = ms * (MODULAR_PREFERENCE if form == "modular" else 1.0)
            best_score = best[3] * (MODULAR_PREFERENCE if best[0] == "modular" else 1.0)
            if ok and score < best_score:
                best = (form, s, bn, ms)
        rows.append((max_n, best))
        log(f"N<={max_n}: {best[0]} s={best[1]} bn={best[2]} ({best[3]:.3f} ms at N={n})")
    native.close()
    if os.path.exists(tmp):
        os.remove(tmp)
    rows.append(FALLBACK)
    return rows


def write(rows, path):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        f.write("# max_n form slices bn groups   (form 0 = native FP64, 1 = digit emulation (slices = digits),\n"
                "#   2 = modular emulation (slices = moduli); groups 0 = automatic)\n")
        f.write(f"# written by paper_1012_2273_gb300.autotune on {time.strftime('%Y-%m-%d %H:%M')}\n")
        for max_n, (form, s, bn, ms) in rows:
            note = f"   # {ms:.3f} ms" if ms else "   # fallback above the modular form's size limit"
            f.write(f"{max_n} {FORM_CODE[form]} {s if s else 7} {bn} 0{note}\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="tune.txt")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    rows = tune(reps=args.reps)
    write(rows, args.out)
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
