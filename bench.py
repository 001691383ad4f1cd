#!/usr/bin/env python3
"""Benchmark: FP64-accurate GEMM throughput on the paper's size sweep, one GB300.

Workload (the sweep the paper times, Sec. 4.1 and Tables 1-3, N from 10 to
2000): one square FP64 product C = A.B at each N in (10, 100, 500, 1000, 1500,
2000), entries uniform [0, 1) from seed 0 (synthetic stand-in for the paper's
unspecified RAND()).  One step = one grouped call of the library over the
six problems (mm_gemm_grouped, automatic plan: native FP64 for the small
sizes, split-precision emulation for the large ones, replayed from a CUDA
graph).  Flops are counted the paper's way, N^2 (2N - 1) per product.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Beside the headline it carries, untimed by
the headline: each form on each size of the sweep and of the precision
configuration (N = 4096, 8192), the 1024-problem batch (configuration 4) by
size bucket, the large configuration (64 problems up to N = 16384 and one
N = 16384), the accuracy certificate's cost, and the oracle's check of the
step's output.  `--impl reference` times the CPU oracle (the plain triple
loop of Alg. 1 on all host cores) on a bounded sample of the same workload
instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workload  # noqa: E402

SWEEP = workload.SWEEP_SIZES
DIST = "uniform01"
SEED = 0
METRIC = "FP64-accurate GEMM TFLOP/s vs N, emulated vs native FP64, % of peak, 1 GB300"
UNIT = "TFLOP/s"
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing on the host")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU-baseline sample")
    return ap.parse_args()


def sweep_flops(sizes=SWEEP) -> int:
    return sum(workload.flops(n) for n in sizes)


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; the sweep is replicated per rank)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group("nccl" if self._cuda() else "gloo")
            self.pg = td

    @staticmethod
    def _cuda():
        import torch
        return torch.cuda.is_available()

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if self._cuda() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# SM clock sampling through NVML (ctypes), nvidia-smi as a fallback
# ---------------------------------------------------------------------------
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, cuda_index: int, period_s: float = 0.002):
        self.period = period_s
        self.samples: list[tuple[int, int]] = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self._nvml = None
        self._handle = None
        self._smi_proc = None
        self._smi_file = None
        try:
            import torch
            props = torch.cuda.get_device_properties(cuda_index)
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            bus = f"{getattr(props, 'pci_domain_id', 0):08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
            if nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
                raise OSError("nvml handle")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = int(mx.value)
            self._reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self._nvml, self._handle = nv, h
        except Exception:
            self._nvml = None

    def _poll(self):
        nv, h = self._nvml, self._handle
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and self._reason_fn(h, ctypes.byref(rs)) == 0:
                self.samples.append((int(clk.value), int(rs.value)))
            time.sleep(self.period)

    def start(self):
        self.samples = []
        self._stop.clear()
        if self._nvml is not None:
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
        else:
            self._smi_file = open(os.path.join(ROOT, ".bench_clocks.csv"), "w")
            self._smi_proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]],
                stdout=self._smi_file, stderr=subprocess.DEVNULL)

    def stop(self) -> dict:
        self._stop.set()
        if self._thread:
            self._thread.join()
        if self._smi_proc:
            self._smi_proc.terminate()
            self._smi_proc.wait()
            self._smi_file.close()
            path = os.path.join(ROOT, ".bench_clocks.csv")
            for line in open(path):
                parts = [p.strip() for p in line.split(",")]
                try:
                    self.samples.append((int(float(parts[0])), int(parts[2], 16)))
                    self.max_mhz = int(float(parts[1]))
                except (ValueError, IndexError):
                    pass
            os.remove(path)
        mhz = [s[0] for s in self.samples]
        reasons = 0
        for _, r in self.samples:
            reasons |= r
        names = [n for b, n in REASON_BITS.items() if reasons & b and b != 0x1]
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": self.max_mhz,
                "reasons": names, "samples": len(mhz),
                "source": "nvml" if self._nvml is not None else "nvidia-smi"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
KERNEL_SOURCES = ("emu_gemm_pair.cu", "common.cuh", "launch.cuh", "modular.cuh", "recombine.cuh", "tile_index.cuh", "guard.cuh")


def source_digest() -> str:
    """Digest of the sources the slice-product kernel is built from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1012_2273_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_digest: str):
    """DRAM bytes per launch of the slice-product kernel from a committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "mod_gemm_pair_traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    if d.get("kernel_sha256_16") != kernel_digest:
        return None, d
    return d.get("dram_bytes_per_launch_full_workload"), d


def run_ours(args, dist: Dist):
    import torch
    import paper_1012_2273_gb300 as mm

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    peaks = load_peaks()
    rank_seed = SEED + dist.rank * 7919  # per-rank inputs (weak scaling)
    host = [workload.pair(DIST, rank_seed, n) for n in SWEEP]
    As = [torch.from_numpy(a).to(dev) for a, _ in host]
    Bs = [torch.from_numpy(b).to(dev) for _, b in host]
    Cs = [torch.empty_like(a) for a in As]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    h = mm.Handle("auto")
    plan = {n: h.plan(n) for n in SWEEP}

    # each handle's grouped call is validated and marshalled once (as a C
    # caller builds its arrays once); the timed step is the library call
    calls = {}

    def step(handle):
        if id(handle) not in calls:
            calls[id(handle)] = handle.grouped_call(As, Bs, Cs)
        calls[id(handle)]()

    # warm-up (builds and caches the CUDA graph)
    for _ in range(max(args.warmup, 3)):
        step(h)
    h.check()
    check = verify(As, Bs, Cs)

    # timed region: K steps, L2 flushed before each, device time by CUDA events
    sampler = ClockSampler(dist.local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step(h)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = dist.max(sum(step_ms) / 1e3)
    h.check()
    flops_step = sweep_flops()
    value = dist.world * args.steps * flops_step / total_s / 1e12

    # roofline pass: same steps with per-kernel events on the launch stream
    hp = mm.Handle("auto", flags=mm.FLAG_PROFILE)
    prof_steps = min(args.steps, 50)
    kinds = {k: [] for k in mm.KERNEL_KINDS}
    launches_per_step = 0
    for i in range(prof_steps + 2):
        flush.fill_(float(i))
        step(hp)
        p = hp.profile()
        if i >= 2:
            for k in kinds:
                kinds[k].append(p[k][0])
            launches_per_step = sum(v[1] for v in p.values())
    hp.check()
    emu_sizes = [n for n in SWEEP if plan[n][0] != 0]
    # tensor products per size: s(s+1)/2 digit pairs, or k residue products
    # (the dominant kernel's launch); the certificate's product of the
    # magnitude planes is a launch of its own, reported beside it
    pairs_of = {n: plan[n][1] * (plan[n][1] + 1) // 2 if plan[n][0] == 1 else plan[n][1] for n in emu_sizes}
    tensor_flops = sum(pairs_of[n] * 2 * n ** 3 for n in emu_sizes)
    cert_flops = sum(2 * n ** 3 for n in emu_sizes)
    gemm_ms = statistics.mean(kinds["slice_products"]) if emu_sizes else None
    cert_ms = statistics.mean(kinds["certificate"]) if emu_sizes else None
    all_modular = bool(emu_sizes) and all(plan[n][0] == 2 for n in emu_sizes)
    # with CTA pairs the certificate's products are units of the same launch
    # (no launch of its own): they count in its work
    cert_folded = bool(emu_sizes) and not cert_ms
    if cert_folded:
        tensor_flops += cert_flops
    digest = source_digest()
    traffic, traffic_meta = profiled_traffic(digest)
    roofline = None
    if gemm_ms:
        achieved = tensor_flops / (gemm_ms / 1e3) / 1e12
        peak = peaks["bf16_tflops"]
        kernel = ("mod_gemm_pair_kernel (tcgen05.mma cta_group::2 bf16 residue products on CTA pairs, "
                  "exact 1024-deep FP32 chunks, int32 sums reduced to paired residues in the epilogue, and the "
                  "accuracy certificate's magnitude products tested in the same epilogue)"
                  if all_modular else "emu_gemm_kernel (tcgen05 bf16 slice products)")
        roofline = {"kernel": kernel,
                    "bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4),
                    "peak_source": f"{peaks['source']} bf16 dense burst (MEASURED_PEAKS.json bf16_tflops)",
                    "traffic": traffic,
                    "algorithmic_flops_per_launch": tensor_flops,
                    "avg_launch_ms": round(gemm_ms, 4),
                    "note": "bf16 products of 2N^3 flops each: " + ", ".join(
                        f"N={n}: " + (f"digits s={plan[n][1]}, {pairs_of[n]} pairs" if plan[n][0] == 1
                                      else f"moduli k={plan[n][1]}, {pairs_of[n]} residue products")
                        for n in emu_sizes) + ("; plus the accuracy certificate's product of the magnitude planes "
                                               "per tile, units of the same launch" if cert_folded else "")
                    + "; one launch per step, timed alone on every SM (profiling pass)"}
        if cert_ms:
            roofline["certificate_launch"] = {
                "kernel": "emu_gemm_kernel<256, false, true> (the accuracy certificate's product of the "
                          "magnitude planes, one per tile, single CTAs)",
                "algorithmic_flops_per_launch": cert_flops, "avg_launch_ms": round(cert_ms, 4),
                "achieved": round(cert_flops / (cert_ms / 1e3) / 1e12, 2),
                "frac": round(cert_flops / (cert_ms / 1e3) / 1e12 / peak, 4),
                "note": "timed alone on every SM in the profiling pass; in the timed step it runs beside the "
                        "residue products on the SMs they leave"}

    # certificate: elements the step's calls sent to native FP64 (uniform
    # inputs: none), and the step without it (MM_FLAG_NO_GUARD) for context
    guard_replaced, guard_problems = h.guard_read()
    hu = mm.Handle("auto", flags=mm.FLAG_NO_GUARD)
    unguarded_ms = timed_calls(lambda: step(hu), flush, stream, 20)
    hu.check()
    hu.close()

    # per-N comparison of the forms (single calls, L2 flushed), the paper's
    # sweep and the precision configuration's larger sizes
    big = [workload.pair_torch(DIST, rank_seed, n, dev) for n in workload.PRECISION_SIZES[1:]]
    per_n = per_size(mm, As + [a for a, _ in big], Bs + [b for _, b in big],
                     Cs + [torch.empty_like(a) for a, _ in big], flush, stream)
    del big
    hn = mm.Handle("native")
    dmma_peak, dfma_peak = hn.probe_fp64_peak()
    int8_peak = hn.probe_int8_peak()
    for n, d in per_n.items():
        N = int(n)
        d["native_frac_of_dmma_peak"] = round(d["native_tflops"] / dmma_peak, 4)
        if N <= 100:  # HBM roofline: 24 N^2 bytes (A, B read, C written) per product
            d["native_frac_of_hbm_peak"] = round(24 * N * N / (d["native_ms"] / 1e3) / 1e9 / peaks["hbm_gbs"], 6)
        if "modular_moduli" in d:  # bf16 tensor work of the whole call (split and recombination included)
            k = d["modular_moduli"]
            d["modular_tensor_frac_whole_call"] = round(
                (k + 1) * 2 * N ** 3 / (d["modular_ms"] / 1e3) / 1e12 / peaks["bf16_tflops"], 4)
        if "int8_slices" in d:  # 8-bit integer MMA work of the whole call, digit pairs and the certificate's
            s8 = d["int8_slices"]
            d["int8_tops_whole_call"] = round((s8 * (s8 + 1) // 2 + 1) * 2 * N ** 3 / (d["int8_ms"] / 1e3) / 1e12, 2)
            d["int8_frac_of_imma_probe"] = round(d["int8_tops_whole_call"] / int8_peak, 4)

    batch = batch_block(mm, dev, flush, stream, peaks, dmma_peak)
    large = large_block(mm, dev, flush, stream)

    # end to end through the public API on host buffers (pinned), per step:
    # H2D of A and B, compute, D2H of C for every problem of the sweep
    e2e = end_to_end(mm, host, dev, steps=min(args.steps, 20))
    e2e_s = dist.max(e2e["seconds"])
    e2e_value = dist.world * e2e["steps"] * flops_step / e2e_s / 1e12

    cpu = None
    if dist.world == 1 and dist.rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
        check["oracle"] = oracle_check(host, Cs)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_s * 1e3 / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: uniform [0,1) FP64 from SplitMix64 seed 0 (stand-in for the paper's RAND())",
        "config": {"workload": "paper size sweep: one square FP64 product at each N in "
                               f"{list(SWEEP)}, one grouped library call per step (plan: "
                               + ", ".join(f"N={n}:" + ("native" if plan[n][0] == 0 else
                                                         f"digits s={plan[n][1]}" if plan[n][0] == 1 else
                                                         f"modular k={plan[n][1]}")
                                           for n in SWEEP) + ")",
                   "flops_per_step": flops_step, "flop_count": "N^2 (2N - 1) per product (paper, Sec. 3.1)",
                   "l2": f"flushed before every timed step ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "timing": "CUDA events on the launching stream around each step; max over ranks"},
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"],
                "how": "mm_gemm_grouped_host on pinned host buffers (uploads, grouped product and downloads "
                       "of the whole sweep, overlapped by chunks), wall clock per step"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "roofline": roofline,
        "kernel_times_ms_per_step": {k: round(statistics.mean(v), 4) for k, v in kinds.items() if v},
        "certificate": {"elements_recomputed_per_step": guard_replaced / max(1, args.steps + max(args.warmup, 3)),
                        "problems_recomputed_whole": guard_problems,
                        "ms_per_step_without_certificate": round(unguarded_ms, 4),
                        "value_without_certificate": round(flops_step / (unguarded_ms / 1e3) / 1e12, 3),
                        "note": "the library's default checks every emulated element's error bound and "
                                "recomputes what it cannot vouch for in native FP64 (MM_FLAG_NO_GUARD skips it)"},
        "per_n": per_n,
        "batch_1024": batch,
        "large": large,
        "fp64_peak_measured": {"dmma_tflops": round(dmma_peak, 4), "dfma_tflops": round(dfma_peak, 4)},
        "int8_mma_peak_measured_tops": round(int8_peak, 2),
        "check": check,
        "cpu_baseline": cpu,
    }
    for hh in (h, hp, hn):
        hh.close()
    return line


def verify(As, Bs, Cs) -> dict:
    """Freivalds-style residual check of the step's output on the device (not timed)."""
    import torch
    worst = 0.0
    for A, B, C in zip(As, Bs, Cs):
        n = A.shape[0]
        x = torch.sign(torch.randn(n, dtype=torch.float64, device=A.device, generator=None))
        y = A @ (B @ x) - C @ x
        tol = (A.abs() @ (B.abs() @ x.abs()) + C.abs() @ x.abs()) * n * 2.0 ** -53
        worst = max(worst, float((y.abs() / tol.clamp_min(1e-300)).max()))
    return {"freivalds_worst_ratio": round(worst, 4), "passed": worst <= 4.0}


def oracle_check(host_pairs, Cs) -> dict:
    """Part of the CPU-baseline leg (rank 0, one GPU): the benchmarked step's
    output checked with the oracle on the host, outside the timed region: the
    oracle's Freivalds test on every product and three rows of each computed
    by the oracle (Alg. 1's left-to-right sums), componentwise error
    |C - C_oracle| / (|A||B|) against 2 N 2^-53."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(2)
    worst, fails = 0.0, 0
    for (A, B), C in zip(host_pairs, Cs):
        C = C.cpu().numpy()
        n = A.shape[0]
        bad, _, _ = oracle.freivalds(A, B, C, rng.choice([-1.0, 1.0], n))
        fails += int(bad)
        rows = sorted({0, n // 2, n - 1})
        ref = oracle.gemm_rows(A, B, rows)
        absab = oracle.absgemm_mnk(np.ascontiguousarray(A[rows]), B)
        m = absab > 0
        if m.any():
            worst = max(worst, float(np.max(np.abs(C[rows] - ref)[m] / absab[m])) / (2 * n * 2.0 ** -53))
    return {"oracle_rows_worst_error_over_2Nu": round(worst, 4), "freivalds_failures": fails,
            "passed": worst <= 1.0 and fails == 0,
            "how": "oracle.freivalds on every product, oracle.gemm_rows on rows 0, N/2, N-1"}


def per_size(mm, As, Bs, Cs, flush, stream, reps: int = 5) -> dict:
    """Each form on each problem alone (single calls, L2 flushed, median of
    `reps`; native FP64 takes fewer repetitions above N = 2000)."""
    import torch
    out = {}
    hn = mm.Handle("native")
    he = mm.Handle("emulated")
    hm = mm.Handle("modular")
    hi = mm.Handle("int8")
    ha = mm.Handle("auto")
    for A, B, C in zip(As, Bs, Cs):
        n = A.shape[0]
        row = {}
        forms = [("native", hn), ("emulated", he), ("auto", ha)]
        if n >= 256:
            forms[2:2] = [("modular", hm), ("int8", hi)]
        for name, hh in forms:
            call = hh.gemm_call(A, B, C)  # validated and marshalled once
            call()  # warm
            ts = []
            for r in range(reps if name != "native" or n <= 2000 else 2):
                flush.fill_(float(r))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            row[f"{name}_ms"] = round(ms, 4)
            row[f"{name}_tflops"] = round(workload.flops(n) / (ms / 1e3) / 1e12, 4)
        row["emulated_slices"] = he.plan(n)[1]
        if n >= 256:
            row["modular_moduli"] = hm.plan(n)[1]
            row["int8_slices"] = hi.plan(n)[1]
        form, k = ha.plan(n)
        row["auto_plan"] = ("native", f"digits s={k}", f"modular k={k}", f"int8 s={k}")[form]
        row["speedup_auto_over_native"] = round(row["native_ms"] / row["auto_ms"], 2)
        out[str(n)] = row
    for hh in (hn, he, hm, hi, ha):
        hh.guard_read()  # (clears the certificate's counts)
        hh.check()
        hh.close()
    return out


def timed_calls(fn, flush, stream, reps: int) -> float:
    """Median device time (ms) of fn() over `reps` calls, L2 flushed before each."""
    import torch
    fn()  # warm (builds a grouped call's graph)
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


def batch_block(mm, dev, flush, stream, peaks, dmma_peak, reps: int = 5) -> dict:
    """Batching: one grouped call of 1024 independent products, N log-uniform
    over the integers [10, 2000] (seed 1), entries uniform [0, 1), automatic
    plan, replayed from its CUDA graph.  Then each size bucket of the plan
    alone (same problems, its own grouped call): time, share, and the roof of
    its form -- bf16 tensor work (residue products, certificate included) for
    emulated buckets, the FP64 DMMA probe (and HBM for N <= 100) for native."""
    sizes = workload.loguniform_sizes(1024, 10, 2000, seed=1)
    pairs = [workload.pair_torch("uniform01", 1 * 1000003 + p, n, dev) for p, n in enumerate(sizes)]
    As = [a for a, _ in pairs]
    Bs = [b for _, b in pairs]
    Cs = [a.new_empty(a.shape) for a in As]
    del pairs
    h = mm.Handle("auto")
    call = h.grouped_call(As, Bs, Cs)  # validated and marshalled once
    ms = timed_calls(call, flush, stream, reps)
    flops = sum(workload.flops(n) for n in sizes)
    replaced, _ = h.guard_read()
    plans = {n: h.plan(n) for n in set(sizes)}
    buckets = {}
    for i, n in enumerate(sizes):
        buckets.setdefault(plans[n], []).append(i)
    rows = {}
    total_bucket_ms = 0.0
    for (form, k), idx in sorted(buckets.items()):
        sub = h.grouped_call([As[i] for i in idx], [Bs[i] for i in idx], [Cs[i] for i in idx])
        bms = timed_calls(sub, flush, stream, reps)
        total_bucket_ms += bms
        ns = [sizes[i] for i in idx]
        bflops = sum(workload.flops(n) for n in ns)
        name = ("native", f"digits s={k}", f"modular k={k}", f"int8 s={k}")[form]
        r = {"problems": len(idx), "N_range": [min(ns), max(ns)], "ms": round(bms, 4),
             "tflops": round(bflops / (bms / 1e3) / 1e12, 3)}
        if form == 0:
            r["frac_of_dmma_probe"] = round(bflops / (bms / 1e3) / 1e12 / dmma_peak, 4)
            if max(ns) <= 100:
                r["frac_of_hbm"] = round(sum(24 * n * n for n in ns) / (bms / 1e3) / 1e9 / peaks["hbm_gbs"], 5)
        elif form == 2:
            tensor = sum((k + 1) * 2 * n ** 3 for n in ns)  # k residue products + the certificate's
            r["tensor_frac_whole_call"] = round(tensor / (bms / 1e3) / 1e12 / peaks["bf16_tflops"], 4)
        rows[name] = r
    for r in rows.values():
        r["share_of_bucket_time"] = round(r["ms"] / total_bucket_ms, 4)
    h.check()
    h.close()
    return {"workload": "1024 square FP64 products, N log-uniform over [10, 2000] (seed 1), uniform [0, 1), "
                        "one grouped call (CUDA graph replay), automatic plan",
            "flops": flops, "ms": round(ms, 4), "tflops": round(flops / (ms / 1e3) / 1e12, 3),
            "elements_recomputed_by_the_certificate": replaced, "buckets": rows,
            "timing": f"median of {reps} calls, L2 flushed before each"}


def large_block(mm, dev, flush, stream, reps: int = 2) -> dict:
    """The combined large configuration: a grouped call of 64 products, N
    log-uniform over [1000, 16384] (seed 5), and a single N = 16384 product,
    entries of magnitude 2^U(-20, 20) with random signs, automatic plan.
    Inputs are generated on the device (the same SplitMix64 streams)."""
    import torch
    sizes = workload.loguniform_sizes(64, 1000, 16384, seed=5)
    need = sum(24 * n * n for n in sizes) + 24 * 16384 ** 2
    free, _ = torch.cuda.mem_get_info(dev)
    if free < 1.6 * need:
        return {"skipped": f"needs about {1.6 * need / 2**30:.0f} GiB free, {free / 2**30:.0f} GiB available"}
    h = mm.Handle("auto")
    out = {"workload": "64 square FP64 products, N log-uniform over [1000, 16384] (seed 5), and one N = 16384, "
                       "entries 2^U(-20,20) with random signs, automatic plan"}
    pairs = [workload.pair_torch("loguniform20", 5 * 1000003 + p, n, dev) for p, n in enumerate(sizes)]
    As = [a for a, _ in pairs]
    Bs = [b for _, b in pairs]
    Cs = [a.new_empty(a.shape) for a in As]
    del pairs
    ms = timed_calls(h.grouped_call(As, Bs, Cs), flush, stream, reps)
    flops = sum(workload.flops(n) for n in sizes)
    out["grouped"] = {"N_range": [min(sizes), max(sizes)], "flops": flops, "ms": round(ms, 3),
                      "tflops": round(flops / (ms / 1e3) / 1e12, 3),
                      "elements_recomputed_by_the_certificate": h.guard_read()[0]}
    del As, Bs, Cs
    torch.cuda.empty_cache()
    n = 16384
    A, B = workload.pair_torch("loguniform20", 16384, n, dev)
    C = torch.empty_like(A)
    ms = timed_calls(h.gemm_call(A, B, C), flush, stream, reps)  # validated and marshalled once
    form, k = h.plan(n)
    out["single_16384"] = {"plan": ("native", f"digits s={k}", f"modular k={k}", f"int8 s={k}")[form],
                           "ms": round(ms, 3), "tflops": round(workload.flops(n) / (ms / 1e3) / 1e12, 3),
                           "elements_recomputed_by_the_certificate": h.guard_read()[0]}
    out["timing"] = f"median of {reps} calls after a warm-up call, L2 flushed before each"
    del A, B, C
    torch.cuda.empty_cache()
    h.check()
    h.close()
    return out


def end_to_end(mm, host_pairs, dev, steps: int) -> dict:
    """The step through the public host API: mm_gemm_grouped_host on pinned
    host matrices (upload of every A and B, the grouped product, download of
    every C, returning when C is on the host), wall clock per step."""
    import torch
    h = mm.Handle("auto")
    As = [torch.from_numpy(a).pin_memory() for a, _ in host_pairs]
    Bs = [torch.from_numpy(b).pin_memory() for _, b in host_pairs]
    Cs = [torch.empty_like(a).pin_memory() for a in As]
    for _ in range(3):  # warm (builds the chunks' graphs)
        h.gemm_grouped_host(As, Bs, Cs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        h.gemm_grouped_host(As, Bs, Cs)
    secs = time.perf_counter() - t0
    h.check()
    h.close()
    h2d = sum(2 * a.numel() * 8 for a in As)
    d2h = sum(a.numel() * 8 for a in As)
    return {"seconds": secs, "steps": steps, "h2d": h2d, "d2h": d2h}


# ---------------------------------------------------------------------------
# CPU oracle timings (baseline and reference arm)
# ---------------------------------------------------------------------------
def _oracle_sample(budget_s: float):
    """Sizes of the sweep (ascending) whose oracle run fits `budget_s`, and the inputs."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    a, b = workload.pair(DIST, SEED, 200)
    t0 = time.perf_counter()
    oracle.gemm(a, b, nthreads=threads)
    rate = workload.flops(200) / max(time.perf_counter() - t0, 1e-6)  # flop/s, rough
    sizes, est = [], 0.0
    for n in SWEEP:
        t = workload.flops(n) / rate
        if est + t > budget_s and sizes:
            break
        sizes.append(n)
        est += t
    pairs = [workload.pair(DIST, SEED, n) for n in sizes]
    return oracle, threads, sizes, pairs


def cpu_baseline(target_s: float) -> dict:
    oracle, threads, sizes, pairs = _oracle_sample(min(target_s, 30.0))
    flops, reps = 0, 0
    t0 = time.perf_counter()
    while True:
        for a, b in pairs:
            oracle.gemm(a, b, nthreads=threads)
        flops += sum(workload.flops(n) for n in sizes)
        reps += 1
        if time.perf_counter() - t0 >= min(target_s, 30.0) or reps >= 200:
            break
    secs = time.perf_counter() - t0
    return {"value": flops / secs / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"oracle (Alg. 1 triple loop, OpenMP over rows) on N={sizes} x {reps} repetitions, "
                      f"{secs:.1f} s on {threads} host threads"}


def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return None
    per_step_budget = max(0.05, min(5.0, 150.0 / max(1, args.steps + args.warmup)))
    oracle, threads, sizes, pairs = _oracle_sample(per_step_budget)
    flops_step = sum(workload.flops(n) for n in sizes)
    for _ in range(args.warmup):
        for a, b in pairs:
            oracle.gemm(a, b, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for a, b in pairs:
            oracle.gemm(a, b, nthreads=threads)
    secs = time.perf_counter() - t0
    value = args.steps * flops_step / secs / 1e12
    sample = f"oracle (Alg. 1 triple loop, OpenMP over rows) on N={sizes} of the sweep per step"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: uniform [0,1) FP64 from SplitMix64 seed 0",
            "config": {"workload": f"paper size sweep, bounded sample N={sizes}", "flops_per_step": flops_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            line = run_reference(args, dist)
        else:
            line = run_ours(args, dist)
        if dist.rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
