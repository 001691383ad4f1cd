"""Python binding of the GB300 dense FP64 product library (include/mm.h).

Argument marshalling only: every step of the product runs in the CUDA
kernels of libmm.so.  PyTorch supplies device memory and streams; tensors are
passed to the C ABI as raw device pointers.  There is no CPU fallback: if the
library cannot be built or loaded, importing a function that needs it raises.

    import torch, paper_1012_2273_gb300 as mm
    h = mm.Handle()                       # MM_AUTO
    C = h.gemm(A, B)                      # A, B: (N, N) float64 CUDA tensors
    Cs = h.gemm_grouped([A1, A2], [B1, B2])
    h.check()                             # device-side errors (timeouts, Inf/NaN)
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

from . import build as _build

NATIVE_FP64 = 0
EMU_BF16 = 1
EMU_INT8 = 2
AUTO = 3
EMU_MODULAR = 4
FLAG_NO_GRAPH = 1
FLAG_PROFILE = 2
FLAG_NO_GUARD = 4

STATUS_NAMES = {
    0: "MM_OK", 1: "MM_ERR_INVALID", 2: "MM_ERR_CUDA", 3: "MM_ERR_NOMEM",
    4: "MM_ERR_UNSUPPORTED", 5: "MM_ERR_TIMEOUT", 6: "MM_ERR_NONFINITE",
}

_MODES = {"native": NATIVE_FP64, "emulated": EMU_BF16, "emu": EMU_BF16, "auto": AUTO,
          "modular": EMU_MODULAR, "int8": EMU_INT8}
# forms reported by plan(): native FP64, digit emulation, modular emulation, INT8 slices
FORMS = ("native", "emulated", "modular", "int8")

_lock = threading.Lock()
_lib = None


class MMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("slices", ctypes.c_int), ("flags", ctypes.c_uint),
                ("tune_path", ctypes.c_char_p)]


SYMBOLS = ("mm_create", "mm_destroy", "mm_gemm", "mm_gemm_grouped", "mm_gemm_ex", "mm_gemm_grouped_ex",
           "mm_gemm_host", "mm_gemm_grouped_host",
           "mm_status_get", "mm_guard_read",
           "mm_last_error", "mm_plan", "mm_profile_read", "mm_probe_fp64_peak", "mm_probe_int8_peak", "mm_selftest_wait", "mm_split",
           "mm_split_noalloc",
           "mm_level_sums", "mm_recombine", "mm_modular_params")
SPLIT_NOALLOC_MAX_N = 65536
KERNEL_KINDS = ("split", "slice_products", "native_fp64", "recombine", "certificate")


def library_path() -> str:
    return _build.LIB


def lib(build_if_needed: bool = True) -> ctypes.CDLL:
    """Loads libmm.so (building it first if sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"libmm.so not found at {path}; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.mm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Config)]
            L.mm_destroy.argtypes = [vp]
            L.mm_gemm.argtypes = [vp, ci, vp, vp, vp, vp]
            L.mm_gemm_grouped.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                          ctypes.POINTER(vp), vp]
            L.mm_gemm_ex.argtypes = [vp, ci, ci, ci, ci, ci, vp, ci, vp, ci, vp, ci, vp]
            pi_ = ctypes.POINTER(ci)
            L.mm_gemm_grouped_ex.argtypes = [vp, ci, pi_, pi_, pi_, pi_, pi_, ctypes.POINTER(vp), pi_,
                                             ctypes.POINTER(vp), pi_, ctypes.POINTER(vp), pi_, vp]
            L.mm_gemm_host.argtypes = [vp, ci, vp, vp, vp, vp]
            L.mm_gemm_grouped_host.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                               ctypes.POINTER(vp), vp]
            L.mm_status_get.argtypes = [vp, vp]
            L.mm_guard_read.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
            L.mm_last_error.argtypes = [vp]
            L.mm_last_error.restype = ctypes.c_char_p
            L.mm_plan.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]
            L.mm_split.argtypes = [vp, ci, vp, ci, ci, vp, vp, ci, ci, vp]
            L.mm_split_noalloc.argtypes = [ci, vp, ci, ci, vp, vp, ci, ci, vp, vp]
            L.mm_level_sums.argtypes = [vp, ci, ci, vp, ci, vp, ci, ci, vp, vp]
            L.mm_recombine.argtypes = [vp, ci, ci, vp, vp, vp, vp, vp]
            L.mm_profile_read.argtypes = [vp, ctypes.POINTER(cd), ctypes.POINTER(ci)]
            L.mm_probe_fp64_peak.argtypes = [vp, ctypes.POINTER(cd), ctypes.POINTER(cd)]
            L.mm_probe_int8_peak.argtypes = [vp, ctypes.POINTER(cd)]
            L.mm_selftest_wait.argtypes = [vp, ci, vp]
            L.mm_modular_params.argtypes = [ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]
            for name in SYMBOLS:
                if name != "mm_last_error":
                    getattr(L, name).restype = ci
            _ = cd
            _lib = L
    return _lib


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check_tensor(t, name: str, n: int | None = None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")
    if t.dim() != 2 or t.shape[0] != t.shape[1] or (n is not None and t.shape[0] != n):
        raise ValueError(f"{name} must be square" + (f" of size {n}" if n is not None else ""))


def _layout(rows: int, cols: int, stride0: int, stride1: int, allow_transposed: bool, name: str = "matrix"):
    """(rows, cols, leading dimension, transposed) of a matrix with element
    strides (stride0, stride1): row-major (unit column stride, row stride >=
    cols) or -- where allowed -- the transpose of a row-major matrix (unit row
    stride, column stride >= rows, e.g. ``X.T``).  Single rows and columns
    take the row-major reading; the leading dimension is at least 1."""
    if cols <= 1 or stride1 == 1:
        ld = stride0 if rows > 1 and cols > 0 else cols
        if ld >= cols:
            return rows, cols, max(ld, 1), 0
    if allow_transposed and (rows <= 1 or stride0 == 1):
        ld = stride1 if cols > 1 and rows > 0 else rows
        if ld >= rows:
            return rows, cols, max(ld, 1), 1
    raise ValueError(f"{name} must be row-major with a row stride >= its row length"
                     + (" (or the transpose of such a matrix)" if allow_transposed else ""))


def _matrix(t, name: str, allow_transposed: bool = False):
    """_layout of a float64 CUDA matrix view."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    return _layout(int(t.shape[0]), int(t.shape[1]), int(t.stride(0)), int(t.stride(1)), allow_transposed, name)


def _square_contiguous(*ts) -> bool:
    n = ts[0].shape[0]
    return all(t.dim() == 2 and t.shape[0] == n and t.shape[1] == n and t.is_contiguous() and t.data_ptr() % 16 == 0
               for t in ts)


def split_noalloc(M, by_columns: bool, slices: int, exps, digits, status=None, stream=None) -> int:
    """mm_split_noalloc: scale and split into caller-provided buffers, allocating nothing.

    For callers that may not allocate device memory: the library's only
    scratch for this step is a fixed static device array (N <= 65536).
    `exps` (int32 [N]) and `digits` (int16 [s][rows][ld], bf16 bit patterns)
    are CUDA tensors the caller owns; `status` an optional int32 CUDA tensor.
    Calls sharing the device must not overlap on the GPU.  Returns the
    mm_status code (0 = enqueued).
    """
    _check_tensor(M, "M")
    n = M.shape[0]
    s_, rows, ld = digits.shape
    return int(lib().mm_split_noalloc(n, M.data_ptr(), int(bool(by_columns)), int(slices), exps.data_ptr(),
                                      digits.data_ptr(), rows, ld, status.data_ptr() if status is not None else None,
                                      _stream_ptr(stream)))


def modular_params(k: int, n: int) -> tuple[int, tuple[int, ...]]:
    """mm_modular_params: (fixed-point width beta, moduli) of the modular form
    with k moduli at size n.  Host-only; needs no GPU."""
    beta = ctypes.c_int(0)
    mods = (ctypes.c_int * 16)()
    rc = int(lib().mm_modular_params(int(k), int(n), ctypes.byref(beta), mods))
    if rc != 0:
        raise MMError(rc, "mm_modular_params: k must be in 1..16 and n >= 1")
    return beta.value, tuple(mods[:k])


class _GroupedCall:
    """See Handle.grouped_call."""

    def __init__(self, handle, As, Bs, Cs, dims, square):
        count = len(As)
        self.handle, self.As, self.Bs, self.Cs = handle, As, Bs, Cs
        self.count = count
        self.pa = (ctypes.c_void_p * count)(*[a.data_ptr() for a in As])
        self.pb = (ctypes.c_void_p * count)(*[b.data_ptr() for b in Bs])
        self.pc = (ctypes.c_void_p * count)(*[c.data_ptr() for c in Cs])
        self.square = square
        if square:
            self.ns = (ctypes.c_int * count)(*[d[1] for d in dims])
        else:
            self.col = [(ctypes.c_int * count)(*[d[j] for d in dims]) for j in range(8)]

    def __call__(self, stream=None):
        h = self.handle
        if self.square:
            h._raise(h._lib.mm_gemm_grouped(h._h, self.count, self.ns, self.pa, self.pb, self.pc, _stream_ptr(stream)))
        else:
            c = self.col
            h._raise(h._lib.mm_gemm_grouped_ex(h._h, self.count, c[6], c[7], c[0], c[1], c[2], self.pa, c[3], self.pb,
                                               c[4], self.pc, c[5], _stream_ptr(stream)))
        return self.Cs


class Handle:
    """One library handle (see mm_create).  Not thread safe."""

    def __init__(self, mode: str | int = "auto", slices: int = 0, flags: int = 0, tune_path: str | None = None):
        self._lib = lib()
        m = _MODES[mode] if isinstance(mode, str) else int(mode)
        self._tune = tune_path.encode() if tune_path else None
        cfg = _Config(m, int(slices), int(flags), self._tune)
        h = ctypes.c_void_p()
        rc = self._lib.mm_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != 0:
            raise MMError(rc, "mm_create failed")
        self._h = h

    # -- helpers ---------------------------------------------------------------
    def _raise(self, rc: int):
        if rc != 0:
            msg = self._lib.mm_last_error(self._h)
            raise MMError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the product -----------------------------------------------------------
    def gemm(self, A, B, C=None, stream=None):
        """C = A.B on the device (asynchronous on `stream`).  A (M x K) and B
        (K x N) are row-major float64 CUDA tensors, possibly views with a row
        stride (mm_gemm_ex); square contiguous operands take mm_gemm."""
        import torch
        m, k, lda, ta = _matrix(A, "A", True)
        k2, n, ldb, tb = _matrix(B, "B", True)
        if k2 != k:
            raise ValueError(f"inner dimensions differ: A is {m} x {k}, B is {k2} x {n}")
        if C is None:
            C = torch.empty((m, n), dtype=torch.float64, device=A.device)
        mc, nc, ldc, _ = _matrix(C, "C")
        if (mc, nc) != (m, n):
            raise ValueError(f"C must be {m} x {n}")
        if _square_contiguous(A, B, C):
            self._raise(self._lib.mm_gemm(self._h, n, A.data_ptr(), B.data_ptr(), C.data_ptr(), _stream_ptr(stream)))
        else:
            self._raise(self._lib.mm_gemm_ex(self._h, ta, tb, m, n, k, A.data_ptr(), lda, B.data_ptr(), ldb,
                                             C.data_ptr(), ldc, _stream_ptr(stream)))
        return C

    def gemm_grouped(self, As: Sequence, Bs: Sequence, Cs: Sequence | None = None, stream=None):
        return self.grouped_call(As, Bs, Cs)(stream)

    def gemm_call(self, A, B, C):
        """One product validated and marshalled once, for repeated use: the
        returned callable runs mm_gemm (or mm_gemm_ex) on the stream it is
        given.  The tensors must keep their storage and shapes meanwhile."""
        m, k, lda, ta = _matrix(A, "A", True)
        k2, n, ldb, tb = _matrix(B, "B", True)
        if k2 != k:
            raise ValueError(f"inner dimensions differ: A is {m} x {k}, B is {k2} x {n}")
        mc, nc, ldc, _ = _matrix(C, "C")
        if (mc, nc) != (m, n):
            raise ValueError(f"C must be {m} x {n}")
        lib, hh, pa, pb, pc = self._lib, self._h, A.data_ptr(), B.data_ptr(), C.data_ptr()
        if _square_contiguous(A, B, C):
            def call(stream=None):
                self._raise(lib.mm_gemm(hh, n, pa, pb, pc, _stream_ptr(stream)))
                return C
        else:
            def call(stream=None):
                self._raise(lib.mm_gemm_ex(hh, ta, tb, m, n, k, pa, lda, pb, ldb, pc, ldc, _stream_ptr(stream)))
                return C
        call.tensors = (A, B, C)  # kept alive with the call
        return call

    def grouped_call(self, As: Sequence, Bs: Sequence, Cs: Sequence | None = None):
        """A grouped call validated and marshalled once, for repeated use: the
        returned object calls mm_gemm_grouped (or mm_gemm_grouped_ex) with the
        pointer and size arrays built here, on the stream it is given, and
        holds references to the tensors.  The tensors must keep their storage
        and shapes while it is in use (their contents may change)."""
        import torch
        count = len(As)
        if len(Bs) != count or (Cs is not None and len(Cs) != count):
            raise ValueError("As, Bs, Cs must have the same length")
        if Cs is None:
            Cs = [torch.empty((a.shape[0], b.shape[1]), dtype=torch.float64, device=a.device) for a, b in zip(As, Bs)]
        dims = []
        for i, (a, b, c) in enumerate(zip(As, Bs, Cs)):
            m, k, lda, ta = _matrix(a, f"As[{i}]", True)
            k2, n, ldb, tb = _matrix(b, f"Bs[{i}]", True)
            mc, nc, ldc, _ = _matrix(c, f"Cs[{i}]")
            if k2 != k or (mc, nc) != (m, n):
                raise ValueError(f"problem {i}: shapes {tuple(a.shape)} x {tuple(b.shape)} -> {tuple(c.shape)}")
            dims.append((m, n, k, lda, ldb, ldc, ta, tb))
        return _GroupedCall(self, list(As), list(Bs), list(Cs), dims,
                            all(_square_contiguous(a, b, c) for a, b, c in zip(As, Bs, Cs)))

    def gemm_host(self, A, B, C=None, stream=None):
        """End-to-end product on host (numpy) arrays: copy in, compute, copy out."""
        import numpy as np
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        n = A.shape[0]
        if A.shape != (n, n) or B.shape != (n, n):
            raise ValueError("A and B must be square and of equal size")
        if C is None:
            C = np.empty((n, n), np.float64)
        self._raise(self._lib.mm_gemm_host(self._h, n, A.ctypes.data, B.ctypes.data, C.ctypes.data,
                                           _stream_ptr(stream)))
        return C

    def gemm_grouped_host(self, As, Bs, Cs=None, stream=None):
        """mm_gemm_grouped_host: uneven products on host matrices (numpy arrays or
        CPU tensors, best pinned); copies overlap the computation.  Returns Cs."""
        import numpy as np
        def ptr(x):
            return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        def n_of(x):
            if len(x.shape) != 2 or x.shape[0] != x.shape[1]:
                raise ValueError("matrices must be square")
            return int(x.shape[0])
        for x in list(As) + list(Bs):
            if hasattr(x, "is_cuda") and x.is_cuda:
                raise TypeError("gemm_grouped_host takes host matrices")
            if hasattr(x, "dtype") and str(x.dtype) not in ("float64", "torch.float64"):
                raise TypeError("matrices must be float64")
        count = len(As)
        Ns = [n_of(a) for a in As]
        if Cs is None:
            Cs = [np.empty((n, n), np.float64) for n in Ns]
        arr_n = (ctypes.c_int * count)(*Ns)
        arr_a = (ctypes.c_void_p * count)(*[ptr(a) for a in As])
        arr_b = (ctypes.c_void_p * count)(*[ptr(b) for b in Bs])
        arr_c = (ctypes.c_void_p * count)(*[ptr(c) for c in Cs])
        self._raise(self._lib.mm_gemm_grouped_host(self._h, count, arr_n, arr_a, arr_b, arr_c, _stream_ptr(stream)))
        return Cs

    def gemm_host_ptr(self, n: int, a_ptr: int, b_ptr: int, c_ptr: int, stream=None):
        """mm_gemm_host on raw host pointers (e.g. pinned torch tensors)."""
        self._raise(self._lib.mm_gemm_host(self._h, n, a_ptr, b_ptr, c_ptr, _stream_ptr(stream)))

    def check(self, stream=None):
        """Synchronises and raises MMError for any device-side error."""
        self._raise(self._lib.mm_status_get(self._h, _stream_ptr(stream)))

    def guard_read(self, stream=None) -> tuple[int, int]:
        """mm_guard_read: (elements, whole problems) the accuracy certificate
        sent to native FP64 since the last read (synchronises)."""
        e, p = ctypes.c_longlong(), ctypes.c_longlong()
        self._raise(self._lib.mm_guard_read(self._h, _stream_ptr(stream), ctypes.byref(e), ctypes.byref(p)))
        return e.value, p.value

    def profile(self) -> dict:
        """Per-kernel-kind device time (ms) and launch counts of the last call (MM_FLAG_PROFILE)."""
        ms = (ctypes.c_double * len(KERNEL_KINDS))()
        n = (ctypes.c_int * len(KERNEL_KINDS))()
        self._raise(self._lib.mm_profile_read(self._h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def probe_fp64_peak(self) -> tuple[float, float]:
        """Measured FP64 roof of this GPU: (DMMA TFLOP/s, DFMA TFLOP/s)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._raise(self._lib.mm_probe_fp64_peak(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def probe_int8_peak(self) -> float:
        """Measured 8-bit integer mma.sync roof of this GPU, tera-operations per second."""
        a = ctypes.c_double()
        self._raise(self._lib.mm_probe_int8_peak(self._h, ctypes.byref(a)))
        return a.value

    def selftest_wait(self, timeout_ms: int = 200, stream=None):
        """Enqueues the bounded-wait self-test (see mm_selftest_wait)."""
        self._raise(self._lib.mm_selftest_wait(self._h, int(timeout_ms), _stream_ptr(stream)))

    def plan(self, n: int) -> tuple[int, int]:
        form, s = ctypes.c_int(), ctypes.c_int()
        self._raise(self._lib.mm_plan(self._h, n, ctypes.byref(form), ctypes.byref(s)))
        return form.value, s.value

    # -- steps of the emulation ------------------------------------------------
    def split(self, M, by_columns: bool, slices: int, rows: int | None = None, ld: int | None = None, stream=None):
        """Exponents (int32 [N]) and digit planes (int16 view of bf16, [s][rows][ld])."""
        import torch
        _check_tensor(M, "M")
        n = M.shape[0]
        rows = rows or -(-n // 128) * 128
        ld = ld or -(-n // 64) * 64
        exps = torch.empty(n, dtype=torch.int32, device=M.device)
        digits = torch.empty((slices, rows, ld), dtype=torch.int16, device=M.device)
        self._raise(self._lib.mm_split(self._h, n, M.data_ptr(), int(bool(by_columns)), slices, exps.data_ptr(),
                                       digits.data_ptr(), rows, ld, _stream_ptr(stream)))
        return exps, digits

    def level_sums(self, n: int, slices: int, a_digits, b_digits, stream=None):
        import torch
        s, a_rows, ld = a_digits.shape
        _, b_rows, ld2 = b_digits.shape
        if ld != ld2 or s != slices or b_digits.shape[0] != slices:
            raise ValueError("digit planes disagree")
        levels = torch.empty((slices, n, n), dtype=torch.int32, device=a_digits.device)
        self._raise(self._lib.mm_level_sums(self._h, n, slices, a_digits.data_ptr(), a_rows, b_digits.data_ptr(),
                                            b_rows, ld, levels.data_ptr(), _stream_ptr(stream)))
        return levels

    def recombine(self, n: int, slices: int, levels, a_exps, b_exps, stream=None):
        import torch
        C = torch.empty((n, n), dtype=torch.float64, device=levels.device)
        self._raise(self._lib.mm_recombine(self._h, n, slices, levels.data_ptr(), a_exps.data_ptr(),
                                           b_exps.data_ptr(), C.data_ptr(), _stream_ptr(stream)))
        return C
