"""The C-ABI library builds, loads without a GPU and exports every declared symbol.

No compute call is made here; only argument checks that return before any
CUDA work.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1012_2273_gb300 as mm
from paper_1012_2273_gb300 import build as mmbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mm.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mm_status|const char\*)\s+(mm_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("mm_create", "mm_gemm", "mm_gemm_grouped", "mm_destroy", "mm_status_get", "mm_last_error"):
        assert name in syms
    assert set(syms) == set(mm.SYMBOLS)


def test_library_exports_every_declared_symbol():
    path = mmbuild.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mm_\w+)$", out, re.M))
    missing = set(declared_symbols()) - exported
    assert not missing, missing
    L = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(L, name)


def test_argument_checks_without_gpu():
    L = mm.lib()
    assert L.mm_create(None, None) == 1  # MM_ERR_INVALID
    assert L.mm_gemm(None, 10, None, None, None, None) == 1
    assert L.mm_destroy(None) == 1
    assert L.mm_last_error(None) == b"invalid handle"
    assert L.mm_gemm_grouped(None, 1, None, None, None, None, None) == 1
    assert L.mm_gemm_ex(None, 0, 0, 4, 4, 4, None, 4, None, 4, None, 4, None) == 1
    assert L.mm_gemm_grouped_ex(None, 1, None, None, None, None, None, None, None, None, None, None, None,
                                None) == 1


@pytest.mark.parametrize("shape,strides,trans_ok,want", [
    ((5, 7), (7, 1), False, (5, 7, 7, 0)),       # contiguous
    ((5, 7), (10, 1), False, (5, 7, 10, 0)),     # window of a wider array
    ((5, 7), (1, 5), True, (5, 7, 5, 1)),        # X.T of a contiguous 7 x 5 X
    ((5, 7), (1, 9), True, (5, 7, 9, 1)),        # X.T of a window
    ((1, 7), (3, 1), False, (1, 7, 7, 0)),       # one row: its stride is irrelevant
    ((5, 1), (1, 1), False, (5, 1, 1, 0)),       # one column: row-major with ld 1
    ((5, 0), (0, 1), False, (5, 0, 1, 0)),       # empty rows: ld clamped to 1
    ((0, 4), (4, 1), False, (0, 4, 4, 0)),
])
def test_binding_layout_rule(shape, strides, trans_ok, want):
    assert mm._layout(shape[0], shape[1], strides[0], strides[1], trans_ok) == want


@pytest.mark.parametrize("shape,strides,trans_ok", [
    ((5, 7), (1, 5), False),   # transposed where only row-major is accepted (C)
    ((5, 7), (7, 2), True),    # neither unit column nor unit row stride
    ((5, 7), (6, 1), False),   # row stride below the row length
    ((5, 7), (1, 4), True),    # transposed, column stride below the column length
])
def test_binding_layout_rule_rejects(shape, strides, trans_ok):
    with pytest.raises(ValueError):
        mm._layout(shape[0], shape[1], strides[0], strides[1], trans_ok)


def test_header_cites_the_paper_and_states_conventions():
    text = open(HEADER).read()
    assert "Alg. 1" in text and "Sec. 3.1" in text
    assert "row-major" in text and "16-byte" in text and "owned by the caller" in text


def test_sources_have_no_cpu_fallback_or_oracle_use():
    pkg = os.path.join(ROOT, "paper_1012_2273_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.c" not in src, f


@pytest.mark.parametrize("flag", ["-gencode", "arch=compute_103a,code=sm_103a"])
def test_build_targets_sm103a_only(flag):
    assert flag in mmbuild.NVCC_FLAGS


def test_tune_file_is_validated_before_any_device_work(tmp_path):
    bad = tmp_path / "bad.txt"
    bad.write_text("1000 1 9 256\n")  # 9 slices: out of range
    L = mm.lib()
    cfg = mm._Config(mm.AUTO, 0, 0, str(bad).encode())
    h = ctypes.c_void_p()
    assert L.mm_create(ctypes.byref(h), ctypes.byref(cfg)) == 1  # MM_ERR_INVALID
    bad.write_text("1000 1 7 192\n")  # tile width must be 128 or 256
    assert L.mm_create(ctypes.byref(h), ctypes.byref(cfg)) == 1
    missing = mm._Config(mm.AUTO, 0, 0, str(tmp_path / "none.txt").encode())
    assert L.mm_create(ctypes.byref(h), ctypes.byref(missing)) == 1
    bad.write_text("1000 2 17 256\n")  # modular form: at most 16 moduli
    assert L.mm_create(ctypes.byref(h), ctypes.byref(cfg)) == 1
    bad.write_text("1000 2 1 256\n")  # and at least 2
    assert L.mm_create(ctypes.byref(h), ctypes.byref(cfg)) == 1


def test_modular_width_rule_matches_the_oracle_statement():
    # Host-side planning of the modular form (no GPU): the fixed-point width
    # and the moduli agree with the oracle's own, independent statement.
    import oracle
    for k in range(1, 17):
        for n in (1, 2, 10, 100, 255, 256, 500, 1000, 2000, 4095, 4096, 8192, 16384, 32767, 65535):
            beta, mods = mm.modular_params(k, n)
            assert beta == oracle.modular_beta(k, n), (k, n)
            assert mods == oracle.MODULI[:k]
    with pytest.raises(mm.MMError):
        mm.modular_params(17, 100)
    with pytest.raises(mm.MMError):
        mm.modular_params(4, 0)
