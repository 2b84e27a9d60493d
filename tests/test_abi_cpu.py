"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/genp.h declares.  No GPU needed: only host-side
argument checks are exercised (they return before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1212_4560_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "genp.h")).read()
    return sorted(set(re.findall(r"GENP_API[^;(]*?\b(genp_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1212_4560_gb300 import _lib
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.genp_version()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.genp_status_string(code).startswith(b"GENP_")


def test_argument_errors_return_before_any_cuda_call(lib):
    out = ctypes.c_void_p()
    ARG = -1
    assert lib.genp_make_multiplier(0, 0, 1, 0, 1.0, 4, 0, None, ctypes.byref(out)) == ARG      # n = 0
    assert lib.genp_make_multiplier(9, 8, 1, 0, 1.0, 4, 0, None, ctypes.byref(out)) == ARG      # bad kind
    assert lib.genp_make_multiplier(0, 8, 1, 0, -1.0, 4, 0, None, ctypes.byref(out)) == ARG     # bad scale
    assert lib.genp_make_multiplier(2, 8, 1, 0, 1.0, 0, 0, None, ctypes.byref(out)) == ARG      # nnz = 0
    assert lib.genp_make_multiplier(0, 8, 1, 0, 1.0, 4, 0, None, None) == ARG                   # no out
    assert lib.genp_factor(None, 8, 8, 0, 0, None, ctypes.byref(out)) == ARG                    # no C
    fake = ctypes.c_void_p(0x1000)
    assert lib.genp_factor(fake, 8, 4, 0, 0, None, ctypes.byref(out)) == ARG                    # ldc < n
    assert lib.genp_factor(fake, 8, 8, 0, 500, None, ctypes.byref(out)) == ARG                  # nb too big
    assert lib.genp_factor(fake, 8, 4, 3, 0, None, ctypes.byref(out)) == ARG                    # FP8, ldc < n
    assert lib.genp_factor(fake, 8, 8, 9, 0, None, ctypes.byref(out)) == ARG                    # bad precision
    buf = ctypes.c_void_p(0x2000)
    assert lib.genp_quantize_e4m3(fake, 8, 2, 8, 8, 0, buf, 16, buf, None) == ARG   # BF16 source
    assert lib.genp_quantize_e4m3(fake, 8, 0, 8, 8, 0, buf, 8, buf, None) == ARG    # ldq not a multiple of 16
    assert lib.genp_quantize_e4m3(fake, 4, 0, 8, 8, 0, buf, 16, buf, None) == ARG   # lds < K
    assert lib.genp_quantize_e4m3(fake, 4, 1, 8, 2, 1, buf, 16, buf, None) == ARG   # transposed: lds < m
    assert lib.genp_gemm_e4m3(8, 8, 8, ctypes.c_float(1.0), buf, 8, buf, buf, 16, buf, ctypes.c_float(0.0),
                              None, 0, buf, 8, None) == ARG                           # lda not a multiple of 16
    assert lib.genp_gemm_e4m3(8, 8, 8, ctypes.c_float(1.0), buf, 16, buf, buf, 16, buf, ctypes.c_float(1.0),
                              None, 0, buf, 8, None) == ARG                           # beta != 0 without Cin
    assert lib.genp_solve(None, None, None, 1, 1, None, 1, None) == ARG
    assert lib.genp_refine(None, 1, None, None, None, 1, 1, None, 1, 1e-15, 3, 0, None) == ARG
    assert lib.genp_adjoint(None, None, None, 1, None, 1, 1, None, 1, None, 1, None) == ARG
    assert lib.genp_precondition(None, None, 1, 0, None, 1, 0, None) == ARG
    assert lib.genp_info_fetch(None, None, None) == ARG
    assert lib.genp_multiplier_query(None, None, None, None) == ARG
    assert lib.genp_block_factor(None, 8, 8, 64, None, ctypes.byref(out)) == ARG            # no C
    assert lib.genp_block_factor(fake, 8, 4, 64, None, ctypes.byref(out)) == ARG            # ldc < n
    assert lib.genp_block_factor(fake, 8, 8, 32, None, ctypes.byref(out)) == -7             # order 64 only
    assert lib.genp_block_factor(fake, 8, 8, 64, None, None) == ARG                         # no out
    d, w, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    assert lib.genp_profile_class(6, ctypes.byref(d), ctypes.byref(w), ctypes.byref(c)) == ARG   # no such class
    assert lib.genp_profile_class(-1, ctypes.byref(d), ctypes.byref(w), ctypes.byref(c)) == ARG
    assert lib.genp_profile_class(1, None, ctypes.byref(w), ctypes.byref(c)) == ARG
    lib.genp_multiplier_destroy(None)
    lib.genp_factors_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1212_4560_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
