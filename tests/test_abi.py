"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/hpmdr.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hpmdr.h")).read()
    return sorted(set(re.findall(r"HPMDR_API\s+[\w\s\*]*?\b(hpmdr_\w+)\s*\(", text)))


def test_header_declares_api():
    names = _declared()
    assert "hpmdr_refactor" in names and "hpmdr_retrieve" in names and len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_2505_00227_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2505_00227_gb300 import binding
    assert sorted(binding.exported_symbols()) == _declared()


def test_strerror_without_gpu():
    from paper_2505_00227_gb300 import binding
    L = binding.lib()
    assert L.hpmdr_strerror(-5) == b"error bound unattainable"
    assert L.hpmdr_strerror(0) == b"ok"


def test_ctx_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2505_00227_gb300 import binding
    p = ctypes.c_void_p()
    st = binding.lib().hpmdr_ctx_create(ctypes.byref(p), None, None, None)
    assert st == binding.ERR_CUDA and not p.value
